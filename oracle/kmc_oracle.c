/*
 * kmc_oracle.c -- plain, slow, FP64 CPU oracle for the periodic Coulomb
 * energy change of a single-charge hop and for the rejection-free KMC step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (the definition the FMM-for-KMC method approximates):
 *
 *   U = 1/2 sum_i sum_j sum'_{n in Z^3} q_i q_j / |r_i - r_j + n a|
 *
 * for a neutral cubic cell of edge a with conducting ("tinfoil") boundary
 * at infinity (n = 0 omitted when i = j).  The paper fixes the boundary in
 * Sec. 2.2.2 and App. B by adding the field that cancels the surface charge
 * at infinity; on a cubic summation order that is exactly the tinfoil Ewald
 * energy.  The pair potential is evaluated by Ewald splitting:
 *
 *   psi(d) = sum_n erfc(beta|d+na|)/|d+na|
 *          + (4 pi / V) sum_{k != 0} exp(-k^2/(4 beta^2)) / k^2 cos(k.d)
 *          - pi / (beta^2 V),                         k = 2 pi m / a,
 *
 *   psi_reg(0) = lim_{d->0} (psi(d) - 1/|d|)
 *              = same sums at d = 0 with the n = 0 real term replaced by
 *                -2 beta / sqrt(pi).
 *
 * The hop of charge k from r to r' changes the energy by (Sec. 3, Eq. for
 * the proposed energy; its periodic form, Sec. 3.1)
 *
 *   dU = q_k [ phi_{-k}(r') - phi_{-k}(r) ],  phi_{-k}(x) = sum_{j!=k} q_j psi(x - r_j)
 *
 * which equals U(after) - U(before) because the self-image energy
 * q_k^2 psi_reg(0) / 2 does not depend on the position.
 *
 * KMC step (Algorithm 1): rates, a sequential FP64 cumulative sum in the
 * canonical event order, selection of j with R_{j-1} < Q zeta <= R_j, and
 * dt = -ln(xi)/Q.
 *
 * Lattice mode: sites are the integer points of an E^3 periodic grid with
 * spacing 1 (a = E).  All displacements between sites are integer vectors,
 * so psi is tabulated once on the E^3 displacement grid (G[d] = psi(d),
 * G[0] = psi_reg(0)), and a site potential phi_s = sum_j q_j G[s - s_j] is
 * maintained; dU then follows from the definition in O(1) per hop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Ewald pair potential                                                */
/* ------------------------------------------------------------------ */

/* Number of reciprocal shells needed so that the first omitted term is
 * below about 1e-17 of the leading one: pi^2 (K+1)^2 / (beta a)^2 > 39.1. */
int oracle_default_kmax(double beta_a) {
  return (int)ceil(2.0 * beta_a);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double wrap_min_image(double x, double a) {
  /* reduce to [-a/2, a/2) */
  double y = x - a * floor(x / a + 0.5);
  return y;
}

/* Real-space part: images |n|_inf <= nreal around the minimum image of d.
 * If exclude_origin, the n = 0 term is left out (used for psi_reg(0)). */
static double psi_real(double a, double beta, int nreal, const double d[3], int exclude_origin) {
  double s = 0.0;
  for (int nx = -nreal; nx <= nreal; nx++)
    for (int ny = -nreal; ny <= nreal; ny++)
      for (int nz = -nreal; nz <= nreal; nz++) {
        if (exclude_origin && nx == 0 && ny == 0 && nz == 0) continue;
        double x = d[0] + nx * a, y = d[1] + ny * a, z = d[2] + nz * a;
        double r = sqrt(x * x + y * y + z * z);
        s += erfc(beta * r) / r;
      }
  return s;
}

/* Reciprocal part: (4 pi / V) sum_{m != 0, |m|_inf <= kmax} exp(-k^2/4b^2)/k^2 cos(k.d) */
static double psi_recip(double a, double beta, int kmax, const double d[3]) {
  double V = a * a * a;
  double s = 0.0;
  for (int mx = -kmax; mx <= kmax; mx++)
    for (int my = -kmax; my <= kmax; my++)
      for (int mz = -kmax; mz <= kmax; mz++) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        double kx = 2.0 * PI * mx / a, ky = 2.0 * PI * my / a, kz = 2.0 * PI * mz / a;
        double k2 = kx * kx + ky * ky + kz * kz;
        s += exp(-k2 / (4.0 * beta * beta)) / k2 * cos(kx * d[0] + ky * d[1] + kz * d[2]);
      }
  return 4.0 * PI / V * s;
}

/* psi(d) for d != 0 (mod a).  beta in 1/length; nreal image shells. */
double oracle_psi(double a, double beta, int nreal, int kmax, double dx, double dy, double dz) {
  double d[3] = {wrap_min_image(dx, a), wrap_min_image(dy, a), wrap_min_image(dz, a)};
  double V = a * a * a;
  return psi_real(a, beta, nreal, d, 0) + psi_recip(a, beta, kmax, d) - PI / (beta * beta * V);
}

double oracle_psi_reg0(double a, double beta, int nreal, int kmax) {
  double d[3] = {0.0, 0.0, 0.0};
  double V = a * a * a;
  return psi_real(a, beta, nreal, d, 1) - 2.0 * beta / sqrt(PI) + psi_recip(a, beta, kmax, d) -
         PI / (beta * beta * V);
}

/* ------------------------------------------------------------------ */
/* Direct (off-lattice) energy and hop energy change                   */
/* ------------------------------------------------------------------ */

/* U = 1/2 sum_{i != j} q_i q_j psi(r_i - r_j) + 1/2 sum_i q_i^2 psi_reg(0). O(N^2) psi calls. */
double oracle_energy(int64_t n, const double* pos, const double* q, double a, double beta, int nreal,
                     int kmax) {
  double p0 = oracle_psi_reg0(a, beta, nreal, kmax);
  double U = 0.0;
#pragma omp parallel for reduction(+ : U) schedule(dynamic, 1)
  for (int64_t i = 0; i < n; i++) {
    double ui = 0.5 * q[i] * q[i] * p0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      ui += 0.5 * q[i] * q[j] *
            oracle_psi(a, beta, nreal, kmax, pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                       pos[3 * i + 2] - pos[3 * j + 2]);
    }
    U += ui;
  }
  return U;
}

/* dU for moving charge k from pos[k] to target: q_k sum_{j != k} q_j [psi(r'-r_j) - psi(r-r_j)].
 * A target that coincides with another charge's position is singular; the caller masks it. */
double oracle_delta_u(int64_t n, const double* pos, const double* q, double a, double beta, int nreal,
                      int kmax, int64_t k, const double target[3]) {
  double s = 0.0;
  for (int64_t j = 0; j < n; j++) {
    if (j == k) continue;
    double pn = oracle_psi(a, beta, nreal, kmax, target[0] - pos[3 * j], target[1] - pos[3 * j + 1],
                           target[2] - pos[3 * j + 2]);
    double po = oracle_psi(a, beta, nreal, kmax, pos[3 * k] - pos[3 * j], pos[3 * k + 1] - pos[3 * j + 1],
                           pos[3 * k + 2] - pos[3 * j + 2]);
    s += q[j] * (pn - po);
  }
  return q[k] * s;
}

/* Many proposals at once (parallel over proposals). */
void oracle_delta_u_many(int64_t n, const double* pos, const double* q, double a, double beta, int nreal,
                         int kmax, int64_t m, const int64_t* particle, const double* target, double* dU) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < m; t++)
    dU[t] = oracle_delta_u(n, pos, q, a, beta, nreal, kmax, particle[t], target + 3 * t);
}

/* ------------------------------------------------------------------ */
/* Lattice mode                                                        */
/* ------------------------------------------------------------------ */

static inline int64_t site_index(int64_t E, int64_t x, int64_t y, int64_t z) {
  return x + E * (y + E * z);
}

/* G[d] = psi(d) for every integer displacement d in [0,E)^3 (lattice spacing 1,
 * box a = E), G[0] = psi_reg(0).  The reciprocal sum is written with the
 * even symmetry of its coefficients: the sine parts cancel between m and -m,
 * leaving sum_m c(|m|) cos(2pi mx dx/E) cos(2pi my dy/E) cos(2pi mz dz/E),
 * folded onto m_i >= 0 with a weight 2 per non-zero component.  psi is
 * even in each component, so only 0 <= d_i <= E/2 is computed and mirrored. */
void oracle_psi_table(int64_t E, double beta, int nreal, int kmax, double* G) {
  double a = (double)E, V = a * a * a;
  int64_t H = E / 2;
  int K = kmax;
  /* coefficients on the folded grid */
  double* c = (double*)malloc(sizeof(double) * (K + 1) * (K + 1) * (K + 1));
  for (int mx = 0; mx <= K; mx++)
    for (int my = 0; my <= K; my++)
      for (int mz = 0; mz <= K; mz++) {
        double v = 0.0;
        if (mx || my || mz) {
          double k2 = (2.0 * PI / a) * (2.0 * PI / a) * (double)(mx * mx + my * my + mz * mz);
          double w = (mx ? 2.0 : 1.0) * (my ? 2.0 : 1.0) * (mz ? 2.0 : 1.0);
          v = w * 4.0 * PI / V * exp(-k2 / (4.0 * beta * beta)) / k2;
        }
        c[(mx * (K + 1) + my) * (K + 1) + mz] = v;
      }
  double p0 = oracle_psi_reg0(a, beta, nreal, kmax);
  double cst = PI / (beta * beta * V);
#pragma omp parallel
  {
    double* cx = (double*)malloc(sizeof(double) * (K + 1));
    double* cy = (double*)malloc(sizeof(double) * (K + 1));
    double* cz = (double*)malloc(sizeof(double) * (K + 1));
#pragma omp for schedule(dynamic, 1) collapse(2)
    for (int64_t dz = 0; dz <= H; dz++)
      for (int64_t dy = 0; dy <= H; dy++) {
        for (int m = 0; m <= K; m++) {
          cy[m] = cos(2.0 * PI * m * (double)dy / a);
          cz[m] = cos(2.0 * PI * m * (double)dz / a);
        }
        for (int64_t dx = 0; dx <= H; dx++) {
          double val;
          if (dx == 0 && dy == 0 && dz == 0) {
            val = p0;
          } else {
            for (int m = 0; m <= K; m++) cx[m] = cos(2.0 * PI * m * (double)dx / a);
            double rec = 0.0;
            for (int mx = 0; mx <= K; mx++)
              for (int my = 0; my <= K; my++) {
                double cxy = cx[mx] * cy[my];
                const double* cc = c + (mx * (K + 1) + my) * (K + 1);
                for (int mz = 0; mz <= K; mz++) rec += cc[mz] * cxy * cz[mz];
              }
            double d[3] = {(double)dx, (double)dy, (double)dz};
            val = psi_real(a, beta, nreal, d, 0) + rec - cst;
          }
          /* mirror into all sign combinations */
          for (int sx = 0; sx < 2; sx++)
            for (int sy = 0; sy < 2; sy++)
              for (int sz = 0; sz < 2; sz++) {
                int64_t x = sx ? (E - dx) % E : dx;
                int64_t y = sy ? (E - dy) % E : dy;
                int64_t z = sz ? (E - dz) % E : dz;
                G[site_index(E, x, y, z)] = val;
              }
        }
      }
    free(cx);
    free(cy);
    free(cz);
  }
  free(c);
}

static inline int64_t disp_index(int64_t E, int64_t s, int64_t t) {
  /* index of the displacement s - t (mod E) for linear site indices s, t */
  int64_t sx = s % E, sy = (s / E) % E, sz = s / (E * E);
  int64_t tx = t % E, ty = (t / E) % E, tz = t / (E * E);
  int64_t dx = (sx - tx + E) % E, dy = (sy - ty + E) % E, dz = (sz - tz + E) % E;
  return site_index(E, dx, dy, dz);
}

/* phi_s = sum_j q_j G[s - s_j] for every site s, directly (O(E^3 N)). */
void oracle_site_potential(int64_t E, const double* G, int64_t n, const int64_t* site, const double* q,
                           double* phi) {
  int64_t S = E * E * E;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < S; s++) {
    double v = 0.0;
    for (int64_t j = 0; j < n; j++) v += q[j] * G[disp_index(E, s, site[j])];
    phi[s] = v;
  }
}

/* After charge q moves from site s_old to s_new: phi_s += q (G[s - s_new] - G[s - s_old]). */
void oracle_site_update(int64_t E, const double* G, double* phi, int64_t s_old, int64_t s_new, double q) {
  int64_t S = E * E * E;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < S; s++) phi[s] += q * (G[disp_index(E, s, s_new)] - G[disp_index(E, s, s_old)]);
}

/* Lattice hop sets (the moves every charge proposes, Algorithm 5 and the
 * benchmark of Sec. 5.3): hops 0..5 go to the six face neighbours in the
 * order +x, -x, +y, -y, +z, -z; hops 6..13 (the 14-hop set of Sec. 5.3) go
 * to the eight body-diagonal neighbours at distance sqrt(3), listed with the
 * x component varying fastest and + before -.  Targets wrap periodically. */
static const int HOP_VEC[14][3] = {
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 1},   {-1, 1, 1},  {1, -1, 1}, {-1, -1, 1},
    {1, 1, -1},  {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

static int64_t hop_target(int64_t E, int64_t s, int k) {
  int64_t x = s % E, y = (s / E) % E, z = s / (E * E);
  x = (x + HOP_VEC[k][0] + E) % E;
  y = (y + HOP_VEC[k][1] + E) % E;
  z = (z + HOP_VEC[k][2] + E) % E;
  return site_index(E, x, y, z);
}

/* Target site of every hop of every charge, out[nhop i + k] (nhop = 6 or 14). */
void oracle_hop_targets(int64_t E, int64_t n, const int64_t* site, int nhop, int64_t* out) {
  for (int64_t i = 0; i < n; i++)
    for (int k = 0; k < nhop; k++) out[(int64_t)nhop * i + k] = hop_target(E, site[i], k);
}

/* Hop vector k (integer lattice offsets). */
void oracle_hop_vector(int k, int64_t* v) {
  for (int a = 0; a < 3; a++) v[a] = HOP_VEC[k][a];
}

int64_t oracle_hop_target(int64_t E, int64_t s, int k) { return hop_target(E, s, k); }

/* dU for every charge i and hop k in (+x,-x,+y,-y,+z,-z):
 *   dU = q_i [ (phi_{s'} - q_i G[s' - s_i]) - (phi_{s_i} - q_i G[0]) ]
 * i.e. the definition with the moving charge's own contribution removed
 * from the site potential.  Hops onto occupied sites are masked (mask 0,
 * dU = NaN).  occ[s] = 1 if site s is occupied. */
void oracle_lattice_delta_u(int64_t E, const double* G, const double* phi, int64_t n, const int64_t* site,
                            const double* q, const uint8_t* occ, double* dU, uint8_t* mask) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    int64_t s = site[i];
    for (int k = 0; k < 6; k++) {
      int64_t t = hop_target(E, s, k);
      if (occ[t]) {
        mask[6 * i + k] = 0;
        dU[6 * i + k] = NAN;
      } else {
        mask[6 * i + k] = 1;
        dU[6 * i + k] = q[i] * ((phi[t] - q[i] * G[disp_index(E, t, s)]) - (phi[s] - q[i] * G[0]));
      }
    }
  }
}

/* dU for an explicit list of (particle, target site) proposals on the lattice. */
void oracle_lattice_delta_u_list(int64_t E, const double* G, const double* phi, const int64_t* site,
                                 const double* q, int64_t m, const int64_t* particle, const int64_t* target,
                                 double* dU) {
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < m; t++) {
    int64_t i = particle[t], s = site[i], u = target[t];
    dU[t] = q[i] * ((phi[u] - q[i] * G[disp_index(E, u, s)]) - (phi[s] - q[i] * G[0]));
  }
}

/* ------------------------------------------------------------------ */
/* KMC step (Algorithm 1)                                              */
/* ------------------------------------------------------------------ */

/* rate = exp(-max(dU,0)/kT) for unmasked entries, 0 for masked ones. */
void oracle_rates(int64_t m, const double* dU, const uint8_t* mask, double kT, double* rate) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < m; j++) {
    if (mask && !mask[j]) {
      rate[j] = 0.0;
    } else {
      double x = dU[j] > 0.0 ? dU[j] : 0.0;
      rate[j] = exp(-x / kT);
    }
  }
}

/* Sequential inclusive cumulative sum R_j in event order; Q = R_{m-1};
 * returns the j with R_{j-1} < Q zeta <= R_j (R_{-1} = 0), or -1 if Q == 0.
 * Also returns dt = -ln(xi)/Q. */
int64_t oracle_select(int64_t m, const double* rate, double zeta, double xi, double* Q_out, double* dt_out) {
  double R = 0.0;
  for (int64_t j = 0; j < m; j++) R += rate[j];
  double Q = R;
  if (Q_out) *Q_out = Q;
  if (dt_out) *dt_out = (Q > 0.0) ? -log(xi) / Q : INFINITY;
  if (!(Q > 0.0)) return -1;
  double target = Q * zeta;
  double prev = 0.0;
  R = 0.0;
  for (int64_t j = 0; j < m; j++) {
    R += rate[j];
    if (prev < target && target <= R) return j;
    prev = R;
  }
  /* Q*zeta can exceed the final R only by rounding when zeta == 1 */
  for (int64_t j = m - 1; j >= 0; j--)
    if (rate[j] > 0.0) return j;
  return -1;
}

/* Inclusive cumulative sum (for near-tie analysis in tests). */
void oracle_cumsum(int64_t m, const double* rate, double* R) {
  double s = 0.0;
  for (int64_t j = 0; j < m; j++) {
    s += rate[j];
    R[j] = s;
  }
}

/* dU for (particle[t], target site[t]) by the direct O(N) sum over the other
 * charges with the tabulated pair potential:
 *   dU = q_i sum_{j != i} q_j [G(s' - s_j) - G(s_i - s_j)]                  */
void oracle_lattice_delta_u_direct(int64_t E, const double* G, int64_t n, const int64_t* site, const double* q,
                                   int64_t m, const int64_t* particle, const int64_t* target, double* dU) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < m; t++) {
    int64_t i = particle[t], si = site[i], u = target[t];
    double s = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      s += q[j] * (G[disp_index(E, u, site[j])] - G[disp_index(E, si, site[j])]);
    }
    dU[t] = q[i] * s;
  }
}
