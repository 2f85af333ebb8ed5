// fmm_kernels.cu -- one-off full FMM on the device (Algorithm 2 with the
// periodic modifications of Sec. 3.1), the lattice-sum far field (Sec. 2.2.1)
// and the per-step downward pass that materialises leaf local expansions.
//
// Local expansions are stored per level: Psi_l[b] holds only the M2L
// contributions of the interaction list of cell b on level l (Algorithm 2,
// inner loop), and level 1 holds the far-field expansion H = R K.  Because a
// local-to-local translation of a degree-p expansion is exact, the leaf
// expansion of Algorithm 2 equals sum_l L2L(Psi_l[ancestor_l] -> leaf); the
// downward kernel rebuilds it each step.  Storing the levels separately is
// the per-level scheme of Sec. 6 (conclusions) and makes an accepted move
// touch O(L) cells per level instead of every leaf.
#include <math.h>
#include <stdio.h>

#include <cuda_bf16.h>

#include "common.cuh"

__constant__ double f_inv_nm[KMC_NTRI];        // 1/((n-m)(n+m)), n > m
__constant__ double f_fact[4 * KMC_MAXP + 2];   // k! for k <= 4p + 1

void fmm_upload_constants(int p) {
  static double inv[KMC_NTRI];
  static double fact[4 * KMC_MAXP + 2];
  for (int n = 0; n <= 2 * KMC_MAXP; n++)
    for (int m = 0; m <= n; m++) inv[tri(n, m)] = (n > m) ? 1.0 / ((double)(n - m) * (double)(n + m)) : 0.0;
  fact[0] = 1.0;
  for (int k = 1; k < 4 * KMC_MAXP + 2; k++) fact[k] = fact[k - 1] * k;
  cudaMemcpyToSymbol(f_inv_nm, inv, sizeof(inv));
  cudaMemcpyToSymbol(f_fact, fact, sizeof(fact));
  void fmm_upload_nm();
  fmm_upload_nm();
  (void)p;
}

// ------------------------------------------------------------------ harmonics
// Full table of regular harmonics R_n^m(x), 0 <= m <= n <= p (FP64).
__device__ void regular_table(double x, double y, double z, int p, double2* out) {
  double r2 = x * x + y * y + z * z;
  double2 mm = make_double2(1.0, 0.0);
  for (int m = 0; m <= p; m++) {
    if (m > 0) {
      // R_m^m = -(x+iy)/(2m) R_{m-1}^{m-1}
      double s = -0.5 / m;
      double2 t = make_double2(s * (x * mm.x - y * mm.y), s * (x * mm.y + y * mm.x));
      mm = t;
    }
    out[tri(m, m)] = mm;
    double2 a2 = make_double2(0.0, 0.0), a1 = mm;
    for (int n = m + 1; n <= p; n++) {
      double c = f_inv_nm[tri(n, m)];
      double zz = (2 * n - 1) * z;
      double2 v = make_double2((zz * a1.x - r2 * a2.x) * c, (zz * a1.y - r2 * a2.y) * c);
      out[tri(n, m)] = v;
      a2 = a1;
      a1 = v;
    }
  }
}

// Column m of the same table, out[tri(n, m)] for n = m .. p (the same
// operations as regular_table, so the same values): p + 1 threads build a table.
__device__ void regular_column(double x, double y, double z, int p, int m, double2* out) {
  const double r2 = x * x + y * y + z * z;
  double2 mm = make_double2(1.0, 0.0);
  for (int j = 1; j <= m; j++) {
    const double s = -0.5 / j;
    mm = make_double2(s * (x * mm.x - y * mm.y), s * (x * mm.y + y * mm.x));
  }
  out[tri(m, m)] = mm;
  double2 a2 = make_double2(0.0, 0.0), a1 = mm;
  for (int n = m + 1; n <= p; n++) {
    const double c = f_inv_nm[tri(n, m)];
    const double zz = (2 * n - 1) * z;
    const double2 v = make_double2((zz * a1.x - r2 * a2.x) * c, (zz * a1.y - r2 * a2.y) * c);
    out[tri(n, m)] = v;
    a2 = a1;
    a1 = v;
  }
}

// Full table of irregular harmonics I_n^m(x), 0 <= m <= n <= p (FP64).
__device__ void irregular_table(double x, double y, double z, int p, double2* out, int64_t stride = 1) {
  double r2 = x * x + y * y + z * z;
  double inv = 1.0 / r2;
  double2 mm = make_double2(1.0 / sqrt(r2), 0.0);
  for (int m = 0; m <= p; m++) {
    if (m > 0) {
      double s = -(2.0 * m - 1.0) * inv;
      double2 t = make_double2(s * (x * mm.x - y * mm.y), s * (x * mm.y + y * mm.x));
      mm = t;
    }
    out[tri(m, m) * stride] = mm;
    double2 a2 = make_double2(0.0, 0.0), a1 = mm;
    for (int n = m + 1; n <= p; n++) {
      double zz = (2 * n - 1) * z;
      double c2 = (double)((n - 1) * (n - 1) - m * m);
      double2 v = make_double2((zz * a1.x - c2 * a2.x) * inv, (zz * a1.y - c2 * a2.y) * inv);
      out[tri(n, m) * stride] = v;
      a2 = a1;
      a1 = v;
    }
  }
}

// R_m^m(x) directly (m complex multiplications)
__device__ __forceinline__ double2 regular_mm(double x, double y, int m) {
  double2 mm = make_double2(1.0, 0.0);
  for (int j = 1; j <= m; j++) {
    double s = -0.5 / j;
    mm = make_double2(s * (x * mm.x - y * mm.y), s * (x * mm.y + y * mm.x));
  }
  return mm;
}

// ------------------------------------------------------------------ binning
__device__ __forceinline__ int leaf_of(const Geo& g, double x, double y, double z) {
  int cx = cell_at(x, g.nL, g.inv_a), cy = cell_at(y, g.nL, g.inv_a), cz = cell_at(z, g.nL, g.inv_a);
  return cx + g.nL * (cy + g.nL * cz);
}

__global__ void k_bin_count(const Geo g, const Dev d) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  int leaf = leaf_of(g, d.pos[3 * i], d.pos[3 * i + 1], d.pos[3 * i + 2]);
  int r = atomicAdd(&d.cnt[leaf], 1);
  if (r < g.cap) d.uid[(int64_t)leaf * g.cap + r] = (int32_t)i;
  else atomicOr(&d.err[0], KMC_DERR_CAPACITY);
}

// deterministic order inside each leaf: ascending user index
__global__ void k_bin_sort(const Geo g, const Dev d) {
  int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (leaf >= g.ML) return;
  int c = min(d.cnt[leaf], g.cap);
  int32_t* u = d.uid + leaf * g.cap;
  for (int a = 1; a < c; a++) {
    int32_t v = u[a];
    int b = a - 1;
    while (b >= 0 && u[b] > v) { u[b + 1] = u[b]; b--; }
    u[b + 1] = v;
  }
}

__global__ void k_bin_fill(const Geo g, const Dev d) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= g.ML * g.cap) return;
  int64_t leaf = s / g.cap;
  int j = (int)(s - leaf * g.cap);
  if (j >= d.cnt[leaf]) return;
  int32_t i = d.uid[s];
  d.slot_of[i] = (int32_t)s;
  double x = d.pos[3 * i], y = d.pos[3 * i + 1], z = d.pos[3 * i + 2], q = d.q[i];
  d.spos64[s] = make_double4_32a(x, y, z, q);
  d.spos32[s] = make_float4((float)x, (float)y, (float)z, (float)q);
}

void fmm_bin(const Geo& g, const Dev& d, cudaStream_t s) {
  cudaMemsetAsync(d.cnt, 0, sizeof(int32_t) * g.ML, s);
  k_bin_count<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g, d);
  k_bin_sort<<<(unsigned)((g.ML + 127) / 128), 128, 0, s>>>(g, d);
  int64_t ns = g.ML * g.cap;
  k_bin_fill<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ P2M
// thread per (leaf, m): Mt_n^m = sum_j q_j R_n^m(r_j - c) for n = m..p
__global__ void k_p2m(const Geo g, const Dev d) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t leaf = t / (g.p + 1);
  int m = (int)(t - leaf * (g.p + 1));
  if (leaf >= g.ML) return;
  int cx = (int)(leaf % g.nL), cy = (int)((leaf / g.nL) % g.nL), cz = (int)(leaf / ((int64_t)g.nL * g.nL));
  double c0 = (cx + 0.5) * g.w, c1 = (cy + 0.5) * g.w, c2 = (cz + 0.5) * g.w;
  double2 acc[KMC_MAXP + 1];
  for (int n = 0; n <= g.p; n++) acc[n] = make_double2(0.0, 0.0);
  int c = d.cnt[leaf];
  const double4_32a* sp = d.spos64 + leaf * g.cap;
  for (int j = 0; j < c; j++) {
    double4_32a v = sp[j];
    double x = v.x - c0, y = v.y - c1, z = v.z - c2, q = v.w;
    double r2 = x * x + y * y + z * z;
    double2 a1 = regular_mm(x, y, m), a2 = make_double2(0.0, 0.0);
    acc[m].x += q * a1.x;
    acc[m].y += q * a1.y;
    for (int n = m + 1; n <= g.p; n++) {
      double cc = f_inv_nm[tri(n, m)];
      double zz = (2 * n - 1) * z;
      double2 vv = make_double2((zz * a1.x - r2 * a2.x) * cc, (zz * a1.y - r2 * a2.y) * cc);
      acc[n].x += q * vv.x;
      acc[n].y += q * vv.y;
      a2 = a1;
      a1 = vv;
    }
  }
  double2* out = d.Mt + (g.cell_off[g.L] + leaf) * g.P;
  for (int n = m; n <= g.p; n++) out[tri(n, m)] = acc[n];
}

// The same P2M with the degree P known at compile time: one warp per leaf, lane
// m (m <= P) the column m.  The leaf's charges are loaded 32 at a time and
// broadcast by shuffles; per charge the lane forms the sectoral value
// R_m^m = prod_{j <= m} -(x + i y) / (2j) and the column's recurrence up to
// degree P (steps below m or beyond P predicated off), all P + 1 accumulators
// in registers.  T: the arithmetic of the recurrence and the sums (FP64; FP32
// in the mixed form, whose M2L keeps 29 bits); the expansion is stored in FP64.
template <int P, typename T>
__global__ void __launch_bounds__(128) k_p2m_w(const Geo g, const Dev d) {
  const int lane = threadIdx.x & 31, m = lane;
  const int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (leaf >= g.ML) return;  // whole warps
  const int cx = (int)(leaf % g.nL), cy = (int)((leaf / g.nL) % g.nL), cz = (int)(leaf / ((int64_t)g.nL * g.nL));
  const double c0 = (cx + 0.5) * g.w, c1 = (cy + 0.5) * g.w, c2 = (cz + 0.5) * g.w;
  T ax[P + 1], ay[P + 1], ci[P + 1];
#pragma unroll
  for (int n = 0; n <= P; n++) {
    ax[n] = ay[n] = (T)0;
    ci[n] = n > m ? (T)(1.0 / ((double)(n - m) * (double)(n + m))) : (T)0;
  }
  const int c = d.cnt[leaf];
  const double4_32a* sp = d.spos64 + leaf * g.cap;
  for (int j0 = 0; j0 < c; j0 += 32) {
    double4_32a v = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (j0 + lane < c) v = sp[j0 + lane];
    const int nj = min(32, c - j0);
    for (int jj = 0; jj < nj; jj++) {
      const T x = (T)(__shfl_sync(0xffffffffu, v.x, jj) - c0), y = (T)(__shfl_sync(0xffffffffu, v.y, jj) - c1);
      const T z = (T)(__shfl_sync(0xffffffffu, v.z, jj) - c2), q = (T)__shfl_sync(0xffffffffu, v.w, jj);
      T mx = (T)1, my = (T)0;
#pragma unroll
      for (int j = 1; j <= P; j++)
        if (j <= m) {
          const T sc = (T)(-0.5 / j);
          const T tx = sc * (x * mx - y * my), ty = sc * (x * my + y * mx);
          mx = tx;
          my = ty;
        }
      const T r2 = x * x + y * y + z * z;
      T a1x = mx, a1y = my, a2x = (T)0, a2y = (T)0;
#pragma unroll
      for (int n = 0; n <= P; n++) {
        if (n == m) {
          ax[n] += q * a1x;
          ay[n] += q * a1y;
        } else if (n > m) {
          const T zz = (T)(2 * n - 1) * z;
          const T vx = (zz * a1x - r2 * a2x) * ci[n], vy = (zz * a1y - r2 * a2y) * ci[n];
          ax[n] += q * vx;
          ay[n] += q * vy;
          a2x = a1x;
          a2y = a1y;
          a1x = vx;
          a1y = vy;
        }
      }
    }
  }
  if (m > P) return;
  double2* out = d.Mt + (g.cell_off[g.L] + leaf) * g.P;
#pragma unroll
  for (int n = 0; n <= P; n++)
    if (n >= m) out[tri(n, m)] = make_double2((double)ax[n], (double)ay[n]);
}

template <typename T>
static bool p2m_fixed(const Geo& g, const Dev& d, cudaStream_t s) {
  const unsigned nb = (unsigned)((g.ML * 32 + 127) / 128);
  switch (g.p) {
#define KMC_P2M_CASE(P) \
  case P: k_p2m_w<P, T><<<nb, 128, 0, s>>>(g, d); return true;
    KMC_P2M_CASE(4) KMC_P2M_CASE(6) KMC_P2M_CASE(8) KMC_P2M_CASE(10) KMC_P2M_CASE(12) KMC_P2M_CASE(14)
    KMC_P2M_CASE(16) KMC_P2M_CASE(18) KMC_P2M_CASE(20) KMC_P2M_CASE(22) KMC_P2M_CASE(24)
#undef KMC_P2M_CASE
    default: return false;
  }
}

void fmm_p2m(const Geo& g, const Dev& d, cudaStream_t s) {
  if (g.prec == 1 ? p2m_fixed<float>(g, d, s) : p2m_fixed<double>(g, d, s)) return;
  int64_t nt = g.ML * (g.p + 1);  // other degrees: one thread per (leaf, column)
  k_p2m<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ child offsets
// Rch[l][o] = R_n^m(c_child - c_parent) for the 8 child octants o of a level-l
// cell's parent: (o - 1/2) w_l per axis.  Used by M2M (level l-1 from l) and
// by the downward L2L (level l from l-1).  Computed once per handle.
__global__ void k_child_tables(const Geo g, const Dev d) {
  int l = 2 + blockIdx.x;
  int o = threadIdx.x;
  if (o >= 8 || l > g.L) return;
  double wc = g.a / (1 << (l - 1));
  double tx = ((o & 1) - 0.5) * wc, ty = (((o >> 1) & 1) - 0.5) * wc, tz = (((o >> 2) & 1) - 0.5) * wc;
  double2* out = d.Rch + ((int64_t)l * 8 + o) * g.P;
  regular_table(tx, ty, tz, g.p, out);
  if (d.Rch32)
    for (int c = 0; c < g.P; c++) d.Rch32[((int64_t)l * 8 + o) * g.P + c] = make_float2((float)out[c].x, (float)out[c].y);
}

// R(c_b - c_a) for every position of a cell b of level l (2 .. KMC_DOWN_COARSE) inside its
// ancestor a of level la: block = table, thread = column m
__global__ void k_coarse_tables(const Geo g, const Dev d) {
  int t = blockIdx.x, l = 2, la = 1;
  for (l = 2; l <= KMC_DOWN_COARSE; l++) {
    for (la = 1; la < l; la++) {
      const int nt = 1 << (3 * (l - la));
      if (t < coarse_table_base(l, la) + nt) goto found;
    }
  }
  return;
found:
  const int i = t - coarse_table_base(l, la), k = 1 << (l - la);  // position of b inside a, k per axis
  const double wl = g.a / (1 << (l - 1)), half = 0.5 * k;
  const double ox = ((i % k) + 0.5 - half) * wl, oy = (((i / k) % k) + 0.5 - half) * wl, oz = ((i / (k * k)) + 0.5 - half) * wl;
  double2* out = d.Rcoarse + (int64_t)t * g.P;
  if ((int)threadIdx.x <= g.p) regular_column(ox, oy, oz, g.p, threadIdx.x, out);
  __syncthreads();
  if (d.Rcoarse32)
    for (int c = threadIdx.x; c < g.P; c += blockDim.x) d.Rcoarse32[(int64_t)t * g.P + c] = make_float2((float)out[c].x, (float)out[c].y);
}

void fmm_child_tables(const Geo& g, const Dev& d, cudaStream_t s) {
  k_child_tables<<<g.L - 1, 32, 0, s>>>(g, d);
  k_coarse_tables<<<KMC_COARSE_TABLES, 32, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ M2M
// level l (parents, n_l per side) from level l+1.  thread per (parent, coefficient)
__global__ void k_m2m(const Geo g, const Dev d, int l) {
  extern __shared__ double2 sh[];  // 8 * P regular tables of the child offsets
  int nl = 1 << (l - 1), nc = 2 * nl;
  for (int c = threadIdx.x; c < 8 * g.P; c += blockDim.x) sh[c] = d.Rch[(int64_t)(l + 1) * 8 * g.P + c];
  __syncthreads();
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t ncl = (int64_t)nl * nl * nl;
  int64_t cell = t / g.P;
  int ci = (int)(t - cell * g.P);
  if (cell >= ncl) return;
  int n = 0;
  while (tri(n + 1, 0) <= ci) n++;
  int m = ci - tri(n, 0);
  int px = (int)(cell % nl), py = (int)((cell / nl) % nl), pz = (int)(cell / ((int64_t)nl * nl));
  double2 acc = make_double2(0.0, 0.0);
  for (int o = 0; o < 8; o++) {
    int cx = 2 * px + (o & 1), cy = 2 * py + ((o >> 1) & 1), cz = 2 * pz + ((o >> 2) & 1);
    int64_t child = cx + (int64_t)nc * (cy + (int64_t)nc * cz);
    const double2* Mc = d.Mt + (g.cell_off[l + 1] + child) * g.P;
    const double2* Rt = sh + o * g.P;
    for (int k = 0; k <= n; k++)
      for (int ll = -k; ll <= k; ll++) {
        int mm = m - ll;
        if (mm > n - k || mm < -(n - k)) continue;
        double2 a = tab_get(Mc, k, ll), b = tab_get(Rt, n - k, mm);
        acc.x += a.x * b.x - a.y * b.y;
        acc.y += a.x * b.y + a.y * b.x;
      }
  }
  d.Mt[(g.cell_off[l] + cell) * g.P + ci] = acc;
}

// The same M2M with the eight children's expansions and the child-offset
// tables staged in shared memory in full (n, m) order (entry n^2 + n + m, m < 0
// by conjugate symmetry): one CTA per parent cell, one output coefficient per
// thread, no global loads in the sums.  T: the arithmetic (FP64; FP32 in the
// mixed form, whose M2L keeps 29 bits); the expansion is stored in FP64.
template <typename T>
__global__ void __launch_bounds__(128) k_m2m_blk(const Geo g, const Dev d, int l) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char m2m_sm[];
  const int F = (g.p + 1) * (g.p + 1);
  C* Ms = (C*)m2m_sm;  // [8][F] children
  C* Rs = Ms + 8 * F;  // [8][F] child-offset tables
  const int nl = 1 << (l - 1), nc = 2 * nl;
  const int64_t cell = blockIdx.x;
  const int px = (int)(cell % nl), py = (int)((cell / nl) % nl), pz = (int)(cell / ((int64_t)nl * nl));
  for (int t = threadIdx.x; t < 16 * F; t += blockDim.x) {
    const int tb = t / F, u = t - tb * F;
    const int n = (int)sqrtf((float)u + 0.5f), m = u - n * n - n;  // exact: sqrt(n^2 - 1/2) < n <= sqrt(n^2 + 1/2)
    const int o = tb & 7;
    double2 v;
    if (tb < 8) {
      const int cx = 2 * px + (o & 1), cy = 2 * py + ((o >> 1) & 1), cz = 2 * pz + ((o >> 2) & 1);
      const int64_t child = cx + (int64_t)nc * (cy + (int64_t)nc * cz);
      v = tab_get(d.Mt + (g.cell_off[l + 1] + child) * g.P, n, m);
    } else {
      v = tab_get(d.Rch + ((int64_t)(l + 1) * 8 + o) * g.P, n, m);
    }
    C w;
    w.x = (T)v.x;
    w.y = (T)v.y;
    (tb < 8 ? Ms : Rs)[o * F + u] = w;
  }
  __syncthreads();
  for (int ci = threadIdx.x; ci < g.P; ci += blockDim.x) {
    int n = 0;
    while (tri(n + 1, 0) <= ci) n++;
    const int m = ci - tri(n, 0);
    T ax = 0, ay = 0;
    for (int o = 0; o < 8; o++) {
      const C* Mo = Ms + o * F;
      const C* Ro = Rs + o * F;
      for (int k = 0; k <= n; k++) {
        const int j = n - k;
        const int lo = max(-k, m - j), hi = min(k, m + j);
        const C* a = Mo + k * k + k;
        const C* b = Ro + j * j + j + m;
        for (int ll = lo; ll <= hi; ll++) {
          const C u = a[ll], v = b[-ll];
          ax += u.x * v.x - u.y * v.y;
          ay += u.x * v.y + u.y * v.x;
        }
      }
    }
    d.Mt[(g.cell_off[l] + cell) * g.P + ci] = make_double2((double)ax, (double)ay);
  }
}

static size_t fmm_m2m_smem(int p, int prec) {
  return (size_t)16 * (p + 1) * (p + 1) * (prec == 1 ? sizeof(float2) : sizeof(double2));
}

void fmm_m2m(const Geo& g, const Dev& d, cudaStream_t s) {
  const size_t sm = fmm_m2m_smem(g.p, g.prec);
  const bool staged = sm <= 200 * 1024;
  if (staged) {
    if (g.prec == 1) cudaFuncSetAttribute(k_m2m_blk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else cudaFuncSetAttribute(k_m2m_blk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  for (int l = g.L - 1; l >= 1; l--) {
    int64_t ncl = (int64_t)1 << (3 * (l - 1));
    if (staged) {
      if (g.prec == 1) k_m2m_blk<float><<<(unsigned)ncl, 128, sm, s>>>(g, d, l);
      else k_m2m_blk<double><<<(unsigned)ncl, 128, sm, s>>>(g, d, l);
    } else {
      int64_t nt = ncl * g.P;
      k_m2m<<<(unsigned)((nt + 127) / 128), 128, 8 * g.P * sizeof(double2), s>>>(g, d, l);
    }
  }
}

// ------------------------------------------------------------------ M2L tables
// Itab[l][v] = I_j^mu(t_v * w_l) for the 343 offsets t_v in [-3,3]^3 (j <= 2p)
__global__ void k_itab(const Geo g, const Dev d) {
  int l = blockIdx.y + 2;
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= 343) return;
  int tx = v % 7 - 3, ty = (v / 7) % 7 - 3, tz = v / 49 - 3;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  double wl = g.a / (1 << (l - 1));
  irregular_table(tx * wl, ty * wl, tz * wl, 2 * g.p, d.Itab + ((int64_t)l * 343 + v) * g.P2);
}

// level 2: offsets t in [-(2 KMC_TOP + 1), 2 KMC_TOP + 1]^3 (the level-2 cells of
// the (2 KMC_TOP + 1)^3 block of domain copies seen from a level-2 cell)
__global__ void k_itab2(const Geo g, const Dev d) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= KMC_TOP_NOFF) return;
  const int h = (KMC_TOP_SPAN - 1) / 2;
  int tx = v % KMC_TOP_SPAN - h, ty = (v / KMC_TOP_SPAN) % KMC_TOP_SPAN - h, tz = v / (KMC_TOP_SPAN * KMC_TOP_SPAN) - h;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  double w2 = g.a / 2;
  irregular_table(tx * w2, ty * w2, tz * w2, 2 * g.p, d.Itab2 + (int64_t)v * g.P2);
}

void fmm_itab(const Geo& g, const Dev& d, cudaStream_t s) {
  dim3 grid((343 + 63) / 64, g.L - 1);
  k_itab<<<grid, 64, 0, s>>>(g, d);
  k_itab2<<<(KMC_TOP_NOFF + 63) / 64, 64, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ M2L
// The M2L of Algorithm 2 as dense real matrix products grouped by translation
// vector.  A cell's coefficients (0 <= m <= n <= p, complex) are a real vector
// of length 2P (re, im interleaved); the translation by t on level l,
//   Psi_n^m += sum_{k, |l| <= k} (-1)^k Mt_k^l conj(I_{n+k}^{m+l}(t w_l)),
// with Mt_k^{-l} = (-1)^l conj(Mt_k^l), is a real-linear map R_t (2P x 2P).
// The wrapped interaction list of cell b (Sec. 3.1) depends only on the
// parity o = b mod 2: offsets t = 2 delta + c - o with delta in {-1,0,1}^3,
// c in {0,1}^3 and |t|_inf > 1 (189 of them), source (b + t) mod n_l.  So for
// each parity class, Psi[:, cells] = sum_t R_t Mt[:, cells + t] is one
// product of [R_t1 .. R_t189] (2P x 189*2P) with the stacked, gathered
// source columns.

// R_t for the 343 offsets t in [-3,3]^3 of level l (offsets with |t|_inf <= 1
// are never used and left unset): R[(v * 2P + kk) * 2P + i] maps input real
// coefficient kk to output real coefficient i.
__global__ void k_m2l_rmat(const Geo g, const Dev d, int l, double* R) {
  const int v = blockIdx.x;
  const int tx = v % 7 - 3, ty = (v / 7) % 7 - 3, tz = v / 49 - 3;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  const double2* It = d.Itab + ((int64_t)l * 343 + v) * g.P2;
  const int n2 = 2 * g.P;
  double* Rv = R + (int64_t)v * n2 * n2;
  for (int ci = threadIdx.x; ci < g.P; ci += blockDim.x) {
    int n = 0;
    while (tri(n + 1, 0) <= ci) n++;
    const int m = ci - tri(n, 0);
    for (int k = 0; k <= g.p; k++) {
      const double sk = (k & 1) ? -1.0 : 1.0;
      for (int lp = 0; lp <= k; lp++) {
        const double2 I1 = It[tri(n + k, m + lp)];
        double rr = I1.x, ri = I1.y, ir = -I1.y, ii = I1.x;  // (re, im) out x (a, b) in
        if (lp > 0) {  // the mirrored input Mt_k^{-lp} = (-1)^lp conj(Mt_k^lp)
          const double2 I2 = tab_get(It, n + k, m - lp);
          const double sl = (lp & 1) ? -1.0 : 1.0;
          rr += sl * I2.x;
          ri -= sl * I2.y;
          ir -= sl * I2.y;
          ii -= sl * I2.x;
        }
        const int kk = 2 * tri(k, lp);
        Rv[(int64_t)kk * n2 + 2 * ci] = sk * rr;
        Rv[(int64_t)(kk + 1) * n2 + 2 * ci] = sk * ri;
        Rv[(int64_t)kk * n2 + 2 * ci + 1] = sk * ir;
        Rv[(int64_t)(kk + 1) * n2 + 2 * ci + 1] = sk * ii;
      }
    }
  }
}

// One parity class, a tile of G_MT output rows x G_NT target cells, FP64:
// 256 threads, 4 x 4 outputs each (rows tm + 16 r, cells tn + 16 c).
#define G_MT 64
#define G_NT 64
#define G_KT 16
__global__ void __launch_bounds__(256) k_m2l_gemm(const Geo g, const Dev d, int l, const double* R) {
  __shared__ double As[G_KT][G_MT];
  __shared__ double Bs[G_KT][G_NT];
  __shared__ int bcell[G_NT];  // target cells of the tile (-1: none)
  __shared__ int scell[G_NT];  // their sources for the current offset
  const int nl = 1 << (l - 1), h2 = nl >> 1;
  const int o = blockIdx.y, ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
  const int64_t ncls = (int64_t)h2 * h2 * h2;
  const int64_t j0 = (int64_t)blockIdx.x * G_NT;
  const int i0 = blockIdx.z * G_MT;
  const int n2 = 2 * g.P;
  const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
  if (tid < G_NT) {
    const int64_t j = j0 + tid;
    int b = -1;
    if (j < ncls) {
      const int jx = (int)(j % h2), jy = (int)((j / h2) % h2), jz = (int)(j / ((int64_t)h2 * h2));
      b = (2 * jx + ox) + nl * ((2 * jy + oy) + nl * (2 * jz + oz));
    }
    bcell[tid] = b;
  }
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
  const double* Mt = (const double*)(d.Mt + g.cell_off[l] * g.P);
  for (int q = 0; q < 216; q++) {
    const int c8 = q & 7, dl = q >> 3;
    const int tx = 2 * (dl % 3 - 1) + (c8 & 1) - ox, ty = 2 * ((dl / 3) % 3 - 1) + ((c8 >> 1) & 1) - oy,
              tz = 2 * (dl / 9 - 1) + (c8 >> 2) - oz;
    if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) continue;
    __syncthreads();  // the previous offset's source list is no longer read
    if (tid < G_NT) {
      const int b = bcell[tid];
      int sc = -1;
      if (b >= 0) {
        const int bx = b % nl, by = (b / nl) % nl, bz = b / (nl * nl);
        const int ux = bx + tx, uy = by + ty, uz = bz + tz;
        if (!g.bc) sc = ((ux + nl) % nl) + nl * (((uy + nl) % nl) + nl * ((uz + nl) % nl));
        else if (ux >= 0 && ux < nl && uy >= 0 && uy < nl && uz >= 0 && uz < nl) sc = ux + nl * (uy + nl * uz);
      }
      scell[tid] = sc;
    }
    const double* Rv = R + (int64_t)((tx + 3) + 7 * ((ty + 3) + 7 * (tz + 3))) * n2 * n2;
    for (int k0 = 0; k0 < n2; k0 += G_KT) {
      __syncthreads();
      for (int e = tid; e < G_KT * G_MT; e += 256) {
        const int kk = e / G_MT, i = e % G_MT;
        As[kk][i] = (k0 + kk < n2 && i0 + i < n2) ? Rv[(int64_t)(k0 + kk) * n2 + i0 + i] : 0.0;
      }
      for (int e = tid; e < G_KT * G_NT; e += 256) {
        const int j = e / G_KT, kk = e % G_KT;
        const int sc = scell[j];
        Bs[kk][j] = (sc >= 0 && k0 + kk < n2) ? Mt[(int64_t)sc * n2 + k0 + kk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < G_KT; kk++) {
        double a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; r++) a[r] = As[kk][tm + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; c++) bb[c] = Bs[kk][tn + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
          for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
      }
    }
  }
  double* Ps = (double*)(d.Psi + g.cell_off[l] * g.P);
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int i = i0 + tm + 16 * r, b = bcell[tn + 16 * c];
      if (i < n2 && b >= 0) Ps[(int64_t)b * n2 + i] = acc[r][c];
    }
}

// Level 2: cell b receives the M2L of every level-2 cell u of the
// (2 KMC_TOP + 1)^3 block of domain copies (coordinates -2 KMC_TOP ..
// 2 KMC_TOP + 1 per axis) except its 27 nearest; u is an image of source
// cell (u mod 2).  The translation operator is linear in the I table, so the
// images of one source are summed first: Iagg[b][s] = sum over those u of
// I((u - b) w_2), then eight M2Ls per cell.
__global__ void k_m2l_top_agg(const Geo g, const Dev d, double2* Iagg) {
  const int b = blockIdx.x >> 3, sv = blockIdx.x & 7;
  const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
  const int lo = -2 * KMC_TOP, hi = 2 * KMC_TOP + 1, h = (KMC_TOP_SPAN - 1) / 2;
  for (int c = threadIdx.x; c < g.P2; c += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int uz = lo; uz <= hi; uz++)
      for (int uy = lo; uy <= hi; uy++)
        for (int ux = lo; ux <= hi; ux++) {
          if ((ux & 1) + 2 * (uy & 1) + 4 * (uz & 1) != sv) continue;
          const int tx = ux - bx, ty = uy - by, tz = uz - bz;
          if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) continue;
          const int v = (tx + h) + KMC_TOP_SPAN * ((ty + h) + KMC_TOP_SPAN * (tz + h));
          const double2 t = d.Itab2[(int64_t)v * g.P2 + c];
          acc.x += t.x;
          acc.y += t.y;
        }
    Iagg[(int64_t)blockIdx.x * g.P2 + c] = acc;
  }
}

__global__ void k_m2l_top(const Geo g, const Dev d, const double2* Iagg) {
  extern __shared__ double2 shM[];
  const int cell = blockIdx.x;
  const int ci = threadIdx.x;
  int n = 0, m = 0;
  if (ci < g.P) {
    while (tri(n + 1, 0) <= ci) n++;
    m = ci - tri(n, 0);
  }
  double2 acc = make_double2(0.0, 0.0);
  for (int sv = 0; sv < 8; sv++) {
    __syncthreads();
    const double2* Ms = d.Mt + (g.cell_off[2] + sv) * g.P;
    for (int k = threadIdx.x; k < g.P; k += blockDim.x) shM[k] = Ms[k];
    __syncthreads();
    if (ci < g.P) {
      const double2* It = Iagg + (int64_t)(cell * 8 + sv) * g.P2;
      for (int k = 0; k <= g.p; k++) {
        double2 s = make_double2(0.0, 0.0);
        for (int ll = -k; ll <= k; ll++) {
          const double2 a = tab_get(shM, k, ll);
          const double2 b = tab_get(It, n + k, m + ll);
          s.x += a.x * b.x + a.y * b.y;  // a * conj(b)
          s.y += a.y * b.x - a.x * b.y;
        }
        if (k & 1) {
          acc.x -= s.x;
          acc.y -= s.y;
        } else {
          acc.x += s.x;
          acc.y += s.y;
        }
      }
    }
  }
  if (ci < g.P) d.Psi[(g.cell_off[2] + cell) * g.P + ci] = acc;
}

// ------------------------------------------------------------------ M2L on the bf16 tensor cores
// The same products with FP64 accuracy from bf16 tensor-core MMAs, by exact
// integer slicing (the Ozaki splitting of a floating-point product into
// error-free partial products).
//  * Scaling by powers of two (exact): the input coefficient kk of every cell
//    of the level is divided by 2^ec(kk) (ec from the level's largest
//    |Mt[., kk]|), the translation entries R_t[i][kk] are multiplied by it, and
//    row i of all R_t is divided by 2^er(i) (er from the row's largest entry),
//    so that every scaled value lies in (-1, 1).
//  * Slicing: x = sum_{s=1..S} x_s 2^(-7 s) + r, |r| <= 2^(-7S - 1), with
//    integer slices, |x_1| <= 128 and -64 <= x_s <= 63 (s > 1), held exactly
//    in bf16: the balanced base-128 digits of N = rint(x 2^(7S)) (|N| <= 2^42,
//    exact in int64), cut with integer arithmetic.
//  * The product keeps the slice pairs with a + b = D <= S + 1 and sums each
//    diagonal D separately: per translation (K = 2P padded, at most 352
//    terms) the FP32 tensor-core accumulation of integers stays below 2^24
//    (at most 2*128*64 + (S-2)*64*64 per term), so it is exact; it is then
//    added into an int32 per diagonal (189 translations below 2^31 for
//    p <= 16), and the diagonals are combined in FP64 with their weight
//    2^(er(i) - 7 D).  S = 6: 43 significant bits per operand (FP64 form).
//  * The mixed form keeps the first four slices (diagonals D <= 5, 10 of the
//    21 slice products): 29 significant bits, an entry error of about K 2^-28
//    of its row and column scales, below the FP32 arithmetic of that form's
//    near field, L2P and dU.

// bf16 bits of a small integer (|v| <= 256: exact in bf16)
__device__ __forceinline__ unsigned short oz_bf16_int(long long v) {
  const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
  return *(const unsigned short*)&b;
}
__device__ __forceinline__ void oz_split(double x, unsigned short* out, size_t stride) {
  // x 2^(7S) is exact (a power-of-two scaling of |x| < 1); its nearest integer has at most 42 bits
  long long n = __double2ll_rn(x * 4398046511104.0);  // 2^42 = 2^(7 OZ_S)
  static_assert(OZ_S == 6, "2^(7 OZ_S)");
#pragma unroll
  for (int sl = OZ_S - 1; sl > 0; sl--) {
    const long long dg = ((n + 64) & 127) - 64;  // balanced digit in [-64, 63]
    out[sl * stride] = oz_bf16_int(dg);
    n = (n - dg) >> 7;  // exact: n - dg is a multiple of 128
  }
  out[0] = oz_bf16_int(n);  // |n| <= 128
}

// largest |Mt[cell][kk]| over the cells of level l, per real coefficient kk
__global__ void k_oz_colmax(const Geo g, const Dev d, int l, unsigned long long* colmax) {
  const int n2 = 2 * g.P;
  const int64_t ncell = (int64_t)1 << (3 * (l - 1));
  const double* Mt = (const double*)(d.Mt + g.cell_off[l] * g.P);
  const int64_t per = (ncell + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = blockIdx.x * per, c1 = min(ncell, c0 + per);
  for (int kk = threadIdx.x; kk < n2; kk += blockDim.x) {
    double m = 0.0;
    for (int64_t c = c0; c < c1; c++) m = fmax(m, fabs(Mt[c * n2 + kk]));
    if (c1 > c0) atomicMax(&colmax[kk], (unsigned long long)__double_as_longlong(m));
  }
}

// largest scaled |R_t[i][kk]| 2^ec(kk) over the used translations, per row i
__global__ void k_oz_rowmax(const Geo g, const double* R, const unsigned long long* colmax,
                            unsigned long long* rowmax) {
  const int v = blockIdx.x;
  const int tx = v % 7 - 3, ty = (v / 7) % 7 - 3, tz = v / 49 - 3;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  const int n2 = 2 * g.P;
  __shared__ int ec[2 * OZ_MAXP_P];
  for (int k = threadIdx.x; k < n2; k += blockDim.x) ec[k] = oz_exp(colmax[k]);
  __syncthreads();
  const double* Rv = R + (int64_t)v * n2 * n2;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    // max of |R| 2^ec over kk, compared as the bit patterns of non-negative doubles; the
    // power-of-two scaling by an exponent add where the result stays normal, else by ldexp
    long long m = 0;
    for (int kk = 0; kk < n2; kk++) {
      long long b = __double_as_longlong(Rv[(int64_t)kk * n2 + i]) & 0x7FFFFFFFFFFFFFFFll;
      const int ex = (int)(b >> 52) + ec[kk];
      if ((b >> 52) != 0 && ex > 0 && ex < 2047)
        b += (long long)ec[kk] << 52;
      else if (b != 0)
        b = __double_as_longlong(ldexp(__longlong_as_double(b), ec[kk]));
      m = b > m ? b : m;
    }
    atomicMax(&rowmax[i], (unsigned long long)m);
  }
}

// A slices: As[((v S + s) rows + i) cols + kk], row-major per translation and slice
__global__ void k_oz_aslice(const Geo g, const double* R, const unsigned long long* colmax,
                            const unsigned long long* rowmax, unsigned short* As) {
  const int v = blockIdx.x;
  const int tx = v % 7 - 3, ty = (v / 7) % 7 - 3, tz = v / 49 - 3;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  const int n2 = 2 * g.P, nr = oz_rows(n2), nc = oz_cols(n2);
  __shared__ int ec[2 * OZ_MAXP_P], er[2 * OZ_MAXP_P];  // the scaling exponents
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    ec[k] = oz_exp(colmax[k]);
    er[k] = oz_exp(rowmax[k]);
  }
  __syncthreads();
  const double* Rv = R + (int64_t)v * n2 * n2;
  const size_t stride = (size_t)nr * nc;
  for (int e = threadIdx.x + blockIdx.y * blockDim.x; e < nr * nc; e += blockDim.x * gridDim.y) {
    const int i = e / nc, kk = e % nc;
    double x = 0.0;
    if (i < n2 && kk < n2) x = ldexp(Rv[(int64_t)kk * n2 + i], ec[kk] - er[i]);
    oz_split(x, As + (size_t)v * OZ_S * stride + e, stride);
  }
}

// A slices in the layout of the tcgen05 M2L: per translation v, slice s and K
// chunk c of 64 one contiguous block of NN rows x 64 values in the order of
// the MMA's 128-byte-swizzled K-major shared-memory operand (row i at
// (i / 8) 512 + (i mod 8) 64 values, its eight pieces of 8 values permuted
// by i mod 8); rows i >= 2P and values kk >= 2P are zero.
__global__ void k_oz_aslice_tc(const Geo g, const double* R, const unsigned long long* colmax,
                               const unsigned long long* rowmax, unsigned short* As, int NN, int nkc) {
  const int v = blockIdx.x;
  const int tx = v % 7 - 3, ty = (v / 7) % 7 - 3, tz = v / 49 - 3;
  if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) return;
  const int n2 = 2 * g.P, K = 64 * nkc;
  __shared__ int ec[2 * OZ_MAXP_P], er[2 * OZ_MAXP_P];  // the scaling exponents
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    ec[k] = oz_exp(colmax[k]);
    er[k] = oz_exp(rowmax[k]);
  }
  __syncthreads();
  const double* Rv = R + (int64_t)v * n2 * n2;
  const size_t stride = (size_t)NN * K;
  for (int e = threadIdx.x + blockIdx.y * blockDim.x; e < NN * K; e += blockDim.x * gridDim.y) {
    const int i = e / K, kk = e % K;
    double x = 0.0;
    if (i < n2 && kk < n2) x = ldexp(Rv[(int64_t)kk * n2 + i], ec[kk] - er[i]);
    const int k = kk & 63;
    const size_t off = (size_t)(kk >> 6) * NN * 64 + (size_t)(i >> 3) * 512 + (i & 7) * 64 +
                       ((((k >> 3) ^ i) & 7) << 3) + (k & 7);
    oz_split(x, As + (size_t)v * OZ_S * stride + off, stride);
  }
}

// B slices: Bs[(s ncell + cell) cols + kk]
__global__ void k_oz_bslice(const Geo g, const Dev d, int l, const unsigned long long* colmax, unsigned short* Bs) {
  const int n2 = 2 * g.P, nc = oz_cols(n2);
  const int64_t ncell = (int64_t)1 << (3 * (l - 1));
  const double* Mt = (const double*)(d.Mt + g.cell_off[l] * g.P);
  const size_t stride = (size_t)ncell * nc;
  __shared__ int ec[2 * OZ_MAXP_P];
  for (int k = threadIdx.x; k < n2; k += blockDim.x) ec[k] = oz_exp(colmax[k]);
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncell * nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / nc;
    const int kk = (int)(e % nc);
    const double x = kk < n2 ? ldexp(Mt[c * n2 + kk], -ec[kk]) : 0.0;
    oz_split(x, Bs + e, stride);
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// One parity class o, a tile of OZ_MT output rows x OZ_NT target cells; four
// warps of 32 x 32 (2 x 4 MMA tiles of 16 x 8).  One pass per diagonal D.
// Levels with few cells split the interaction list over gridDim.x / ntile
// CTAs per tile; those add their exact per-diagonal integer sums into acc64
// (integer adds: the result does not depend on their order) and
// k_oz_finish converts.  Otherwise acc64 is null and the CTA writes Psi.
__global__ void __launch_bounds__(128) k_m2l_oz(const Geo g, const Dev d, int l, const unsigned short* As,
                                                const unsigned short* Bs, const unsigned long long* rowmax,
                                                int ntile, long long* acc64) {
  extern __shared__ __align__(128) unsigned short oz_sm[];
  const int S = oz_slices(g);                   // slices in use
  unsigned short* sA = oz_sm;                   // [S][OZ_MT][OZ_LD]
  unsigned short* sB = sA + S * OZ_MT * OZ_LD;  // [S][OZ_NT][OZ_LD]
  __shared__ int bcell[OZ_NT], scell[OZ_NT];
  const int nl = 1 << (l - 1), h2 = nl >> 1;
  const int o = blockIdx.y, ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
  const int64_t ncls = (int64_t)h2 * h2 * h2, ncell = (int64_t)nl * nl * nl;
  const int tile = blockIdx.x % ntile, split = blockIdx.x / ntile, nsplit = gridDim.x / ntile;
  const int q_begin = 216 * split / nsplit, q_end = 216 * (split + 1) / nsplit;
  const int64_t j0 = (int64_t)tile * OZ_NT;
  const int i0 = blockIdx.z * OZ_MT;
  const int n2 = 2 * g.P, nr = oz_rows(n2), nc = oz_cols(n2);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wm = warp & 1, wn = warp >> 1;
  if (tid < OZ_NT) {
    const int64_t j = j0 + tid;
    int b = -1;
    if (j < ncls) {
      const int jx = (int)(j % h2), jy = (int)((j / h2) % h2), jz = (int)(j / ((int64_t)h2 * h2));
      b = (2 * jx + ox) + nl * ((2 * jy + oy) + nl * (2 * jz + oz));
    }
    bcell[tid] = b;
  }
  const uint32_t sA0 = (uint32_t)__cvta_generic_to_shared(sA), sB0 = (uint32_t)__cvta_generic_to_shared(sB);
  // ldmatrix lane addresses (bytes, within one slice's tile, k offset 0)
  const int q = lane >> 3, rr = lane & 7;
  uint32_t aoff[2], boff[2];
#pragma unroll
  for (int mf = 0; mf < 2; mf++) aoff[mf] = 2u * ((32 * wm + 16 * mf + rr + 8 * (q & 1)) * OZ_LD + 8 * (q >> 1));
#pragma unroll
  for (int np = 0; np < 2; np++) boff[np] = 2u * ((32 * wn + 16 * np + rr + 8 * (q >> 1)) * OZ_LD + 8 * (q & 1));
  const size_t astride = (size_t)nr * nc, bstride = (size_t)ncell * nc;
  const unsigned short* Bl = Bs;
  double* Ps = (double*)(d.Psi + g.cell_off[l] * g.P);

  for (int D = 2; D <= S + 1; D++) {
    const int ns = D - 1;  // slices 0 .. ns - 1 of both operands meet on this diagonal
    int iacc[2][4][4];
#pragma unroll
    for (int mf = 0; mf < 2; mf++)
#pragma unroll
      for (int nf = 0; nf < 4; nf++)
#pragma unroll
        for (int c = 0; c < 4; c++) iacc[mf][nf][c] = 0;
    for (int qo = q_begin; qo < q_end; qo++) {
      const int c8 = qo & 7, dl = qo >> 3;
      const int tx = 2 * (dl % 3 - 1) + (c8 & 1) - ox, ty = 2 * ((dl / 3) % 3 - 1) + ((c8 >> 1) & 1) - oy,
                tz = 2 * (dl / 9 - 1) + (c8 >> 2) - oz;
      if (abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1) continue;
      __syncthreads();  // the previous offset's tiles and source list are no longer read
      if (tid < OZ_NT) {
        const int b = bcell[tid];
        int sc = -1;
        if (b >= 0) {
          const int bx = b % nl, by = (b / nl) % nl, bz = b / (nl * nl);
          const int ux = bx + tx, uy = by + ty, uz = bz + tz;
          if (!g.bc) sc = ((ux + nl) % nl) + nl * (((uy + nl) % nl) + nl * ((uz + nl) % nl));
          else if (ux >= 0 && ux < nl && uy >= 0 && uy < nl && uz >= 0 && uz < nl) sc = ux + nl * (uy + nl * uz);
        }
        scell[tid] = sc;
      }
      const int v = (tx + 3) + 7 * ((ty + 3) + 7 * (tz + 3));
      const unsigned short* Av = As + (size_t)v * OZ_S * astride;
      float facc[2][4][4];
#pragma unroll
      for (int mf = 0; mf < 2; mf++)
#pragma unroll
        for (int nf = 0; nf < 4; nf++)
#pragma unroll
          for (int c = 0; c < 4; c++) facc[mf][nf][c] = 0.f;
      for (int k0 = 0; k0 < nc; k0 += OZ_KC) {
        __syncthreads();  // scell written; previous chunk consumed
        // 16-byte pieces: per slice OZ_MT rows x (OZ_KC / 8) pieces of A, the same of B
        for (int e = tid; e < ns * OZ_MT * (OZ_KC / 8); e += 128) {
          const int sl = e / (OZ_MT * (OZ_KC / 8)), rem = e % (OZ_MT * (OZ_KC / 8));
          const int row = rem / (OZ_KC / 8), pc = rem % (OZ_KC / 8);
          cp_async16(sA0 + 2u * ((sl * OZ_MT + row) * OZ_LD + 8 * pc),
                     Av + (size_t)sl * astride + (size_t)(i0 + row) * nc + k0 + 8 * pc);
          const int sc = scell[row];
          const uint32_t db = sB0 + 2u * ((sl * OZ_NT + row) * OZ_LD + 8 * pc);
          if (sc >= 0)
            cp_async16(db, Bl + (size_t)sl * bstride + (size_t)sc * nc + k0 + 8 * pc);
          else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(db), "r"(0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < OZ_KC; ks += 16) {
          for (int a = 0; a < ns; a++) {
            const int bsl = ns - 1 - a;
            uint32_t af[2][4], bfr[2][4];
#pragma unroll
            for (int mf = 0; mf < 2; mf++)
              ldsm_x4(sA0 + 2u * (a * OZ_MT * OZ_LD + ks) + aoff[mf], af[mf][0], af[mf][1], af[mf][2], af[mf][3]);
#pragma unroll
            for (int np = 0; np < 2; np++)
              ldsm_x4(sB0 + 2u * (bsl * OZ_NT * OZ_LD + ks) + boff[np], bfr[np][0], bfr[np][1], bfr[np][2],
                      bfr[np][3]);
#pragma unroll
            for (int mf = 0; mf < 2; mf++)
#pragma unroll
              for (int nf = 0; nf < 4; nf++)
                mma_bf16(facc[mf][nf], af[mf], bfr[nf >> 1][2 * (nf & 1)], bfr[nf >> 1][2 * (nf & 1) + 1]);
          }
        }
      }
      // this translation's exact integer sums into the diagonal's int32 accumulator
#pragma unroll
      for (int mf = 0; mf < 2; mf++)
#pragma unroll
        for (int nf = 0; nf < 4; nf++)
#pragma unroll
          for (int c = 0; c < 4; c++) iacc[mf][nf][c] += __float2int_rn(facc[mf][nf][c]);
    }
    // the diagonal's weight 2^(er(i) - 7 D), accumulated in FP64 into Psi
    const int g4 = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mf = 0; mf < 2; mf++)
#pragma unroll
      for (int nf = 0; nf < 4; nf++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const int i = i0 + 32 * wm + 16 * mf + g4 + 8 * (c >> 1);
          const int b = bcell[32 * wn + 8 * nf + 2 * t4 + (c & 1)];
          if (i < n2 && b >= 0) {
            if (acc64) {
              atomicAdd((unsigned long long*)(acc64 + ((int64_t)(D - 2) * ncell + b) * n2 + i),
                        (unsigned long long)(long long)iacc[mf][nf][c]);
            } else {
              const double val = ldexp((double)iacc[mf][nf][c], oz_exp(rowmax[i]) - 7 * D);
              double* out = Ps + (int64_t)b * n2 + i;
              *out = (D == 2 ? 0.0 : *out) + val;
            }
          }
        }
  }
}

// Psi from the split CTAs' per-diagonal integer sums
// B slices in the layout of the tcgen05 M2L: per slice and parity class
// (cls = (x & 1) + 2 (y & 1) + 4 (z & 1)) the class's cells on a grid of
// (h2 + 4)^3 positions, two ghost layers on each side (their periodic images,
// zero in free space), so that the source cells of a box of target cells
// under one translation form one box of this array:
// Bp[(((s 8 + cls) Xp + z') Xp + y') Xp + x'][kk], cell x = 2 (x' - 2) + (cls & 1).
__global__ void k_oz_bslice_tc(const Geo g, const Dev d, int l, const unsigned long long* colmax, unsigned short* Bp) {
  const int n2 = 2 * g.P, nc = oz_cols(n2);
  const int nl = 1 << (l - 1), Xp = (nl >> 1) + 4;
  const int64_t npos = (int64_t)8 * Xp * Xp * Xp;
  const double* Mt = (const double*)(d.Mt + g.cell_off[l] * g.P);
  const size_t stride = (size_t)npos * nc;
  __shared__ int ec[2 * OZ_MAXP_P];
  for (int k = threadIdx.x; k < n2; k += blockDim.x) ec[k] = oz_exp(colmax[k]);
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npos * nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pi = e / nc;
    const int kk = (int)(e % nc);
    const int xp = (int)(pi % Xp), yp = (int)((pi / Xp) % Xp), zp = (int)((pi / Xp / Xp) % Xp), cls = (int)(pi / Xp / Xp / Xp);
    int x = 2 * (xp - 2) + (cls & 1), y = 2 * (yp - 2) + ((cls >> 1) & 1), z = 2 * (zp - 2) + (cls >> 2);
    bool in = true;
    if (g.bc) {
      in = x >= 0 && x < nl && y >= 0 && y < nl && z >= 0 && z < nl;
    } else {
      x = (x + 2 * nl) % nl;
      y = (y + 2 * nl) % nl;
      z = (z + 2 * nl) % nl;
    }
    double v = 0.0;
    if (in && kk < n2) v = ldexp(Mt[((int64_t)x + nl * ((int64_t)y + nl * z)) * n2 + kk], -ec[kk]);
    oz_split(v, Bp + e, stride);
  }
}

__global__ void k_oz_finish(const Geo g, const Dev d, int l, const long long* acc64, const unsigned long long* rowmax) {
  const int n2 = 2 * g.P;
  const int64_t ncell = (int64_t)1 << (3 * (l - 1));
  double* Ps = (double*)(d.Psi + g.cell_off[l] * g.P);
  const int S = oz_slices(g);
  __shared__ double pw[OZ_S][2 * OZ_MAXP_P];  // 2^(er(i) - 7 D): exact powers of two
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    const int er = oz_exp(rowmax[k]);
    for (int D = 2; D <= S + 1; D++) pw[D - 2][k] = ldexp(1.0, er - 7 * D);
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncell * n2; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n2);
    double v = 0.0;  // the diagonals in order D = 2, 3, ...; each term exact (an integer times a power of two)
    for (int D = 2; D <= S + 1; D++) v += (double)acc64[(int64_t)(D - 2) * ncell * n2 + e] * pw[D - 2][i];
    Ps[e] = v;
  }
}

static size_t oz_dyn_smem(int S) { return (size_t)2 * S * OZ_MT * OZ_LD * sizeof(unsigned short); }

// interaction-list splits of level l: enough CTAs for three per SM (152 SMs)
static int oz_splits(const Geo& g, int l) {
  const int64_t h2 = (int64_t)1 << (l - 2);
  const int64_t ctas = (h2 * h2 * h2 + OZ_NT - 1) / OZ_NT * 8 * (oz_rows(2 * g.P) / OZ_MT);
  const int64_t want = (3 * 152 + ctas - 1) / ctas;
  return (int)(want < 1 ? 1 : (want > 24 ? 24 : want));
}

// scratch: R tables of one level (343 (2P)^2 doubles), 64 aggregated I
// tables and, for the tensor-core form, the scaling maxima and the slices
// elements of the B-slice scratch: the mma.sync layout, or the ghost-padded
// class layout of the tcgen05 form at the leaf level
static size_t oz_bs_elems(const Geo& g) {
  const size_t nc = oz_cols(2 * g.P);
  size_t e = (size_t)OZ_S * (size_t)g.ML * nc;
  if (fmm_m2l_tc_rows(g) > 0) {
    const size_t xp = (size_t)g.nL / 2 + 4, t = (size_t)OZ_S * 8 * xp * xp * xp * nc;
    e = t > e ? t : e;
  }
  return e;
}

size_t fmm_m2l_scratch_bytes(const Geo& g) {
  const size_t n2 = 2 * (size_t)g.P;
  size_t b = 343 * n2 * n2 * sizeof(double) + 64 * (size_t)g.P2 * sizeof(double2);
  if ((g.m2l == 0 || g.m2l == 2) && g.p <= OZ_MAXP) {
    const size_t nr = oz_rows((int)n2), nc = oz_cols((int)n2);
    b += 2 * nr * sizeof(unsigned long long);                      // colmax, rowmax
    const size_t tce = (size_t)fmm_m2l_tc_rows(g) * 64 * fmm_m2l_tc_kchunks(g);  // tcgen05 layout
    const size_t ase = nr * nc > tce ? nr * nc : tce;
    b += 343 * OZ_S * ase * sizeof(unsigned short);                 // A slices (either layout)
    b += oz_bs_elems(g) * sizeof(unsigned short);  // B slices (leaf level is the largest)
    size_t acc = 0;  // per-diagonal integer sums (split levels; every level of the tcgen05 form)
    for (int l = 3; l <= g.L; l++)
      if (oz_splits(g, l) > 1 || fmm_m2l_tc_rows(g) > 0) {
        const size_t a = (size_t)(OZ_S) * ((size_t)1 << (3 * (l - 1))) * n2 * sizeof(long long);
        acc = a > acc ? a : acc;
      }
    b += acc;
  }
  return b;
}

void fmm_m2l(const Geo& g, const Dev& d, void* scratch, cudaStream_t s, cudaEvent_t* ev) {
  const size_t n2 = 2 * (size_t)g.P;
  double* R = (double*)scratch;
  double2* Iagg = (double2*)(R + 343 * n2 * n2);
  const int bs = g.P <= 128 ? 128 : 256;
  if (g.bc) {  // free space: the 8 level-2 cells are all neighbours, the level-2 list is empty
    cudaMemsetAsync(d.Psi + g.cell_off[2] * g.P, 0, sizeof(double2) * 8 * g.P, s);
  } else {
    k_m2l_top_agg<<<64, 128, 0, s>>>(g, d, Iagg);
    k_m2l_top<<<8, bs, g.P * sizeof(double2), s>>>(g, d, Iagg);
  }
  const bool tensor = (g.m2l == 0 || g.m2l == 2) && g.p <= OZ_MAXP;
  const bool tc = tensor && fmm_m2l_tc_ok(g);  // the tcgen05 form
  unsigned long long *colmax = nullptr, *rowmax = nullptr;
  unsigned short *As = nullptr, *Bs = nullptr;
  long long* acc64 = nullptr;
  if (tensor) {
    const size_t nr = oz_rows((int)n2), nc = oz_cols((int)n2);
    colmax = (unsigned long long*)(Iagg + 64 * (size_t)g.P2);
    rowmax = colmax + nr;
    As = (unsigned short*)(rowmax + nr);
    const size_t tce = (size_t)fmm_m2l_tc_rows(g) * 64 * fmm_m2l_tc_kchunks(g);
    Bs = As + 343 * OZ_S * (nr * nc > tce ? nr * nc : tce);
    acc64 = (long long*)(Bs + oz_bs_elems(g));
    cudaFuncSetAttribute(k_m2l_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_dyn_smem(OZ_S));
  }
  for (int l = 3; l <= g.L; l++) {
    k_m2l_rmat<<<343, 128, 0, s>>>(g, d, l, R);
    const int64_t h2 = (int64_t)1 << (l - 2);
    if (tensor) {
      const int nr = oz_rows((int)n2);
      cudaMemsetAsync(colmax, 0, 2 * nr * sizeof(unsigned long long), s);
      k_oz_colmax<<<256, 256, 0, s>>>(g, d, l, colmax);
      k_oz_rowmax<<<343, 256, 0, s>>>(g, R, colmax, rowmax);
      const int64_t ncell = (int64_t)1 << (3 * (l - 1));
      const unsigned nfin = (unsigned)((ncell * n2 + 255) / 256 < 4096 ? (ncell * n2 + 255) / 256 : 4096);
      bool done = false;
      if (tc) {  // tcgen05: slices in its layouts, every level's diagonals through acc64
        k_oz_aslice_tc<<<dim3(343, 8), 256, 0, s>>>(g, R, colmax, rowmax, As, fmm_m2l_tc_rows(g),
                                                     fmm_m2l_tc_kchunks(g));
        const int xp = (int)(h2 / 2) + 4;
        const int64_t nbp = ((int64_t)8 * xp * xp * xp * oz_cols((int)n2) + 255) / 256;
        k_oz_bslice_tc<<<(unsigned)(nbp < 4096 ? nbp : 4096), 256, 0, s>>>(g, d, l, colmax, Bs);
        cudaMemsetAsync(acc64, 0, (size_t)OZ_S * ncell * n2 * sizeof(long long), s);
        if (ev) cudaEventRecord(ev[2 * l], s);
        done = fmm_m2l_tc(g, d, l, As, Bs, acc64, s);
        if (ev) cudaEventRecord(ev[2 * l + 1], s);
        if (done) k_oz_finish<<<nfin, 256, 0, s>>>(g, d, l, acc64, rowmax);
      }
      if (!done) {  // the mma.sync form (also when the tcgen05 launch was not possible)
        k_oz_aslice<<<dim3(343, 8), 256, 0, s>>>(g, R, colmax, rowmax, As);
        const int64_t nb = ((ncell * oz_cols((int)n2)) + 255) / 256;
        k_oz_bslice<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, s>>>(g, d, l, colmax, Bs);
        const int ntile = (int)((h2 * h2 * h2 + OZ_NT - 1) / OZ_NT), nsplit = oz_splits(g, l);
        if (nsplit > 1) cudaMemsetAsync(acc64, 0, (size_t)OZ_S * ncell * n2 * sizeof(long long), s);
        dim3 grid((unsigned)(ntile * nsplit), 8, (unsigned)(nr / OZ_MT));
        if (ev) cudaEventRecord(ev[2 * l], s);
        k_m2l_oz<<<grid, 128, oz_dyn_smem(oz_slices(g)), s>>>(g, d, l, As, Bs, rowmax, ntile, nsplit > 1 ? acc64 : nullptr);
        if (ev) cudaEventRecord(ev[2 * l + 1], s);
        if (nsplit > 1) k_oz_finish<<<nfin, 256, 0, s>>>(g, d, l, acc64, rowmax);
      }
    } else {
      dim3 grid((unsigned)((h2 * h2 * h2 + G_NT - 1) / G_NT), 8, (unsigned)((n2 + G_MT - 1) / G_MT));
      if (ev) cudaEventRecord(ev[2 * l], s);
      k_m2l_gemm<<<grid, 256, 0, s>>>(g, d, l, R);
      if (ev) cudaEventRecord(ev[2 * l + 1], s);
    }
  }
}

// ------------------------------------------------------------------ lattice sums
// S_j^mu = sum over far images nu (|nu|_inf > KMC_TOP) of I_j^mu(a nu), evaluated by
// Ewald splitting of I_j^mu = (j-mu)!(j+mu)! R_j^mu(x)/|x|^{2j+1}:
//   sum_{nu != 0} R(a nu)/|a nu|^{2j+1}
//     = sum_{nu != 0} R(a nu) Q(j+1/2, beta^2 |a nu|^2) / |a nu|^{2j+1}
//     + (-i)^j pi^{j-1/2} / (a^3 Gamma(j+1/2)) sum_{k = m/a != 0} R(k) exp(-pi^2 k^2 / beta^2) / k^2
// (Poisson summation of the harmonic Gaussian; Q, P = regularised upper,
// lower incomplete gamma).  The images of the near block (|nu|_inf <= KMC_TOP)
// are removed by dropping their real-space terms and subtracting their smooth
// parts R P(..)/|x|^{2j+1}.
// Degrees j <= 3 vanish in cubic summation order (j = 0 multiplies the zero
// net charge; j = 1, 2, 3 vanish by cubic symmetry).
#define LS_NR 6
#define LS_KM 9
#define LS_BETA_A 3.0

__global__ void k_lattice_terms(const Geo g, double2* terms, int nvec) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const int P2 = g.P2, p2 = 2 * g.p;
  double2* out = terms + (int64_t)v * P2;
  const int nr = 2 * LS_NR + 1, nk = 2 * LS_KM + 1;
  const double a = g.a, beta = LS_BETA_A / a;
  if (v < nr * nr * nr) {
    int nx = v % nr - LS_NR, ny = (v / nr) % nr - LS_NR, nz = v / (nr * nr) - LS_NR;
    int ninf = max(abs(nx), max(abs(ny), abs(nz)));
    if (ninf == 0) {
      for (int c = 0; c < P2; c++) out[c] = make_double2(0.0, 0.0);
      return;
    }
    double x = a * nx, y = a * ny, z = a * nz;
    double r2 = x * x + y * y + z * z, r = sqrt(r2);
    double X = beta * beta * r2;
    regular_table(x, y, z, p2, out);  // R_j^mu(a nu), scaled in place below
    double qj = erfc(sqrt(X));                                     // Q(1/2, X)
    double tj = 2.0 * sqrt(X) * exp(-X) / sqrt(M_PI);              // X^{1/2} e^{-X} / Gamma(3/2)
    double rp = 1.0 / r;                                           // 1/r^{2j+1}
    for (int j = 0; j <= p2; j++) {
      double wgt;
      if (ninf > KMC_TOP) {
        wgt = qj;  // far image: real-space part
      } else {
        // near image: minus the smooth part P(j+1/2, X) by its positive series
        double s = j + 0.5;
        double term = exp(s * log(X) - X - lgamma(s + 1.0));
        double sum = 0.0;
        for (int k = 0; k < 400 && term > 1e-300; k++) {
          sum += term;
          term *= X / (s + k + 1.0);
          if (k > X && term < 1e-18 * sum) break;
        }
        wgt = -sum;
      }
      for (int mu = 0; mu <= j; mu++) {
        double f = f_fact[j - mu] * f_fact[j + mu] * wgt * rp;
        double2 rv = out[tri(j, mu)];
        out[tri(j, mu)] = make_double2(f * rv.x, f * rv.y);
      }
      qj += tj;
      tj *= X / (j + 1.5);
      rp /= r2;
    }
  } else {
    int u = v - nr * nr * nr;
    int mx = u % nk - LS_KM, my = (u / nk) % nk - LS_KM, mz = u / (nk * nk) - LS_KM;
    if (mx == 0 && my == 0 && mz == 0) {
      for (int c = 0; c < P2; c++) out[c] = make_double2(0.0, 0.0);
      return;
    }
    double kx = mx / a, ky = my / a, kz = mz / a;
    double k2 = kx * kx + ky * ky + kz * kz;
    regular_table(kx, ky, kz, p2, out);  // R_j^mu(k), scaled in place below
    double gk = exp(-M_PI * M_PI * k2 / (beta * beta)) / k2;
    for (int j = 0; j <= p2; j++) {
      double pre = exp((j - 0.5) * log(M_PI) - lgamma(j + 0.5)) / (a * a * a) * gk;
      for (int mu = 0; mu <= j; mu++) {
        double f = f_fact[j - mu] * f_fact[j + mu] * pre;
        double2 rv = out[tri(j, mu)];
        double2 t = make_double2(f * rv.x, f * rv.y);
        // multiply by (-i)^j
        double2 o;
        switch (j & 3) {
          case 0: o = t; break;
          case 1: o = make_double2(t.y, -t.x); break;
          case 2: o = make_double2(-t.x, -t.y); break;
          default: o = make_double2(-t.y, t.x); break;
        }
        out[tri(j, mu)] = o;
      }
    }
  }
}

__global__ void k_lattice_reduce(const Geo g, const double2* terms, int nvec, double2* S) {
  __shared__ double sx[256], sy[256];
  int c = blockIdx.x;
  int j = 0;
  while (tri(j + 1, 0) <= c) j++;
  double ax = 0.0, ay = 0.0;
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    double2 t = terms[(int64_t)v * g.P2 + c];
    ax += t.x;
    ay += t.y;
  }
  sx[threadIdx.x] = ax;
  sy[threadIdx.x] = ay;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sx[threadIdx.x] += sx[threadIdx.x + st];
      sy[threadIdx.x] += sy[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) S[c] = (j <= 3) ? make_double2(0.0, 0.0) : make_double2(sx[0], sy[0]);
}

void fmm_lattice_sums(const Geo& g, const Dev& d, cudaStream_t s) {
  if (g.bc) {  // free space: no images, no far field
    cudaMemsetAsync(d.S, 0, sizeof(double2) * g.P2, s);
    return;
  }
  const int nr = 2 * LS_NR + 1, nk = 2 * LS_KM + 1;
  int nvec = nr * nr * nr + nk * nk * nk;
  // scratch: nvec * P2 complex (reuses the per-step phi_new / dU buffers is not
  // safe in general, so it is a dedicated temporary owned by the caller)
  double2* terms = (double2*)d.scratch;
  k_lattice_terms<<<(nvec + 63) / 64, 64, 0, s>>>(g, terms, nvec);
  k_lattice_reduce<<<g.P2, 256, 0, s>>>(g, terms, nvec, d.S);
}

// ------------------------------------------------------------------ far field
// H = R K: H_n^m = sum_{k,l} (-1)^k K_k^l conj(S_{n+k}^{m+l}), K = level-1 multipole
__global__ void k_far_field(const Geo g, const Dev d) {
  int ci = threadIdx.x;
  if (ci >= g.P) return;
  int n = 0;
  while (tri(n + 1, 0) <= ci) n++;
  int m = ci - tri(n, 0);
  const double2* K = d.Mt + g.cell_off[1] * g.P;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k <= g.p; k++) {
    double sgn = (k & 1) ? -1.0 : 1.0;
    for (int ll = -k; ll <= k; ll++) {
      double2 a = tab_get(K, k, ll), b = tab_get(d.S, n + k, m + ll);
      acc.x += sgn * (a.x * b.x + a.y * b.y);
      acc.y += sgn * (a.y * b.x - a.x * b.y);
    }
  }
  d.Psi[g.cell_off[1] * g.P + ci] = acc;
}

void fmm_far_field(const Geo& g, const Dev& d, cudaStream_t s) {
  k_far_field<<<1, g.P <= 128 ? 128 : 256, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ dipole, self term
// M = sum q r over user-order positions: KMC_DIP_BLOCKS blocks each sum a
// fixed strided subset (tree within the block), then one block adds the
// partial sums in block order -- a fixed order, so M is deterministic
__global__ void __launch_bounds__(256) k_dipole_part(const Geo g, const Dev d) {
  __shared__ double sh[3][256];
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double q = d.q[i];
    a0 += q * d.pos[3 * i];
    a1 += q * d.pos[3 * i + 1];
    a2 += q * d.pos[3 * i + 2];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int c = 0; c < 3; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 3) d.dip_part[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_dipole(const Geo g, const Dev d) {
  if (threadIdx.x >= 3) return;
  double a = 0.0;
  for (int b = 0; b < KMC_DIP_BLOCKS; b++) a += d.dip_part[3 * b + threadIdx.x];
  d.dip[threadIdx.x] = a;
  d.fdip[threadIdx.x] = (float)(g.dipc * a);
}

// C(d) = sum_{nu in V} 1/|d - a nu| - sum_{nu in V, nu != 0} 1/|a nu| + g(d) - g(0) + 2 pi |d|^2 / (3V)
// with V the near block |nu|_inf <= KMC_TOP and g(d) = Re sum conj(S_n^m) R_n^m(d) (n <= p): the
// moving charge's interaction with its own images, equal to psi(d) - psi_reg(0)
// of the tinfoil pair potential.
__device__ double self_corr_dev(const Geo& g, const double2* S, double dx, double dy, double dz) {
  if (g.bc) return 1.0 / sqrt(dx * dx + dy * dy + dz * dz);  // free space: the direct pair alone
  double s = 0.0;
  for (int a = -KMC_TOP; a <= KMC_TOP; a++)
    for (int b = -KMC_TOP; b <= KMC_TOP; b++)
      for (int c = -KMC_TOP; c <= KMC_TOP; c++) {
        double x = dx - g.a * a, y = dy - g.a * b, z = dz - g.a * c;
        s += 1.0 / sqrt(x * x + y * y + z * z);
        if (a || b || c) s -= 1.0 / (g.a * sqrt((double)(a * a + b * b + c * c)));
      }
  // g(d) - g(0): accumulate the regular harmonics along each m column
  double r2 = dx * dx + dy * dy + dz * dz;
  double2 mm = make_double2(1.0, 0.0);
  double gd = 0.0;
  for (int m = 0; m <= g.p; m++) {
    if (m > 0) {
      double sc = -0.5 / m;
      mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
    }
    double2 a2 = make_double2(0.0, 0.0), a1 = mm;
    double col = 0.0;
    for (int n = m; n <= g.p; n++) {
      double2 v;
      if (n == m) v = mm;
      else {
        double cc = f_inv_nm[tri(n, m)];
        double zz = (2 * n - 1) * dz;
        v = make_double2((zz * a1.x - r2 * a2.x) * cc, (zz * a1.y - r2 * a2.y) * cc);
        a2 = a1;
        a1 = v;
      }
      if (n == 0) continue;  // the constant term cancels in g(d) - g(0)
      double2 sv = S[tri(n, m)];
      col += sv.x * v.x + sv.y * v.y;  // Re(conj(S) R)
    }
    gd += (m == 0 ? 1.0 : 2.0) * col;
  }
  double V = g.a * g.a * g.a;
  return s + gd + 2.0 * M_PI / (3.0 * V) * r2;
}

__global__ void k_selfcorr(const Geo g, const Dev d) {
  int k = threadIdx.x;
  if (k >= (g.nhop > 0 ? g.nhop : KMC_NHOP)) return;
  double h = (g.E > 0) ? g.h : 1.0;
  const double dx = hop_c(k, 0) * h, dy = hop_c(k, 1) * h, dz = hop_c(k, 2) * h;
  double c = self_corr_dev(g, d.S, dx, dy, dz);
  d.selfc[k] = c;
  if (d.selfc32) d.selfc32[k] = (float)c;
}

// Dirichlet walls: the C(d) values the mirror terms of a hop need (d between a
// charge or its hop target and a mirror; all z-only or hop-shaped, so tabulated
// per z-site of the physical half)
__global__ void k_dirichlet_tables(const Geo g, const Dev d) {
  const int half = g.E / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= half * (1 + g.nhop)) return;
  double dx = 0.0, dy = 0.0, dz;
  if (t < half) {
    dz = (2.0 * t + 1.0 - g.E) * g.h;
  } else {
    const int k = (t - half) / half, z = (t - half) % half;
    dx = hop_c(k, 0) * g.h;
    dy = hop_c(k, 1) * g.h;
    dz = (2.0 * z + hop_c(k, 2) + 1.0 - g.E) * g.h;
  }
  const double c = self_corr_dev(g, d.S, dx, dy, dz);
  if (t < half) {
    d.dirA[t] = c;
    if (d.dirA32) d.dirA32[t] = (float)c;
  } else {
    d.dirB[t - half] = c;
    if (d.dirB32) d.dirB32[t - half] = (float)c;
  }
}

void fmm_dirichlet_tables(const Geo& g, const Dev& d, cudaStream_t s) {
  const int nt = (g.E / 2) * (1 + g.nhop);
  k_dirichlet_tables<<<(nt + 127) / 128, 128, 0, s>>>(g, d);
}

void fmm_self_and_dipole(const Geo& g, const Dev& d, cudaStream_t s) {
  k_dipole_part<<<KMC_DIP_BLOCKS, 256, 0, s>>>(g, d);
  k_dipole<<<1, 32, 0, s>>>(g, d);
  k_selfcorr<<<1, 32, 0, s>>>(g, d);
}

// general-d self correction used by the off-lattice assembly
__global__ void k_selfcorr_list(const Geo g, const double2* S, int64_t m, const double* dvec, double* out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  out[t] = self_corr_dev(g, S, dvec[3 * t], dvec[3 * t + 1], dvec[3 * t + 2]);
}

void fmm_selfcorr_list(const Geo& g, const Dev& d, int64_t m, const double* dvec, double* out, cudaStream_t s) {
  k_selfcorr_list<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(g, d.S, m, dvec, out);
}

// FP32 shadow of every per-level local expansion (after a full FMM)
__global__ void k_shadow_all(const double2* a, float2* b, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

void fmm_shadow_all(const Geo& g, const Dev& d, cudaStream_t s) {
  if (!d.Psi32) return;
  k_shadow_all<<<1024, 256, 0, s>>>(d.Psi, d.Psi32, g.ncell_total * g.P);
}

// ------------------------------------------------------------------ downward pass
// Peff_1 = H; Peff_l[b] = L2L(Peff_{l-1}[parent] -> c_b) + Psi_l[b]   (precision T)
// One CTA per parent cell computes all 8 children: the parent expansion and
// the 8 child-offset harmonic tables sit in shared memory.
__constant__ short2 f_nm[ncoef(KMC_MAXP)];  // (n, m) of coefficient index tri(n, m)

void fmm_upload_nm() {
  static short2 nm[ncoef(KMC_MAXP)];
  for (int n = 0; n <= KMC_MAXP; n++)
    for (int m = 0; m <= n; m++) nm[tri(n, m)] = make_short2((short)n, (short)m);
  cudaMemcpyToSymbol(f_nm, nm, sizeof(nm));
}

// the level's own per-level expansion in precision T (FP32 shadow in the mixed form)
template <typename T> __device__ __forceinline__ typename cplx<T>::type own_coef(const Dev& d, int64_t idx);
template <> __device__ __forceinline__ float2 own_coef<float>(const Dev& d, int64_t idx) { return d.Psi32[idx]; }
template <> __device__ __forceinline__ double2 own_coef<double>(const Dev& d, int64_t idx) { return d.Psi[idx]; }
template <typename T> __device__ __forceinline__ typename cplx<T>::type child_coef(const Dev& d, int64_t idx);
template <> __device__ __forceinline__ float2 child_coef<float>(const Dev& d, int64_t idx) { return d.Rch32[idx]; }
template <> __device__ __forceinline__ double2 child_coef<double>(const Dev& d, int64_t idx) { return d.Rch[idx]; }


template <typename T> __device__ __forceinline__ const typename cplx<T>::type* child_table(const Dev& d);
template <> __device__ __forceinline__ const float2* child_table<float>(const Dev& d) { return d.Rch32; }
template <> __device__ __forceinline__ const double2* child_table<double>(const Dev& d) { return d.Rch; }


// Downward pass of the levels with few cells, 2 .. lc, in one launch (CTA per
// cell, thread per output coefficient).  The expansion of cell b on level l is
// the sum over its ancestors a on levels 1 .. l - 1 (level 1: H) of the L2L of
// their interaction-list expansions to its centre, plus its own:
//   Peff_l[b] = Psi_l[b] + sum_{l' < l} L2L(Psi_l'[a_l'(b)] -> c_b).
// The L2L of a degree-p local expansion is exact and L2L(a -> b) L2L(c -> a) =
// L2L(c -> b), so this equals the level-by-level recursion up to rounding,
// without one dependent launch per level.  The offset tables R(c_b - c_a) are
// built at init (k_coarse_tables), one per position of b inside a.
template <typename T> __device__ __forceinline__ const typename cplx<T>::type* own_ptr(const Dev& d);
template <> __device__ __forceinline__ const float2* own_ptr<float>(const Dev& d) { return d.Psi32; }
template <> __device__ __forceinline__ const double2* own_ptr<double>(const Dev& d) { return d.Psi; }

#define DC_PER 3  // output coefficients per thread: 128 threads cover P <= 384
template <typename T> __device__ __forceinline__ const typename cplx<T>::type* coarse_tab(const Dev& d);
template <> __device__ __forceinline__ const float2* coarse_tab<float>(const Dev& d) { return d.Rcoarse32; }
template <> __device__ __forceinline__ const double2* coarse_tab<double>(const Dev& d) { return d.Rcoarse; }

template <typename T>
__device__ __forceinline__ void downward_coarse_blk(const Geo& g, const Dev& d, const int lc, const int blk0) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char shraw[];
  const int F = (g.p + 1) * (g.p + 1);
  C* Lf = (C*)shraw;  // [F] ancestor expansion, entry n^2 + n + m
  C* Rf = Lf + F;     // [F] offset table, same order
  int64_t b = (int64_t)blockIdx.x - blk0;
  int l = 2;
  while (l < lc && b >= ((int64_t)1 << (3 * (l - 1)))) {
    b -= (int64_t)1 << (3 * (l - 1));
    l++;
  }
  const int nl = 1 << (l - 1);
  const int bx = (int)(b % nl), by = (int)((b / nl) % nl), bz = (int)(b / ((int64_t)nl * nl));
  T ax[DC_PER], ay[DC_PER];
#pragma unroll
  for (int j = 0; j < DC_PER; j++) ax[j] = ay[j] = (T)0;
  const C* own = own_ptr<T>(d);
  for (int la = 1; la < l; la++) {
    const int na = 1 << (la - 1), sh = l - la;
    const int Ax = bx >> sh, Ay = by >> sh, Az = bz >> sh;
    const int64_t acell = Ax + (int64_t)na * (Ay + (int64_t)na * Az);
    const int k = 1 << sh;  // b's position inside a, k per axis
    const C* Ro = coarse_tab<T>(d) +
                  (int64_t)(coarse_table_base(l, la) + (bx & (k - 1)) + k * ((by & (k - 1)) + k * (bz & (k - 1)))) * g.P;
    __syncthreads();  // the previous ancestor's tables are consumed
    const C* Pa = own + (g.cell_off[la] + acell) * g.P;
    for (int t = threadIdx.x; t < F; t += blockDim.x) {
      const int n = (int)sqrtf((float)t + 0.5f), m = t - n * n - n;  // exact: sqrt(n^2 - 1/2) < n <= sqrt(n^2 + 1/2)
      Lf[t] = tab_get(Pa, n, m);
      Rf[t] = tab_get(Ro, n, m);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < DC_PER; j++) {
      const int ci = threadIdx.x + j * blockDim.x;
      if (ci >= g.P) break;
      const short2 km = f_nm[ci];
      const int k = km.x, lo = km.y;
      T sx = 0, sy = 0;
      for (int n = k; n <= g.p; n++) {
        const int jj = n - k;
        const int mlo = max(lo - jj, -n), mhi = min(lo + jj, n);
        const C* a = Lf + n * n + n;
        const C* r = Rf + jj * jj + jj - lo;
        for (int m = mlo; m <= mhi; m++) {
          const C u = a[m], v = r[m];
          sx += u.x * v.x - u.y * v.y;
          sy += u.x * v.y + u.y * v.x;
        }
      }
      ax[j] += sx;
      ay[j] += sy;
    }
  }
  C* Pe = (C*)d.Peff;
#pragma unroll
  for (int j = 0; j < DC_PER; j++) {
    const int ci = threadIdx.x + j * blockDim.x;
    if (ci >= g.P) break;
    const int64_t at = (g.cell_off[l] + b) * g.P + ci;
    const C o = own[at];
    C v;
    v.x = ax[j] + o.x;
    v.y = ay[j] + o.y;
    Pe[at] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_downward_coarse(const Geo g, const Dev d, int lc) {
  downward_coarse_blk<T>(g, d, lc, 0);
}

// level 1 of every member of a batch: H (the parent expansion of level 2)
template <typename T>
__global__ void k_downward_root_batch(const BatchRep* reps) {
  typedef typename cplx<T>::type C;
  const Geo& g = reps[blockIdx.x].g;
  const Dev& d = reps[blockIdx.x].d;
  C* Pe = (C*)d.Peff;
  const C* own = own_ptr<T>(d);
  for (int c = threadIdx.x; c < g.P; c += blockDim.x) Pe[g.cell_off[1] * g.P + c] = own[g.cell_off[1] * g.P + c];
}

// cells of levels 2 .. lc
static __host__ __device__ __forceinline__ int64_t coarse_cells(int lc) {
  int64_t n = 0;
  for (int l = 2; l <= lc; l++) n += (int64_t)1 << (3 * (l - 1));
  return n;
}
size_t fmm_coarse_smem(int p, int prec) {
  const int F = (p + 1) * (p + 1);
  return 2 * (size_t)F * (prec == 0 ? sizeof(double2) : sizeof(float2));
}

// Downward pass, one level per launch: CTA per parent cell of level l - 1,
// computing its 8 children.  The parent's expansion and the 8 child-offset
// tables are expanded to every order -n..n in shared memory (the conjugate
// symmetry applied once).  A warp task is 4 consecutive output coefficients x
// the 8 children (lane = 8 c + o): the lanes of a warp run the same (or a
// neighbouring) degree's loop bounds, so the sums do not diverge, and each
// parent coefficient read is shared by 8 lanes.  Tasks go to warps in snake
// order (their cost falls with the degree).
template <typename T>
__device__ __forceinline__ void downward_par_blk(const Geo& g, const Dev& d, const int l, const int blk0) {
  typedef typename cplx<T>::type C;
  extern __shared__ __align__(16) unsigned char shraw[];
  const int F = (g.p + 1) * (g.p + 1);
  C* Lf = (C*)shraw;  // [F] parent expansion, entry n^2 + n + m
  C* Rf = Lf + F;     // [8][F] child-offset tables, same order
  const int nl = 1 << (l - 1), np = nl >> 1, sh = l - 2;  // np = 2^(l-2)
  const int64_t par = (int64_t)blockIdx.x - blk0;
  const int px = (int)(par & (np - 1)), py = (int)((par >> sh) & (np - 1)), pz = (int)(par >> (2 * sh));
  const C* Pp = (const C*)d.Peff + (g.cell_off[l - 1] + par) * g.P;
  const C* Rt = child_table<T>(d) + (int64_t)l * 8 * g.P;
  for (int t = threadIdx.x; t < 9 * F; t += blockDim.x) {
    const int tb = t / F, u = t - tb * F;
    const int n = (int)sqrtf((float)u + 0.5f), m = u - n * n - n;  // exact: sqrt(n^2 - 1/2) < n <= sqrt(n^2 + 1/2)
    if (tb == 0) Lf[u] = tab_get(Pp, n, m);
    else Rf[(tb - 1) * F + u] = tab_get(Rt + (tb - 1) * g.P, n, m);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int o = lane & 7, cl = lane >> 3;
  const int64_t child = (2 * px + (o & 1)) + (int64_t)nl * ((2 * py + ((o >> 1) & 1)) + (int64_t)nl * (2 * pz + (o >> 2)));
  const C* Ro = Rf + o * F;
  C* Pe = (C*)d.Peff;
  const int ntask = (g.P + 3) / 4;
  for (int r = 0; r * nw < ntask; r++) {
    const int task = r * nw + ((r & 1) ? nw - 1 - warp : warp);
    const int ci = 4 * task + cl;
    if (task >= ntask || ci >= g.P) continue;
    const short2 km = f_nm[ci];
    const int k = km.x, lo = km.y;
    T ax = 0, ay = 0;
    for (int n = k; n <= g.p; n++) {
      const int j = n - k;
      const int mlo = max(lo - j, -n), mhi = min(lo + j, n);
      const C* a = Lf + n * n + n;
      const C* b = Ro + j * j + j - lo;
      for (int m = mlo; m <= mhi; m++) {
        const C u = a[m], v = b[m];
        ax += u.x * v.x - u.y * v.y;
        ay += u.x * v.y + u.y * v.x;
      }
    }
    const int64_t at = (g.cell_off[l] + child) * g.P + ci;
    const C own = own_coef<T>(d, at);
    C v;
    v.x = ax + own.x;
    v.y = ay + own.y;
    Pe[at] = v;
    if (sizeof(T) == 4 && d.l2lA && l == g.L - 1) {  // the next level's tensor-core operand: hi / lo planes
      const int K = l2l_K(g.P);
      const int64_t at2 = l2l_sw_off(child, 2 * ci, 128, K / 32), plane = l2l_npad(g.L) * K;
      const float x = (float)v.x, y = (float)v.y, hx = l2l_tf32(x), hy = l2l_tf32(y);
      *(float2*)(d.l2lA + at2) = make_float2(hx, hy);  // columns 2 ci, 2 ci + 1: one 8-byte pair
      *(float2*)(d.l2lA + plane + at2) = make_float2(l2l_tf32(x - hx), l2l_tf32(y - hy));
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_downward_par(const Geo g, const Dev d, int l) {
  downward_par_blk<T>(g, d, l, 0);
}

// level l of every member of a batch that has it (blocks of member r: its parent cells)
template <typename T>
__global__ void __launch_bounds__(256) k_downward_par_batch(const BatchRep* reps, const int* off, int R, int l) {
  const int r = batch_find(off, R, blockIdx.x);
  downward_par_blk<T>(reps[r].g, reps[r].d, l, off[r]);
}


void fmm_prepare(const Geo& g, int prec) {
  // load every per-step kernel now: with lazy module loading a first launch
  // inside a stream capture would invalidate the capture
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_downward_par<double>);
  cudaFuncGetAttributes(&fa, k_downward_par<float>);
  const int smax = 9 * (KMC_MAXP + 1) * (KMC_MAXP + 1) * (int)sizeof(double2);
  cudaFuncSetAttribute(k_downward_par<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  cudaFuncSetAttribute(k_downward_par<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax / 2);
  const int csm = (int)fmm_coarse_smem(KMC_MAXP, 0);
  cudaFuncSetAttribute(k_downward_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, csm);
  cudaFuncSetAttribute(k_downward_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, csm);
  cudaFuncGetAttributes(&fa, k_downward_root_batch<double>);
  cudaFuncGetAttributes(&fa, k_downward_root_batch<float>);
  cudaFuncSetAttribute(k_downward_par_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  cudaFuncSetAttribute(k_downward_par_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax / 2);
  (void)g;
  (void)prec;
}

// the levels with fewer than 512 parents (2 .. 4) in one launch, the rest one launch per level
static int coarse_top(int L) { return L < KMC_DOWN_COARSE ? L : KMC_DOWN_COARSE; }

void fmm_downward(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  const int lc = coarse_top(g.L);
  const size_t smc = fmm_coarse_smem(g.p, prec);
  const size_t smp = (size_t)9 * (g.p + 1) * (g.p + 1) * (prec == 0 ? sizeof(double2) : sizeof(float2));
  if (prec == 0) k_downward_coarse<double><<<(unsigned)coarse_cells(lc), 128, smc, s>>>(g, d, lc);
  else k_downward_coarse<float><<<(unsigned)coarse_cells(lc), 128, smc, s>>>(g, d, lc);
  for (int l = lc + 1; l <= g.L; l++) {
    const unsigned parents = 1u << (3 * (l - 2));
    if (prec == 1 && fmm_l2l_tc(g, d, l, s)) continue;  // the finest levels on the tensor cores
    if (prec == 0) k_downward_par<double><<<parents, 256, smp, s>>>(g, d, l);
    else k_downward_par<float><<<parents, 256, smp, s>>>(g, d, l);
  }
}

// downward pass of every member of a batch: H into level 1, then one launch
// per level (members with fewer levels take no blocks of the deeper launches)
void fmm_downward_batch(const BatchPlan& bp, cudaStream_t s) {
  if (bp.prec == 0) k_downward_root_batch<double><<<bp.R, 128, 0, s>>>(bp.reps);
  else k_downward_root_batch<float><<<bp.R, 128, 0, s>>>(bp.reps);
  for (int l = 2; l <= bp.Lmax; l++) {
    if (bp.nblk_down[l] <= 0) continue;
    if (bp.prec == 0)
      k_downward_par_batch<double><<<bp.nblk_down[l], 256, bp.smem_down, s>>>(bp.reps, bp.off_down[l], bp.R, l);
    else
      k_downward_par_batch<float><<<bp.nblk_down[l], 256, bp.smem_down, s>>>(bp.reps, bp.off_down[l], bp.R, l);
  }
}

// ------------------------------------------------------------------ drift
// out2[0] = max |a - b|, out2[1] = max |b| (as non-negative doubles via integer max)
__global__ void k_drift(const double2* a, const double2* b, int64_t count, unsigned long long* out2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0.0, m = 0.0;
  for (; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double2 x = a[i], y = b[i];
    e = fmax(e, fmax(fabs(x.x - y.x), fabs(x.y - y.y)));
    m = fmax(m, fmax(fabs(y.x), fabs(y.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    e = fmax(e, __shfl_xor_sync(0xffffffff, e, o));
    m = fmax(m, __shfl_xor_sync(0xffffffff, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out2[0], (unsigned long long)__double_as_longlong(e));
    atomicMax(&out2[1], (unsigned long long)__double_as_longlong(m));
  }
}

void fmm_drift(const Geo& g, const double2* a, const double2* b, int64_t count, double* out2, cudaStream_t s) {
  (void)g;
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), s);
  k_drift<<<1024, 256, 0, s>>>(a, b, count, (unsigned long long*)out2);
}

// out2[0] = max |a - b|, out2[1] = max |b| over real arrays
__global__ void k_drift1(const double* a, const double* b, int64_t count, unsigned long long* out2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0.0, m = 0.0;
  for (; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    e = fmax(e, fabs(a[i] - b[i]));
    m = fmax(m, fabs(b[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    e = fmax(e, __shfl_xor_sync(0xffffffff, e, o));
    m = fmax(m, __shfl_xor_sync(0xffffffff, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out2[0], (unsigned long long)__double_as_longlong(e));
    atomicMax(&out2[1], (unsigned long long)__double_as_longlong(m));
  }
}

void fmm_drift1(const double* a, const double* b, int64_t count, double* out2, cudaStream_t s) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), s);
  k_drift1<<<1024, 256, 0, s>>>(a, b, count, (unsigned long long*)out2);
}
