// kmc_kernels.cu -- the per-step hot path of FMM-for-KMC on sm_103a:
//   propose  (Sec. 3, Eq. (proposed_energy); periodic form Eq. (proposed_energy_sr))
//   rates, scan and selection  (Algorithm 1)
//   accept   (Sec. 3 "Accept move", per-level form)
//
// dU of a hop of charge q from r to r' (both in the primary cell, d = r' - r)
// is assembled as
//   dU = q [Phi(r') - Phi_self(r)] - (4 pi / 3V) q M.d - q^2 C(d_min)
// where Phi is the potential of all charges and of their images in cubic
// summation order (leaf local expansion from the downward pass plus the
// direct sum over the 27 neighbouring leaves, Fig. "fmm_point_eval"),
// Phi_self omits the singular own term, M is the cell dipole, and
// C(d) = psi(d) - psi_reg(0) is the moving charge's interaction with its own
// images (the 19.104/a self-image term of Eq. (proposed_energy_sr) and its
// far-field part).  The M.d term and the |d|^2 part of C together are the
// change of the surface term that the dipole correction of Sec. 2.2.2 removes.
#include <math.h>
#include <stdio.h>

#include "common.cuh"

__constant__ float c_inv_f[KMC_NTRI];
__constant__ double c_inv_d[KMC_NTRI];
__constant__ float c_halfm_f[KMC_MAXP + 2];   // -1/(2m)
__constant__ double c_halfm_d[KMC_MAXP + 2];
__constant__ int c_hop[KMC_NHOP][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

void kmc_upload_constants(int p) {
  static float invf[KMC_NTRI];
  static double invd[KMC_NTRI];
  static float hf[KMC_MAXP + 2];
  static double hd[KMC_MAXP + 2];
  for (int n = 0; n <= 2 * KMC_MAXP; n++)
    for (int m = 0; m <= n; m++) {
      double v = (n > m) ? 1.0 / ((double)(n - m) * (double)(n + m)) : 0.0;
      invd[tri(n, m)] = v;
      invf[tri(n, m)] = (float)v;
    }
  hd[0] = 0.0;
  hf[0] = 0.0f;
  for (int m = 1; m < KMC_MAXP + 2; m++) {
    hd[m] = -0.5 / m;
    hf[m] = (float)(-0.5 / m);
  }
  cudaMemcpyToSymbol(c_inv_f, invf, sizeof(invf));
  cudaMemcpyToSymbol(c_inv_d, invd, sizeof(invd));
  cudaMemcpyToSymbol(c_halfm_f, hf, sizeof(hf));
  cudaMemcpyToSymbol(c_halfm_d, hd, sizeof(hd));
  (void)p;
}

template <typename T> __device__ __forceinline__ T inv_nm(int i);
template <> __device__ __forceinline__ float inv_nm<float>(int i) { return c_inv_f[i]; }
template <> __device__ __forceinline__ double inv_nm<double>(int i) { return c_inv_d[i]; }
template <typename T> __device__ __forceinline__ T halfm(int m);
template <> __device__ __forceinline__ float halfm<float>(int m) { return c_halfm_f[m]; }
template <> __device__ __forceinline__ double halfm<double>(int m) { return c_halfm_d[m]; }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// L2P: Re sum_{n,m} L_n^m R_n^m(x), x relative to the expansion centre.
template <typename T, typename C>
__device__ __forceinline__ T l2p_eval(const C* L, int p, T x, T y, T z) {
  T r2 = x * x + y * y + z * z;
  T mmx = 1, mmy = 0;
  T acc = 0;
  for (int m = 0; m <= p; m++) {
    if (m > 0) {
      T s = halfm<T>(m);
      T tx = s * (x * mmx - y * mmy);
      T ty = s * (x * mmy + y * mmx);
      mmx = tx;
      mmy = ty;
    }
    C lv = L[tri(m, m)];
    T col = lv.x * mmx - lv.y * mmy;
    T a1x = mmx, a1y = mmy, a2x = 0, a2y = 0;
    T zz = (T)(2 * m + 1) * z;
    T z2 = z + z;
    for (int n = m + 1; n <= p; n++) {
      T c = inv_nm<T>(tri(n, m));
      T vx = (zz * a1x - r2 * a2x) * c;
      T vy = (zz * a1y - r2 * a2y) * c;
      lv = L[tri(n, m)];
      col += lv.x * vx - lv.y * vy;
      a2x = a1x; a2y = a1y;
      a1x = vx; a1y = vy;
      zz += z2;
    }
    acc += (m == 0) ? col : col + col;
  }
  return acc;
}

// ------------------------------------------------------------------ propose (lattice)
// One CTA per leaf cell.  Evaluation points of the CTA are every position in
// the leaf at which a potential is needed: the leaf's own charges (old
// positions, own charge excluded) and every unmasked hop target that lies in
// the leaf, whether the hopping charge sits in this leaf or in one of its six
// face neighbours.  Sources are the charges of the 27 neighbouring leaves
// (periodically wrapped images), staged in shared memory.
struct PtRec {
  uint32_t a;  // local site index (bits 0..15), hop k (16..18), old flag (bit 19)
  int32_t u;   // user index of the hopping charge
};

#define PROP_THREADS 128

template <typename T>
__global__ void __launch_bounds__(PROP_THREADS) k_propose_lattice(const Geo g, const Dev d, int pmax, int chunk) {
  typedef typename cplx<T>::type C;
  typedef typename vec4<T>::type V4;
  extern __shared__ __align__(32) unsigned char sm[];
  V4* src = (V4*)sm;
  C* Lc = (C*)(src + chunk);
  PtRec* pts = (PtRec*)(Lc + g.P);
  const int W = g.W, W3 = W * W * W;
  const int nbw = (W3 + 31) / 32;
  uint32_t* bits = (uint32_t*)(pts + pmax);
  int* ctr = (int*)(bits + nbw);  // [0] npts, [1..28] source prefix offsets

  const int tid = threadIdx.x;
  const int nL = g.nL, E = g.E;
  const int64_t leaf = blockIdx.x;
  const int lx = (int)(leaf % nL), ly = (int)((leaf / nL) % nL), lz = (int)(leaf / ((int64_t)nL * nL));
  const int gx0 = lx * W, gy0 = ly * W, gz0 = lz * W;
  const T h = (T)g.h;
  const V4* spos = (const V4*)((sizeof(T) == 4) ? (const void*)d.spos32 : (const void*)d.spos64);

  // leaf local expansion (downward-accumulated)
  const C* Pe = (const C*)d.Peff + (g.cell_off[g.L] + leaf) * g.P;
  for (int c = tid; c < g.P; c += blockDim.x) Lc[c] = Pe[c];
  for (int c = tid; c < nbw; c += blockDim.x) bits[c] = 0u;
  if (tid == 0) ctr[0] = 0;
  __syncthreads();

  // occupancy bitmap of this leaf's sites
  const int cnt_own = d.cnt[leaf];
  const int64_t base_own = leaf * g.cap;
  for (int j = tid; j < cnt_own; j += blockDim.x) {
    int32_t u = d.uid[base_own + j];
    int s = d.site[u];
    int sx = s % E - gx0, sy = (s / E) % E - gy0, sz = s / (E * E) - gz0;
    int ls = sx + W * (sy + W * sz);
    atomicOr(&bits[ls >> 5], 1u << (ls & 31));
  }
  __syncthreads();

  // evaluation points: own charges, own hops staying in the leaf
  for (int j = tid; j < cnt_own; j += blockDim.x) {
    int32_t u = d.uid[base_own + j];
    int s = d.site[u];
    int gx = s % E, gy = (s / E) % E, gz = s / (E * E);
    int ls = (gx - gx0) + W * ((gy - gy0) + W * (gz - gz0));
    int slot = atomicAdd(&ctr[0], 1);
    if (slot < pmax) pts[slot] = PtRec{(uint32_t)ls | (1u << 19), u};
    for (int k = 0; k < KMC_NHOP; k++) {
      int tx = gx + c_hop[k][0], ty = gy + c_hop[k][1], tz = gz + c_hop[k][2];
      tx = (tx + E) % E; ty = (ty + E) % E; tz = (tz + E) % E;
      int ux = tx - gx0, uy = ty - gy0, uz = tz - gz0;
      if (ux < 0 || ux >= W || uy < 0 || uy >= W || uz < 0 || uz >= W) continue;  // other leaf's CTA
      int lt = ux + W * (uy + W * uz);
      if (bits[lt >> 5] & (1u << (lt & 31))) {
        d.mask[6 * (int64_t)u + k] = 0;
        d.phi_new[6 * (int64_t)u + k] = __longlong_as_double(0x7ff8000000000000LL);
      } else {
        int sl = atomicAdd(&ctr[0], 1);
        if (sl < pmax) pts[sl] = PtRec{(uint32_t)lt | ((uint32_t)k << 16), u};
      }
    }
  }
  // hops entering from the six face neighbours
  for (int f = 0; f < KMC_NHOP; f++) {
    int mx = (lx + c_hop[f][0] + nL) % nL, my = (ly + c_hop[f][1] + nL) % nL, mz = (lz + c_hop[f][2] + nL) % nL;
    int64_t mu = mx + (int64_t)nL * (my + (int64_t)nL * mz);
    int kin = f ^ 1;  // direction from the neighbour back into this leaf
    int cm = d.cnt[mu];
    for (int j = tid; j < cm; j += blockDim.x) {
      int32_t u = d.uid[mu * g.cap + j];
      int s = d.site[u];
      int tx = s % E + c_hop[kin][0], ty = (s / E) % E + c_hop[kin][1], tz = s / (E * E) + c_hop[kin][2];
      tx = (tx + E) % E; ty = (ty + E) % E; tz = (tz + E) % E;
      int ux = tx - gx0, uy = ty - gy0, uz = tz - gz0;
      if (ux < 0 || ux >= W || uy < 0 || uy >= W || uz < 0 || uz >= W) continue;
      int lt = ux + W * (uy + W * uz);
      if (bits[lt >> 5] & (1u << (lt & 31))) {
        d.mask[6 * (int64_t)u + kin] = 0;
        d.phi_new[6 * (int64_t)u + kin] = __longlong_as_double(0x7ff8000000000000LL);
      } else {
        int sl = atomicAdd(&ctr[0], 1);
        if (sl < pmax) pts[sl] = PtRec{(uint32_t)lt | ((uint32_t)kin << 16), u};
      }
    }
  }
  // source offsets of the 26 other neighbour leaves (fixed order)
  if (tid == 0) {
    int off = 0, q = 0;
    for (int oz = -1; oz <= 1; oz++)
      for (int oy = -1; oy <= 1; oy++)
        for (int ox = -1; ox <= 1; ox++) {
          if (!ox && !oy && !oz) continue;
          int sx = (lx + ox + nL) % nL, sy = (ly + oy + nL) % nL, sz = (lz + oz + nL) % nL;
          ctr[1 + q] = off;
          off += d.cnt[sx + (int64_t)nL * (sy + (int64_t)nL * sz)];
          q++;
        }
    ctr[27] = off;
  }
  __syncthreads();
  int npts = ctr[0];
  if (npts > pmax) {
    if (tid == 0) atomicOr(&d.err[0], KMC_DERR_CAPACITY);
    npts = pmax;
  }

  // ---- near-field pair sums, then L2P.  Points are processed in rounds of
  // 2 * blockDim (two per thread, accumulators in registers); each round
  // streams the sources: pass 0 = own leaf (self pair skipped by r2 > 0),
  // passes 1.. = the 26 other leaves in chunks.
  const int nsrc_other = ctr[27];
  const int npass = 1 + (nsrc_other + chunk - 1) / chunk;
  for (int rb = 0; rb < npts; rb += 2 * blockDim.x) {
    const int b0 = rb + tid, b1 = rb + tid + blockDim.x;
    T x0 = (T)1e18, y0 = (T)1e18, z0 = (T)1e18, x1 = (T)1e18, y1 = (T)1e18, z1 = (T)1e18;
    if (b0 < npts) {
      int l0 = pts[b0].a & 0xffff;
      x0 = ((T)(gx0 + l0 % W) + (T)0.5) * h;
      y0 = ((T)(gy0 + (l0 / W) % W) + (T)0.5) * h;
      z0 = ((T)(gz0 + l0 / (W * W)) + (T)0.5) * h;
    }
    if (b1 < npts) {
      int l1 = pts[b1].a & 0xffff;
      x1 = ((T)(gx0 + l1 % W) + (T)0.5) * h;
      y1 = ((T)(gy0 + (l1 / W) % W) + (T)0.5) * h;
      z1 = ((T)(gz0 + l1 / (W * W)) + (T)0.5) * h;
    }
    T s0 = 0, s1 = 0;
    for (int pass = 0; pass < npass; pass++) {
      __syncthreads();
      int ns;
      if (pass == 0) {
        ns = cnt_own;
        for (int j = tid; j < ns; j += blockDim.x) src[j] = spos[base_own + j];
      } else {
        int c0 = (pass - 1) * chunk;
        ns = min(chunk, nsrc_other - c0);
        for (int e = tid; e < ns; e += blockDim.x) {
          int ge = c0 + e;
          int q = 0;
          while (q < 25 && ctr[2 + q] <= ge) q++;
          int qq = q >= 13 ? q + 1 : q;  // skip the centre in the 27-neighbourhood order
          int ox = qq % 3 - 1, oy = (qq / 3) % 3 - 1, oz = qq / 9 - 1;
          int ux = lx + ox, uy = ly + oy, uz = lz + oz;
          int sx = (ux + nL) % nL, sy = (uy + nL) % nL, sz = (uz + nL) % nL;
          int64_t sl = (sx + (int64_t)nL * (sy + (int64_t)nL * sz)) * g.cap + (ge - ctr[1 + q]);
          V4 v = spos[sl];
          v.x += (T)((ux - sx) * W) * h;
          v.y += (T)((uy - sy) * W) * h;
          v.z += (T)((uz - sz) * W) * h;
          src[e] = v;
        }
      }
      __syncthreads();
      if (pass == 0) {
        for (int j = 0; j < ns; j++) {
          V4 v = src[j];
          T dx0 = v.x - x0, dy0 = v.y - y0, dz0 = v.z - z0;
          T dx1 = v.x - x1, dy1 = v.y - y1, dz1 = v.z - z1;
          T q0 = dx0 * dx0 + dy0 * dy0 + dz0 * dz0;
          T q1 = dx1 * dx1 + dy1 * dy1 + dz1 * dz1;
          T i0 = q0 > (T)0 ? rsq(q0) : (T)0;
          T i1 = q1 > (T)0 ? rsq(q1) : (T)0;
          s0 += v.w * i0;
          s1 += v.w * i1;
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < ns; j++) {
          V4 v = src[j];
          T dx0 = v.x - x0, dy0 = v.y - y0, dz0 = v.z - z0;
          T dx1 = v.x - x1, dy1 = v.y - y1, dz1 = v.z - z1;
          T q0 = dx0 * dx0 + dy0 * dy0 + dz0 * dz0;
          T q1 = dx1 * dx1 + dy1 * dy1 + dz1 * dz1;
          s0 += v.w * rsq(q0);
          s1 += v.w * rsq(q1);
        }
      }
    }
    // L2P of the leaf local expansion and write-out
    for (int side = 0; side < 2; side++) {
      int b = side ? b1 : b0;
      if (b >= npts) continue;
      PtRec r = pts[b];
      int lt = r.a & 0xffff;
      T x = ((T)(lt % W) + (T)0.5 - (T)(0.5 * W)) * h;
      T y = ((T)((lt / W) % W) + (T)0.5 - (T)(0.5 * W)) * h;
      T z = ((T)(lt / (W * W)) + (T)0.5 - (T)(0.5 * W)) * h;
      T v = (side ? s1 : s0) + l2p_eval<T, C>(Lc, g.p, x, y, z);
      if (r.a & (1u << 19)) {
        d.phi_old[r.u] = (double)v;
      } else {
        int k = (r.a >> 16) & 7;
        d.phi_new[6 * (int64_t)r.u + k] = (double)v;
        d.mask[6 * (int64_t)r.u + k] = 1;
      }
    }
  }
}

static size_t propose_smem(const Geo& g, int prec, int pmax, int chunk) {
  size_t ts = prec == 0 ? 8 : 4;
  int nbw = (g.W * g.W * g.W + 31) / 32;
  return 4 * ts * (size_t)chunk + 2 * ts * (size_t)g.P + 8 * (size_t)pmax + 4 * (size_t)nbw + 4 * 32;
}

static void propose_shape(const Geo& g, int* pmax, int* chunk) {
  int W3 = g.W * g.W * g.W;
  *pmax = W3 + 6 * W3 + 6 * g.W * g.W;  // every own charge, its hops, every entering hop
  *chunk = 1024 > g.cap ? 1024 : g.cap;
}

void kmc_prepare(const Geo& g, int prec) {
  if (g.E <= 0) return;
  int pmax, chunk;
  propose_shape(g, &pmax, &chunk);
  size_t sm = propose_smem(g, prec, pmax, chunk);
  if (prec == 0) cudaFuncSetAttribute(k_propose_lattice<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  else cudaFuncSetAttribute(k_propose_lattice<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

void kmc_propose_lattice(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  int pmax, chunk;
  propose_shape(g, &pmax, &chunk);
  size_t sm = propose_smem(g, prec, pmax, chunk);
  if (prec == 0) k_propose_lattice<double><<<(unsigned)g.ML, PROP_THREADS, sm, s>>>(g, d, pmax, chunk);
  else k_propose_lattice<float><<<(unsigned)g.ML, PROP_THREADS, sm, s>>>(g, d, pmax, chunk);
}

// ------------------------------------------------------------------ dU, rates, block sums
// thread per particle; FP64 assembly.  Block sums are sequential over the
// block's threads so that the selection walk reproduces them exactly.
#define FIN_THREADS 256
__global__ void __launch_bounds__(FIN_THREADS) k_finalize(const Geo g, const Dev d) {
  __shared__ double ts[FIN_THREADS];
  int64_t i = blockIdx.x * (int64_t)FIN_THREADS + threadIdx.x;
  double tsum = 0.0;
  if (i < g.n) {
    const double q = d.q[i];
    const int E = g.E;
    const int s = d.site[i];
    const int gx = s % E, gy = (s / E) % E, gz = s / (E * E);
    const double V = g.a * g.a * g.a;
    const double cdip = 4.0 * M_PI / (3.0 * V) * q;
    const double po = d.phi_old[i];
    const double M0 = d.dip[0], M1 = d.dip[1], M2 = d.dip[2];
    for (int k = 0; k < KMC_NHOP; k++) {
      int64_t j = 6 * i + k;
      double du, r;
      if (!d.mask[j]) {
        du = __longlong_as_double(0x7ff8000000000000LL);
        r = 0.0;
      } else {
        int tx = gx + c_hop[k][0], ty = gy + c_hop[k][1], tz = gz + c_hop[k][2];
        double dx = c_hop[k][0] * g.h, dy = c_hop[k][1] * g.h, dz = c_hop[k][2] * g.h;
        if (tx < 0) dx += g.a; else if (tx >= E) dx -= g.a;
        if (ty < 0) dy += g.a; else if (ty >= E) dy -= g.a;
        if (tz < 0) dz += g.a; else if (tz >= E) dz -= g.a;
        du = q * (d.phi_new[j] - po) - cdip * (M0 * dx + M1 * dy + M2 * dz) - q * q * d.selfc[k];
        r = exp(-fmax(du, 0.0) / g.kT);
      }
      d.dU[j] = du;
      d.rate[j] = r;
      tsum += r;
    }
  }
  ts[threadIdx.x] = tsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int t = 0; t < FIN_THREADS; t++) b += ts[t];
    d.bsum[blockIdx.x] = b;
  }
}

// block sums of caller-provided rates (same block structure as k_finalize)
__global__ void __launch_bounds__(FIN_THREADS) k_rate_bsum(const Geo g, const Dev d) {
  __shared__ double ts[FIN_THREADS];
  int64_t i = blockIdx.x * (int64_t)FIN_THREADS + threadIdx.x;
  double tsum = 0.0;
  if (i < g.n)
    for (int k = 0; k < KMC_NHOP; k++) tsum += d.rate[6 * i + k];
  ts[threadIdx.x] = tsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int t = 0; t < FIN_THREADS; t++) b += ts[t];
    d.bsum[blockIdx.x] = b;
  }
}

void kmc_finalize_rates(const Geo& g, const Dev& d, cudaStream_t s) {
  unsigned nb = (unsigned)((g.n + FIN_THREADS - 1) / FIN_THREADS);
  k_finalize<<<nb, FIN_THREADS, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ selection
// Q = sum of all rates; event j with R_{j-1} < Q zeta <= R_j (Algorithm 1),
// where R is the cumulative sum taken block by block (block sums from the
// finalize kernel, chunks of block sums per thread here); dt = -ln(xi)/Q.
#define SEL_THREADS 1024
__global__ void __launch_bounds__(SEL_THREADS) k_select(const Geo g, const Dev d, int use_counter) {
  __shared__ double cs[SEL_THREADS];
  __shared__ double ts[FIN_THREADS];
  __shared__ double sh_res;
  __shared__ int64_t sh_blk;
  const int tid = threadIdx.x;
  const int64_t nb = (g.n + FIN_THREADS - 1) / FIN_THREADS;
  const int64_t per = (nb + SEL_THREADS - 1) / SEL_THREADS;
  const double* uni = use_counter ? d.uni_run + 2 * (int64_t)(*d.stepc) : d.uni_small;
  double zeta = uni[0];
  double xi = uni[1];
  double c = 0.0;
  for (int64_t b = tid * per; b < min(nb, (tid + 1) * per); b++) c += d.bsum[b];
  cs[tid] = c;
  __syncthreads();
  if (tid == 0) {
    double Q = 0.0;
    for (int t = 0; t < SEL_THREADS; t++) Q += cs[t];
    d.dtq[1] = Q;
    d.dtq[0] = (Q > 0.0) ? -log(xi) / Q : __longlong_as_double(0x7ff0000000000000LL);
    int64_t blk = -1;
    double res = 0.0;
    if (Q > 0.0) {
      double target = Q * zeta;
      double run = 0.0;
      int tsel = -1;
      for (int t = 0; t < SEL_THREADS; t++) {
        if (run + cs[t] >= target && cs[t] > 0.0) { tsel = t; break; }
        run += cs[t];
      }
      if (tsel < 0) {  // rounding at zeta = 1: last chunk with weight
        for (int t = SEL_THREADS - 1; t >= 0; t--)
          if (cs[t] > 0.0) { tsel = t; break; }
        run = 0.0;
        for (int t = 0; t < tsel; t++) run += cs[t];
        target = run + cs[tsel];
      }
      double r2 = run;
      int64_t bend = min(nb, (tsel + 1) * per);
      for (int64_t b = tsel * per; b < bend; b++) {
        double bs = d.bsum[b];
        if (bs > 0.0 && (r2 + bs >= target || b == bend - 1)) { blk = b; break; }
        r2 += bs;
      }
      if (blk < 0) {
        for (int64_t b = bend - 1; b >= tsel * per; b--)
          if (d.bsum[b] > 0.0) { blk = b; break; }
      }
      res = target - r2;
    }
    sh_blk = blk;
    sh_res = res;
  }
  __syncthreads();
  int64_t blk = sh_blk;
  if (blk < 0) {
    if (tid == 0) *d.event = -1;
    return;
  }
  if (tid < FIN_THREADS) {
    int64_t i = blk * FIN_THREADS + tid;
    double t = 0.0;
    if (i < g.n)
      for (int k = 0; k < KMC_NHOP; k++) t += d.rate[6 * i + k];
    ts[tid] = t;
  }
  __syncthreads();
  if (tid == 0) {
    double res = sh_res, run = 0.0;
    int tsel = -1;
    for (int t = 0; t < FIN_THREADS; t++) {
      if (ts[t] > 0.0 && run + ts[t] >= res) { tsel = t; break; }
      run += ts[t];
    }
    if (tsel < 0) {
      for (int t = FIN_THREADS - 1; t >= 0; t--)
        if (ts[t] > 0.0) { tsel = t; break; }
      run = 0.0;
      for (int t = 0; t < tsel; t++) run += ts[t];
      res = run + ts[tsel];
    }
    int64_t i = blk * FIN_THREADS + tsel;
    int ksel = -1;
    for (int k = 0; k < KMC_NHOP; k++) {
      double r = d.rate[6 * i + k];
      if (r > 0.0 && run + r >= res) { ksel = k; break; }
      run += r;
    }
    if (ksel < 0)
      for (int k = KMC_NHOP - 1; k >= 0; k--)
        if (d.rate[6 * i + k] > 0.0) { ksel = k; break; }
    *d.event = 6 * i + ksel;
  }
}

void kmc_rate_bsum(const Geo& g, const Dev& d, cudaStream_t s) {
  unsigned nb = (unsigned)((g.n + FIN_THREADS - 1) / FIN_THREADS);
  k_rate_bsum<<<nb, FIN_THREADS, 0, s>>>(g, d);
}

void kmc_select(const Geo& g, const Dev& d, int use_counter, cudaStream_t s) {
  k_select<<<1, SEL_THREADS, 0, s>>>(g, d, use_counter);
}

// store the step's event and dt, advance the device step counter
__global__ void k_record(const Dev d) {
  int st = *d.stepc;
  d.ev_hist[st] = *d.event;
  d.dt_hist[st] = d.dtq[0];
  *d.stepc = st + 1;
}

void kmc_record(const Geo& g, const Dev& d, cudaStream_t s) {
  (void)g;
  k_record<<<1, 1, 0, s>>>(d);
}

// ------------------------------------------------------------------ accept
// Move record from a lattice event index (device resident, no host sync).
__global__ void k_move_from_event(const Geo g, const Dev d) {
  MoveRec mv;
  int64_t j = *d.event;
  mv.valid = 0;
  if (j >= 0) {
    int64_t i = j / 6;
    int k = (int)(j - 6 * i);
    int E = g.E;
    int s = d.site[i];
    int gx = s % E, gy = (s / E) % E, gz = s / (E * E);
    int tx = (gx + c_hop[k][0] + E) % E, ty = (gy + c_hop[k][1] + E) % E, tz = (gz + c_hop[k][2] + E) % E;
    mv.valid = 1;
    mv.i = (int32_t)i;
    mv.site_old = s;
    mv.site_new = tx + E * (ty + E * tz);
    mv.q = d.q[i];
    mv.r[0] = d.pos[3 * i];
    mv.r[1] = d.pos[3 * i + 1];
    mv.r[2] = d.pos[3 * i + 2];
    mv.rn[0] = (tx + 0.5) * g.h;
    mv.rn[1] = (ty + 0.5) * g.h;
    mv.rn[2] = (tz + 0.5) * g.h;
    mv.dU = d.dU[j];
  }
  *d.move = mv;
}

void kmc_accept_from_event(const Geo& g, const Dev& d, cudaStream_t s) { k_move_from_event<<<1, 1, 0, s>>>(g, d); }

__device__ __forceinline__ int cell_coord(double x, double w, int n) {
  int c = (int)floor(x / w);
  return min(max(c, 0), n - 1);
}

// multipoles of the ancestors of the old and new positions, all levels:
// Mt_l[anc(r)] -= q R(r - c), Mt_l[anc(r')] += q R(r' - c).  thread per (level, m)
__global__ void k_acc_multipole(const Geo g, const Dev d) {
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int l = 1 + t / (g.p + 1), m = t % (g.p + 1);
  if (l > g.L) return;
  int nl = 1 << (l - 1);
  double wl = g.a / nl;
  for (int side = 0; side < 2; side++) {
    const double* x = side ? mv.rn : mv.r;
    double q = side ? mv.q : -mv.q;
    int cx = cell_coord(x[0], wl, nl), cy = cell_coord(x[1], wl, nl), cz = cell_coord(x[2], wl, nl);
    double dx = x[0] - (cx + 0.5) * wl, dy = x[1] - (cy + 0.5) * wl, dz = x[2] - (cz + 0.5) * wl;
    double r2 = dx * dx + dy * dy + dz * dz;
    double2 mm = make_double2(1.0, 0.0);
    for (int j = 1; j <= m; j++) {
      double sc = c_halfm_d[j];
      mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
    }
    double2* out = d.Mt + (g.cell_off[l] + cx + (int64_t)nl * (cy + (int64_t)nl * cz)) * g.P;
    double2 a1 = mm, a2 = make_double2(0.0, 0.0);
    out[tri(m, m)].x += q * mm.x;
    out[tri(m, m)].y += q * mm.y;
    for (int n = m + 1; n <= g.p; n++) {
      double cc = c_inv_d[tri(n, m)];
      double zz = (2 * n - 1) * dz;
      double2 v = make_double2((zz * a1.x - r2 * a2.x) * cc, (zz * a1.y - r2 * a2.y) * cc);
      out[tri(n, m)].x += q * v.x;
      out[tri(n, m)].y += q * v.y;
      a2 = a1;
      a1 = v;
    }
  }
}

// far field: H += R dK, dK = q [R(r' - c) - R(r - c)] about the domain centre
__global__ void k_acc_far(const Geo g, const Dev d) {
  extern __shared__ double2 dK[];
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  int tid = threadIdx.x;
  if (tid < g.p + 1) {
    int m = tid;
    double c = 0.5 * g.a;
    for (int side = 0; side < 2; side++) {
      const double* x = side ? mv.rn : mv.r;
      double q = side ? mv.q : -mv.q;
      double dx = x[0] - c, dy = x[1] - c, dz = x[2] - c;
      double r2 = dx * dx + dy * dy + dz * dz;
      double2 mm = make_double2(1.0, 0.0);
      for (int j = 1; j <= m; j++) {
        double sc = c_halfm_d[j];
        mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
      }
      double2 a1 = mm, a2 = make_double2(0.0, 0.0);
      double2 v = mm;
      for (int n = m; n <= g.p; n++) {
        if (n > m) {
          double cc = c_inv_d[tri(n, m)];
          double zz = (2 * n - 1) * dz;
          v = make_double2((zz * a1.x - r2 * a2.x) * cc, (zz * a1.y - r2 * a2.y) * cc);
          a2 = a1;
          a1 = v;
        }
        if (side == 0) dK[tri(n, m)] = make_double2(q * v.x, q * v.y);
        else { dK[tri(n, m)].x += q * v.x; dK[tri(n, m)].y += q * v.y; }
      }
    }
  }
  __syncthreads();
  if (tid >= g.P) return;
  int n = 0;
  while (tri(n + 1, 0) <= tid) n++;
  int m = tid - tri(n, 0);
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k <= g.p; k++) {
    double sgn = (k & 1) ? -1.0 : 1.0;
    for (int ll = -k; ll <= k; ll++) {
      double2 a = tab_get(dK, k, ll), b = tab_get(d.S, n + k, m + ll);
      acc.x += sgn * (a.x * b.x + a.y * b.y);
      acc.y += sgn * (a.y * b.x - a.x * b.y);
    }
  }
  double2* H = d.Psi + g.cell_off[1] * g.P;
  H[tid].x += acc.x;
  H[tid].y += acc.y;
}

// per-level interaction-list locals.  For level l, the candidate cells are the
// children of the (wrapped) 3x3x3 parent neighbourhoods of the old and new
// positions' parent cells; for each candidate b and each of the 27 images of
// both positions, the image (cell u) is added when it lies in IL(b):
// |floor(u/2) - floor(b/2)|_inf <= 1 and |u - b|_inf >= 2.  thread per
// (level, candidate, m); FP64 P2L  L_n^m += q conj(I_n^m(y - c_b)).
__device__ __forceinline__ int fdiv2(int u) { return (u >= 0) ? (u >> 1) : -((1 - u) >> 1); }
__device__ __forceinline__ int wdist(int a, int b, int n) {
  int t = ((a - b) % n + n) % n;
  return min(t, n - t);
}

__global__ void k_acc_locals(const Geo g, const Dev d) {
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  const int l = 2 + blockIdx.y;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int cand = t / (g.p + 1), m = t % (g.p + 1);
  if (cand >= 432) return;
  const int nl = 1 << (l - 1), np = nl >> 1;
  const double wl = g.a / nl;
  int side0 = cand / 216, rem = cand % 216;
  int di = rem >> 3, o = rem & 7;
  int dlt[3] = {di % 3 - 1, (di / 3) % 3 - 1, di / 9 - 1};
  for (int c = 0; c < 3; c++) {
    if (np == 1 && dlt[c] != 0) return;
    if (np == 2 && dlt[c] == -1) return;
  }
  const double* x0 = side0 ? mv.rn : mv.r;
  int P0[3], Pold[3];
  for (int c = 0; c < 3; c++) {
    P0[c] = cell_coord(x0[c], 2.0 * wl, np);
    Pold[c] = cell_coord(mv.r[c], 2.0 * wl, np);
  }
  int b[3];
  for (int c = 0; c < 3; c++) b[c] = 2 * (((P0[c] + dlt[c]) % np + np) % np) + ((o >> c) & 1);
  if (side0 == 1) {  // already covered by the old position's list?
    bool in_old = true;
    for (int c = 0; c < 3; c++)
      if (wdist(b[c] >> 1, Pold[c], np) > 1) in_old = false;
    if (in_old) return;
  }
  double cb[3] = {(b[0] + 0.5) * wl, (b[1] + 0.5) * wl, (b[2] + 0.5) * wl};
  double2 acc[KMC_MAXP + 1];
  for (int n = 0; n <= g.p; n++) acc[n] = make_double2(0.0, 0.0);
  bool any = false;
  for (int side = 0; side < 2; side++) {
    const double* x = side ? mv.rn : mv.r;
    double q = side ? mv.q : -mv.q;
    int u0[3];
    for (int c = 0; c < 3; c++) u0[c] = cell_coord(x[c], wl, nl);
    for (int nu = 0; nu < 27; nu++) {
      int nv[3] = {nu % 3 - 1, (nu / 3) % 3 - 1, nu / 9 - 1};
      bool in = true, far = false;
      for (int c = 0; c < 3; c++) {
        int u = u0[c] + nl * nv[c];
        if (abs(fdiv2(u) - (b[c] >> 1)) > 1) in = false;
        if (abs(u - b[c]) >= 2) far = true;
      }
      if (!in || !far) continue;
      any = true;
      double dx = x[0] + g.a * nv[0] - cb[0], dy = x[1] + g.a * nv[1] - cb[1], dz = x[2] + g.a * nv[2] - cb[2];
      double r2 = dx * dx + dy * dy + dz * dz, inv = 1.0 / r2;
      double2 mm = make_double2(1.0 / sqrt(r2), 0.0);
      for (int j = 1; j <= m; j++) {
        double sc = -(2.0 * j - 1.0) * inv;
        mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
      }
      double2 a1 = mm, a2 = make_double2(0.0, 0.0);
      acc[m].x += q * mm.x;
      acc[m].y -= q * mm.y;
      for (int n = m + 1; n <= g.p; n++) {
        double zz = (2 * n - 1) * dz;
        double c2 = (double)((n - 1) * (n - 1) - m * m);
        double2 v = make_double2((zz * a1.x - c2 * a2.x) * inv, (zz * a1.y - c2 * a2.y) * inv);
        acc[n].x += q * v.x;
        acc[n].y -= q * v.y;
        a2 = a1;
        a1 = v;
      }
    }
  }
  if (!any) return;
  double2* out = d.Psi + (g.cell_off[l] + b[0] + (int64_t)nl * (b[1] + (int64_t)nl * b[2])) * g.P;
  for (int n = m; n <= g.p; n++) {
    out[tri(n, m)].x += acc[n].x;
    out[tri(n, m)].y += acc[n].y;
  }
}

// move the charge between leaf slots; dipole, energy and bookkeeping
__global__ void k_acc_move(const Geo g, const Dev d) {
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  int32_t i = mv.i;
  int32_t so = d.slot_of[i];
  int64_t lo = so / g.cap;
  int ln = 0;
  {
    int cx = cell_coord(mv.rn[0], g.w, g.nL), cy = cell_coord(mv.rn[1], g.w, g.nL), cz = cell_coord(mv.rn[2], g.w, g.nL);
    ln = cx + g.nL * (cy + g.nL * cz);
  }
  // remove: move the leaf's last entry into the hole
  int64_t last = lo * g.cap + d.cnt[lo] - 1;
  if (last != so) {
    int32_t ul = d.uid[last];
    d.uid[so] = ul;
    d.spos64[so] = d.spos64[last];
    d.spos32[so] = d.spos32[last];
    d.slot_of[ul] = so;
  }
  d.cnt[lo] -= 1;
  int c = d.cnt[ln];
  if (c >= g.cap) {  // cannot place: undo the removal accounting and flag
    atomicOr(&d.err[0], KMC_DERR_CAPACITY);
    d.cnt[lo] += 1;
    return;
  }
  int64_t sn = (int64_t)ln * g.cap + c;
  d.cnt[ln] = c + 1;
  d.uid[sn] = i;
  d.spos64[sn] = make_double4_32a(mv.rn[0], mv.rn[1], mv.rn[2], mv.q);
  d.spos32[sn] = make_float4((float)mv.rn[0], (float)mv.rn[1], (float)mv.rn[2], (float)mv.q);
  d.slot_of[i] = (int32_t)sn;
  d.pos[3 * i] = mv.rn[0];
  d.pos[3 * i + 1] = mv.rn[1];
  d.pos[3 * i + 2] = mv.rn[2];
  d.site[i] = mv.site_new;
  for (int c3 = 0; c3 < 3; c3++) d.dip[c3] += mv.q * (mv.rn[c3] - mv.r[c3]);
  d.U[0] += mv.dU;
}

void kmc_accept_apply(const Geo& g, const Dev& d, cudaStream_t s) {
  int nt = g.L * (g.p + 1);
  k_acc_multipole<<<(nt + 63) / 64, 64, 0, s>>>(g, d);
  k_acc_far<<<1, g.P <= 128 ? 128 : 256, g.P * sizeof(double2), s>>>(g, d);
  dim3 grid((432 * (g.p + 1) + 127) / 128, g.L - 1);
  k_acc_locals<<<grid, 128, 0, s>>>(g, d);
  k_acc_move<<<1, 1, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ general points
// warp per point: phi(x) = L2P(leaf) + sum over the 27 neighbour leaves,
// skipping user index excl[t] (or none if excl == NULL / -1).  A source at
// distance 0 that is not excluded marks the result NaN (singular target).
template <typename T>
__global__ void k_eval_points(const Geo g, const Dev d, int64_t m, const double* pts, const int32_t* excl,
                              double* out) {
  typedef typename cplx<T>::type C;
  typedef typename vec4<T>::type V4;
  int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (wid >= m) return;
  double X = pts[3 * wid], Y = pts[3 * wid + 1], Z = pts[3 * wid + 2];
  int ex = excl ? excl[wid] : -1;
  int cx = cell_coord(X, g.w, g.nL), cy = cell_coord(Y, g.w, g.nL), cz = cell_coord(Z, g.w, g.nL);
  int64_t leaf = cx + (int64_t)g.nL * (cy + (int64_t)g.nL * cz);
  const V4* spos = (const V4*)((sizeof(T) == 4) ? (const void*)d.spos32 : (const void*)d.spos64);
  T x = (T)X, y = (T)Y, z = (T)Z;
  T s = 0;
  int sing = 0;
  for (int o = 0; o < 27; o++) {
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    int ux = cx + ox, uy = cy + oy, uz = cz + oz;
    int sx = (ux + g.nL) % g.nL, sy = (uy + g.nL) % g.nL, sz = (uz + g.nL) % g.nL;
    int64_t lf = sx + (int64_t)g.nL * (sy + (int64_t)g.nL * sz);
    T shx = (T)((ux - sx) * g.w), shy = (T)((uy - sy) * g.w), shz = (T)((uz - sz) * g.w);
    int c = d.cnt[lf];
    for (int j = lane; j < c; j += 32) {
      int64_t sl = lf * g.cap + j;
      if (d.uid[sl] == ex) continue;
      V4 v = spos[sl];
      T dx = v.x + shx - x, dy = v.y + shy - y, dz = v.z + shz - z;
      T r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > (T)0) s += v.w * rsq(r2);
      else sing = 1;
    }
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    s += __shfl_xor_sync(0xffffffff, s, o2);
    sing |= __shfl_xor_sync(0xffffffff, sing, o2);
  }
  // L2P: lane m evaluates column m
  const C* L = (const C*)d.Peff + (g.cell_off[g.L] + leaf) * g.P;
  T px = (T)(X - (cx + 0.5) * g.w), py = (T)(Y - (cy + 0.5) * g.w), pz = (T)(Z - (cz + 0.5) * g.w);
  T col = 0;
  if (lane <= g.p) {
    int mm = lane;
    T r2 = px * px + py * py + pz * pz;
    T ax = 1, ay = 0;
    for (int j = 1; j <= mm; j++) {
      T sc = halfm<T>(j);
      T tx = sc * (px * ax - py * ay), ty = sc * (px * ay + py * ax);
      ax = tx;
      ay = ty;
    }
    C lv = L[tri(mm, mm)];
    col = lv.x * ax - lv.y * ay;
    T a1x = ax, a1y = ay, a2x = 0, a2y = 0;
    for (int n = mm + 1; n <= g.p; n++) {
      T cc = inv_nm<T>(tri(n, mm));
      T zz = (T)(2 * n - 1) * pz;
      T vx = (zz * a1x - r2 * a2x) * cc, vy = (zz * a1y - r2 * a2y) * cc;
      lv = L[tri(n, mm)];
      col += lv.x * vx - lv.y * vy;
      a2x = a1x; a2y = a1y;
      a1x = vx; a1y = vy;
    }
    if (mm > 0) col += col;
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) col += __shfl_xor_sync(0xffffffff, col, o2);
  if (lane == 0) {
    out[wid] = sing ? __longlong_as_double(0x7ff8000000000000LL) : (double)(s + col);
    if (sing) atomicOr(&d.err[0], KMC_DERR_SINGULAR);
  }
}

void kmc_eval_points(const Geo& g, const Dev& d, int prec, int64_t m, const double* pts, const int32_t* excl,
                     double* out, cudaStream_t s) {
  if (m <= 0) return;
  unsigned blocks = (unsigned)((m * 32 + 127) / 128);
  if (prec == 0) k_eval_points<double><<<blocks, 128, 0, s>>>(g, d, m, pts, excl, out);
  else k_eval_points<float><<<blocks, 128, 0, s>>>(g, d, m, pts, excl, out);
}

// dU for general proposals from the evaluated potentials (FP64 assembly);
// tgt holds the wrapped targets and phi_new/phi_old the two potentials;
// selfc_list (in dU on entry) holds C(d_min) per proposal.
__global__ void k_assemble_general(const Geo g, const Dev d, int64_t m, const int32_t* particle,
                                   const double* tgt, const uint8_t* mask, const double* phi_new,
                                   const double* phi_old, double* dU) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  if (mask && !mask[t]) {
    dU[t] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  int32_t i = particle[t];
  double q = d.q[i];
  double dx = tgt[3 * t] - d.pos[3 * i], dy = tgt[3 * t + 1] - d.pos[3 * i + 1], dz = tgt[3 * t + 2] - d.pos[3 * i + 2];
  double V = g.a * g.a * g.a;
  double cself = dU[t];
  double v = q * (phi_new[t] - phi_old[t]) - 4.0 * M_PI / (3.0 * V) * q * (d.dip[0] * dx + d.dip[1] * dy + d.dip[2] * dz) -
             q * q * cself;
  double dmx = dx - g.a * rint(dx / g.a), dmy = dy - g.a * rint(dy / g.a), dmz = dz - g.a * rint(dz / g.a);
  if (dmx == 0.0 && dmy == 0.0 && dmz == 0.0) {
    v = __longlong_as_double(0x7ff8000000000000LL);
    atomicOr(&d.err[0], KMC_DERR_SINGULAR);
  }
  dU[t] = v;
}

void kmc_assemble_general(const Geo& g, const Dev& d, int64_t m, const int32_t* particle, const double* tgt,
                          const uint8_t* mask, const double* phi_new, const double* phi_old, double* dU,
                          cudaStream_t s) {
  if (m <= 0) return;
  k_assemble_general<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(g, d, m, particle, tgt, mask, phi_new, phi_old, dU);
}

// ------------------------------------------------------------------ energy
// U = 1/2 sum q_i Phi_self(r_i) - 2 pi |M|^2 / (3V)  (Algorithm 3 with the far
// field in Phi and the dipole term of Sec. 2.2.2); fixed-order reduction.
__global__ void k_energy(const Geo g, const Dev d) {
  __shared__ double sh[1024];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) a += d.q[i] * d.phi_old[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double V = g.a * g.a * g.a;
    double M2 = d.dip[0] * d.dip[0] + d.dip[1] * d.dip[1] + d.dip[2] * d.dip[2];
    d.U[0] = 0.5 * sh[0] - 2.0 * M_PI / (3.0 * V) * M2;
  }
}

void kmc_energy_reduce(const Geo& g, const Dev& d, cudaStream_t s) { k_energy<<<1, 1024, 0, s>>>(g, d); }

// ------------------------------------------------------------------ validation
// positions finite and inside [0, a); lattice mode: on a site centre; sets site[]
__global__ void k_validate(const Geo g, const Dev d) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double x = d.pos[3 * i], y = d.pos[3 * i + 1], z = d.pos[3 * i + 2];
  bool ok = isfinite(x) && isfinite(y) && isfinite(z) && x >= 0.0 && y >= 0.0 && z >= 0.0 && x < g.a && y < g.a &&
            z < g.a && isfinite(d.q[i]);
  if (!ok) {
    atomicOr(&d.err[0], KMC_DERR_BADPOS);
    return;
  }
  if (g.E > 0) {
    double fx = x / g.h - 0.5, fy = y / g.h - 0.5, fz = z / g.h - 0.5;
    double rx = rint(fx), ry = rint(fy), rz = rint(fz);
    if (fabs(fx - rx) > 1e-9 || fabs(fy - ry) > 1e-9 || fabs(fz - rz) > 1e-9) {
      atomicOr(&d.err[0], KMC_DERR_BADSITE);
      return;
    }
    int ix = (int)rx, iy = (int)ry, iz = (int)rz;
    d.site[i] = ix + g.E * (iy + g.E * iz);
    // snap to the exact site centre
    d.pos[3 * i] = (ix + 0.5) * g.h;
    d.pos[3 * i + 1] = (iy + 0.5) * g.h;
    d.pos[3 * i + 2] = (iz + 0.5) * g.h;
  } else {
    d.site[i] = -1;
  }
}

void kmc_validate(const Geo& g, const Dev& d, cudaStream_t s) {
  k_validate<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ general staging
// wrap targets into [0, a), gather old positions, minimum-image displacement
// (for the self term C(d_min)); out-of-range particle indices flag an error.
__global__ void k_stage_general(const Geo g, const Dev d, int64_t m, const int32_t* part, const double* tin,
                                const uint8_t* min_, double* tout, double* old, double* dv, uint8_t* mout) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  int32_t i = part[t];
  bool ok = i >= 0 && i < g.n;
  mout[t] = (min_ ? min_[t] : 1) && ok;
  if (!ok) atomicOr(&d.err[0], KMC_DERR_BADPOS);
  for (int k = 0; k < 3; k++) {
    double x = tin[3 * t + k];
    if (!isfinite(x)) {
      atomicOr(&d.err[0], KMC_DERR_BADPOS);
      x = 0.0;
      mout[t] = 0;
    }
    x -= g.a * floor(x / g.a);
    if (x >= g.a) x -= g.a;
    double o = ok ? d.pos[3 * (int64_t)i + k] : 0.0;
    tout[3 * t + k] = x;
    old[3 * t + k] = o;
    double dd = x - o;
    dv[3 * t + k] = dd - g.a * rint(dd / g.a);
  }
}

void kmc_stage_general(const Geo& g, const Dev& d, int64_t m, const int32_t* part, const double* tin,
                       const uint8_t* min_, double* tout, double* old, double* dv, uint8_t* mout, cudaStream_t s) {
  if (m <= 0) return;
  k_stage_general<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(g, d, m, part, tin, min_, tout, old, dv, mout);
}
