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
// images (the self-image term of Eq. (proposed_energy_sr), here summed over
// the 5x5x5 block of domain copies the tree covers, and its far-field part).  The M.d term and the |d|^2 part of C together are the
// change of the surface term that the dipole correction of Sec. 2.2.2 removes.
#include <math.h>
#include <stdio.h>

#include <type_traits>

#include "common.cuh"
#include <cuda_fp16.h>

__constant__ float c_inv_f[KMC_NTRI];
__constant__ double c_inv_d[KMC_NTRI];
__constant__ float2 c_inv2_f[KMC_NTRI];      // (1/((n-m)(n+m)), same) pairs for packed FP32
__constant__ float c_halfm_f[KMC_MAXP + 2];   // -1/(2m)
__constant__ double c_halfm_d[KMC_MAXP + 2];
// Hop entries of a leaf's propose CTA, per hop set (0: the 6 faces, 1: the
// 14 faces and body diagonals): entry 0 is the leaf itself (every hop), the
// others the neighbour leaves from which a hop can enter it -- the 6 face
// neighbours for the face set, all 26 for the 14-hop set.  c_ent_leaf is the
// entry's index in the 27-neighbourhood list, c_ent_hops the bit set of the
// hops that can enter from there (component -o_a on every axis a where the
// neighbour's offset o_a is not 0).
__constant__ int c_ent_leaf[2][27];
__constant__ uint32_t c_ent_hops[2][27];

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
  static float2 inv2[KMC_NTRI];
  for (int t = 0; t < KMC_NTRI; t++) inv2[t] = make_float2(invf[t], invf[t]);
  cudaMemcpyToSymbol(c_inv2_f, inv2, sizeof(inv2));
  cudaMemcpyToSymbol(c_inv_d, invd, sizeof(invd));
  cudaMemcpyToSymbol(c_halfm_f, hf, sizeof(hf));
  cudaMemcpyToSymbol(c_halfm_d, hd, sizeof(hd));
  static int el[2][27];
  static uint32_t eh[2][27];
  for (int hs = 0; hs < 2; hs++) {
    const int nhop = hs ? KMC_MAXHOP : KMC_NHOP, ne = hs ? 27 : 1 + KMC_NHOP;
    for (int e = 0; e < 27; e++) {
      el[hs][e] = 0;
      eh[hs][e] = 0;
      if (e >= ne) continue;
      int li = e, off[3] = {0, 0, 0};
      if (!hs && e > 0)  // the neighbour across face e - 1
        for (int a = 0; a < 3; a++) off[a] = hop_c(e - 1, a);
      if (hs && e > 0) {
        const int qq = e <= 13 ? e - 1 : e;
        off[0] = qq % 3 - 1;
        off[1] = (qq / 3) % 3 - 1;
        off[2] = qq / 9 - 1;
      }
      if (!hs && e > 0) {
        const int qq = (off[0] + 1) + 3 * (off[1] + 1) + 9 * (off[2] + 1);
        li = qq < 13 ? qq + 1 : qq;
      }
      el[hs][e] = li;
      for (int k = 0; k < nhop; k++) {
        bool ok = true;
        for (int a = 0; a < 3; a++)
          if (off[a] != 0 && hop_c(k, a) != -off[a]) ok = false;
        if (ok) eh[hs][e] |= 1u << k;
      }
    }
  }
  cudaMemcpyToSymbol(c_ent_leaf, el, sizeof(el));
  cudaMemcpyToSymbol(c_ent_hops, eh, sizeof(eh));
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


// ------------------------------------------------------------------ near-field helpers
// Lattice proposals take coordinates in lattice units relative to the target
// leaf's corner, so that for source s and target t every term of
// |s - t|^2 = |s|^2 + |t|^2 - 2 s.t is a small integer and the squared
// distance is exact.  FP32: the squared distances from f16 tensor-core
// products (nfmma below), 1/r from the MUFU rsqrt.approx (relative error
// < 2^-22), scaled by 1/h once per target.  FP64: 1/r from a table of
// 1/sqrt(n) (below), one source per iteration.
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename T> struct NearField;

// small integer (|i| < 2^22) to float on the FMA pipe: the float with bits
// 0x4B400000 + i is 1.5 2^23 + i
__device__ __forceinline__ float i2f(int i) { return __int_as_float(0x4B400000 + i) - 12582912.f; }

// FP32 form: the pair sums on the tensor cores and the MUFU.  On the lattice
// the squared distance between a site t and a source s (lattice units, the
// target leaf's frame) is the integer n = t.t + s.s - 2 t.s, and for leaf
// edges W <= 12 every coordinate and every term of that sum is an integer
// of at most 11 bits (|s| < 2W per axis, n <= 3 (2W - 1)^2 < 2^11), exact in
// f16.  One m16n8k8 f16 MMA with FP32 accumulation therefore gives n exactly
// for 16 sites x 8 sources, from site features (tx, ty, tz, 1, t.t, 0, 0, 0)
// and source features (-2sx, -2sy, -2sz, s.s, 1, 0, 0, 0): the distance
// arithmetic leaves the FP32 pipes, which carry only the accumulation
// q / sqrt(n); 1 / sqrt(n) comes from the MUFU.
// Fragments (PTX m16n8k8, lane = 4 g + c): A rows g and g + 8, columns 2c and
// 2c + 1; B column (source) g, rows 2c and 2c + 1; D rows g and g + 8, columns
// 2c and 2c + 1.  Staged source (16 bytes, written over the copied slot
// position): word 0 = f16x2 (-2sx, -2sy), word 1 = f16x2 (-2sz, s.s), word 2 =
// q (FP32), word 3 unused; feature rows 4..7 (1, 0, 0, 0) are constants of the
// lanes with c = 2, 3.
namespace nfmma {
constexpr int TMAX = 2;  // site tiles of 16 per round (32 sites; four tiles measured 3% slower)
// shared-memory bytes of a pass of `chunk` sources, padded to a whole tile of eight
__host__ __device__ __forceinline__ size_t bytes(int chunk) { return 16 * ((size_t)chunk + 8); }
__device__ __forceinline__ uint32_t h2bits(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// the staged record of a source at (sx, sy, sz) (frame lattice units) with charge q
__device__ __forceinline__ float4 record(int sx, int sy, int sz, float q) {
  const float x = i2f(sx), y = i2f(sy), z = i2f(sz);
  return make_float4(__uint_as_float(h2bits(-2.f * x, -2.f * y)),
                     __uint_as_float(h2bits(-2.f * z, fmaf(x, x, fmaf(y, y, z * z)))), q, 0.f);
}
// padding record: no charge, n = t.t + 1024 > 0
__device__ __forceinline__ float4 pad_record() {
  return make_float4(0.f, __uint_as_float(h2bits(0.f, 1024.f)), 0.f, 0.f);
}
// A fragment word of a site (x, y, z) for this lane's columns 2c, 2c + 1
__device__ __forceinline__ uint32_t site_word(int c, int x, int y, int z) {
  const float fx = i2f(x), fy = i2f(y), fz = i2f(z);
  const float tt = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
  const float lo = c == 0 ? fx : (c == 1 ? fz : (c == 2 ? tt : 0.f));
  const float hi = c == 0 ? fy : (c == 1 ? 1.f : 0.f);
  return h2bits(lo, hi);
}
__device__ __forceinline__ void mma(uint32_t a0, uint32_t a1, uint32_t b, float& d0, float& d1, float& d2,
                                    float& d3) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, {%7, %7, %7, %7};"
      : "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
      : "r"(a0), "r"(a1), "r"(b), "f"(0.f));
}
// source tiles [j0, j1) (8 staged records each, R = first record) against
// the NT site tiles of a[]; GUARD: the tiles hold the sites' own charges
// (the pair at n = 0 adds nothing)
template <int NT, bool GUARD>
__device__ __forceinline__ void run(const uint32_t* R, int j0, int j1, const uint32_t (&a)[TMAX][2],
                                    float2 (&acc)[TMAX][2], int g, int c, uint32_t bc) {
#pragma unroll 2  // 1: 1.6% slower on the 1M-charge workload, 4: 2.4% slower
  for (int j = j0; j < j1; j++) {
    const uint32_t* T = R + 32 * j;
    const uint32_t bw = T[4 * g + c];
    const uint32_t b = c < 2 ? bw : bc;
    const float2 qv = make_float2(__uint_as_float(T[8 * c + 2]), __uint_as_float(T[8 * c + 6]));
    // all products, then all rsqrts, then the accumulation: no rsqrt waits
    // behind an accumulation that waits for an earlier rsqrt
    float dd[TMAX][4];
#pragma unroll
    for (int s = 0; s < NT; s++) mma(a[s][0], a[s][1], b, dd[s][0], dd[s][1], dd[s][2], dd[s][3]);
    float2 uu[TMAX][2];
#pragma unroll
    for (int s = 0; s < NT; s++) {
      uu[s][0] = make_float2(rsqrt_mufu(dd[s][0]), rsqrt_mufu(dd[s][1]));
      uu[s][1] = make_float2(rsqrt_mufu(dd[s][2]), rsqrt_mufu(dd[s][3]));
    }
#pragma unroll
    for (int s = 0; s < NT; s++) {
      if (GUARD) {
        uu[s][0].x = dd[s][0] > 0.f ? uu[s][0].x : 0.f;
        uu[s][0].y = dd[s][1] > 0.f ? uu[s][0].y : 0.f;
        uu[s][1].x = dd[s][2] > 0.f ? uu[s][1].x : 0.f;
        uu[s][1].y = dd[s][3] > 0.f ? uu[s][1].y : 0.f;
      }
      acc[s][0] = __ffma2_rn(uu[s][0], qv, acc[s][0]);
      acc[s][1] = __ffma2_rn(uu[s][1], qv, acc[s][1]);
    }
  }
}
// one round: site tiles [t0, t0 + NT) of the compacted site list against this
// warp's source tiles [j0, j1) (the first jg of them guarded); the row sums
// go to the fixed-point accumulators accs (scaled by `scale`)
template <int NT>
__device__ __forceinline__ void round(const uint32_t* R, const uint16_t* sites, int nsites, int W, int t0, int j0,
                                      int jg, int j1, int* accs, float scale, int lane, int* err) {
  const int g = lane >> 2, c = lane & 3;
  uint32_t a[TMAX][2];
  float2 acc[TMAX][2];
#pragma unroll
  for (int s = 0; s < NT; s++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int i = 16 * (t0 + s) + g + 8 * h;
      const int sv = i < nsites ? sites[i] : 0;
      a[s][h] = site_word(c, sv & 15, (sv >> 4) & 15, sv >> 8);
      acc[s][h] = make_float2(0.f, 0.f);
    }
  const uint32_t bc = c == 2 ? 0x3C00u : 0u;  // f16x2 (1, 0) for rows 4, 5; 0 for rows 6, 7
  if (jg > j0) run<NT, true>(R, j0, jg, a, acc, g, c, bc);
  if (j1 > jg) run<NT, false>(R, jg, j1, a, acc, g, c, bc);
#pragma unroll
  for (int s = 0; s < NT; s++) {
    float v0 = acc[s][0].x + acc[s][0].y, v1 = acc[s][1].x + acc[s][1].y;
    v0 += __shfl_xor_sync(0xffffffffu, v0, 1);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    v0 += __shfl_xor_sync(0xffffffffu, v0, 2);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
    const int i = 16 * (t0 + s) + g + 8 * c;  // lane c = 0: row g, c = 1: row g + 8
    if (c < 2 && i < nsites) {
      const int sv = sites[i];
      const int l = (sv & 15) + W * (((sv >> 4) & 15) + W * (sv >> 8));
      if (KMC_IN(l >= 0 && l < W * W * W, err)) atomicAdd(&accs[l], __float2int_rn((c ? v1 : v0) * scale));
    }
  }
}
}  // namespace nfmma

// FP64 form.  On the lattice every squared distance is an exact integer n in
// lattice units (|d| < 2W per axis, so n <= 3 (2W - 1)^2 < 2^24), so 1/|d|
// comes from a table of correctly rounded 1/sqrt(n) (entry 0 = 0: the pair at
// distance 0 adds nothing), indexed by the FP32-exact n; the only FP64
// operation per pair is the accumulation q / |d|.  Staged source: (x, y, z,
// |s|^2) in lattice units in the target leaf's frame (FP32, exact integers),
// then the FP64 charge.
template <> struct NearField<double> {
  struct Src {
    float4 p;
    double q, pad;
  };
  double a0, a1;
  __device__ __forceinline__ void reset() { a0 = a1 = 0.0; }
  static __host__ __device__ __forceinline__ size_t bytes(int chunk) { return (size_t)chunk * sizeof(Src); }
  static __device__ __forceinline__ void stage(unsigned char* sm, int e, int x, int y, int z, double q) {
    Src v;
    v.p = make_float4((float)x, (float)y, (float)z, (float)(x * x + y * y + z * z));
    v.q = q;
    v.pad = 0.0;
    ((Src*)sm)[e] = v;
  }
  // sources [j0, j1) against the leaf-local targets t0 and t1 (t1 only when
  // two is set; warp-uniform)
  __device__ __forceinline__ void run2(const unsigned char* sm, const double* isq, int j0, int j1, bool two, int tx0,
                                       int ty0, int tz0, int tx1, int ty1, int tz1, int nisq, int* err) {
    const Src* src = (const Src*)sm;
    const float ax0 = (float)(-2 * tx0), ay0 = (float)(-2 * ty0), az0 = (float)(-2 * tz0);
    const float ax1 = (float)(-2 * tx1), ay1 = (float)(-2 * ty1), az1 = (float)(-2 * tz1);
    const float w0 = (float)(tx0 * tx0 + ty0 * ty0 + tz0 * tz0), w1 = (float)(tx1 * tx1 + ty1 * ty1 + tz1 * tz1);
    double s0 = a0, s1 = a1;
    for (int j = j0; j < j1; j++) {
      const float4 v = src[j].p;
      const double q = src[j].q;
      // n = |s|^2 + |t|^2 - 2 s.t, exact; n + 2^23 holds n in its low mantissa bits
      const float n0 = fmaf(ax0, v.x, fmaf(ay0, v.y, fmaf(az0, v.z, v.w + w0)));
      const int k0 = __float_as_int(n0 + 8388608.f) - 0x4B000000;
      if (KMC_IN(k0 >= 0 && k0 < nisq, err)) s0 = fma(q, isq[k0], s0);
      if (two) {
        const float n1 = fmaf(ax1, v.x, fmaf(ay1, v.y, fmaf(az1, v.z, v.w + w1)));
        const int k1 = __float_as_int(n1 + 8388608.f) - 0x4B000000;
        if (KMC_IN(k1 >= 0 && k1 < nisq, err)) s1 = fma(q, isq[k1], s1);
      }
    }
    a0 = s0;
    a1 = s1;
  }
  __device__ __forceinline__ double sum(int side) const { return side ? a1 : a0; }
};

// packed FP32 L2P: the complex recurrence and the accumulation use FP32x2
// (real and imaginary parts in one instruction); 1/((n-m)(n+m)) pairs from
// constant memory.
__device__ __forceinline__ float l2p_packed(const float2* L, int p, float x, float y, float z) {
  const float r2 = x * x + y * y + z * z;
  const float2 nr2 = make_float2(-r2, -r2);
  const float2 z2 = make_float2(2.f * z, 2.f * z);
  float mmx = 1.f, mmy = 0.f;
  float total = 0.f;
  for (int m = 0; m <= p; m++) {
    if (m > 0) {
      float s = c_halfm_f[m];
      float tx = s * (x * mmx - y * mmy);
      float ty = s * (x * mmy + y * mmx);
      mmx = tx;
      mmy = ty;
    }
    float2 a1 = make_float2(mmx, mmy), a2 = make_float2(0.f, 0.f);
    float2 col = __fmul2_rn(L[tri(m, m)], a1);
    float zz0 = (float)(2 * m + 1) * z;
    float2 zz = make_float2(zz0, zz0);
    for (int n = m + 1; n <= p; n++) {
      float2 v = __ffma2_rn(zz, a1, __fmul2_rn(nr2, a2));
      v = __fmul2_rn(v, c_inv2_f[tri(n, m)]);
      col = __ffma2_rn(L[tri(n, m)], v, col);
      a2 = a1;
      a1 = v;
      zz = __fadd2_rn(zz, z2);
    }
    float cm = col.x - col.y;
    total += (m == 0) ? cm : cm + cm;
  }
  return total;
}

// the same evaluation with the degree known at compile time: fully unrolled,
// the recurrence factors 1/((n-m)(n+m)) and -1/(2m) as immediates and the
// coefficient addresses as constant offsets
template <int P> __device__ __forceinline__ float l2p_fixed(const float2* L, float x, float y, float z) {
  const float r2 = x * x + y * y + z * z;
  const float2 nr2 = make_float2(-r2, -r2);
  const float2 z2 = make_float2(2.f * z, 2.f * z);
  float mmx = 1.f, mmy = 0.f;
  float total = 0.f;
#pragma unroll
  for (int m = 0; m <= P; m++) {
    if (m > 0) {
      const float s = -0.5f / (float)m;
      const float tx = s * (x * mmx - y * mmy);
      const float ty = s * (x * mmy + y * mmx);
      mmx = tx;
      mmy = ty;
    }
    float2 a1 = make_float2(mmx, mmy), a2 = make_float2(0.f, 0.f);
    float2 col = __fmul2_rn(L[tri(m, m)], a1);
    const float zz0 = (float)(2 * m + 1) * z;
    float2 zz = make_float2(zz0, zz0);
#pragma unroll
    for (int n = m + 1; n <= P; n++) {
      const float c = 1.f / (float)((n - m) * (n + m));
      float2 v = __ffma2_rn(zz, a1, __fmul2_rn(nr2, a2));
      v = __fmul2_rn(v, make_float2(c, c));
      col = __ffma2_rn(L[tri(n, m)], v, col);
      a2 = a1;
      a1 = v;
      zz = __fadd2_rn(zz, z2);
    }
    const float cm = col.x - col.y;
    total += (m == 0) ? cm : cm + cm;
  }
  return total;
}

// FP32 L2P with the common degrees unrolled (p is uniform over the launch)
__device__ __forceinline__ float l2p_f32(const float2* L, int p, float x, float y, float z) {
  switch (p) {
    case 8: return l2p_fixed<8>(L, x, y, z);
    case 10: return l2p_fixed<10>(L, x, y, z);
    case 12: return l2p_fixed<12>(L, x, y, z);
    default: return l2p_packed(L, p, x, y, z);
  }
}

template <typename T, typename C> __device__ __forceinline__ T l2p_point(const C* L, int p, T x, T y, T z);
template <> __device__ __forceinline__ float l2p_point<float, float2>(const float2* L, int p, float x, float y, float z) {
  return l2p_f32(L, p, x, y, z);
}
template <> __device__ __forceinline__ double l2p_point<double, double2>(const double2* L, int p, double x, double y,
                                                                        double z) {
  return l2p_eval<double, double2>(L, p, x, y, z);
}

// ------------------------------------------------------------------ propose (lattice)
// One CTA per leaf cell.  Evaluation points of the CTA are every position in
// the leaf at which a potential is needed: the leaf's own charges (old
// positions, own charge excluded) and every unmasked hop target that lies in
// the leaf, whether the hopping charge sits in this leaf or in one of its six
// face neighbours.  Sources are the charges of the 27 neighbouring leaves
// (periodically wrapped images), staged in shared memory.
#define PROP_THREADS 128

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// Site coordinate of a lattice position (i + 1/2) h: floor(x / h) = i exactly
// for the lattice sizes accepted at init (E^3 < 2^31).
// (FP32 form without the conversion unit, which the pair loop's rsqrt
// occupies: x ih - 1/2 = i + delta with |delta| far below 1/2, and adding
// 1.5 2^23 rounds it to the integer 1.5 2^23 + i, whose low bits are i)
__device__ __forceinline__ int lattice_coord(float x, float ih) {
  return __float_as_int(fmaf(x, ih, -0.5f) + 12582912.f) - 0x4B400000;
}
__device__ __forceinline__ int lattice_coord(double x, double ih) { return (int)floor(x * ih); }

template <typename T> __device__ __forceinline__ T small_to(int i);
template <> __device__ __forceinline__ float small_to<float>(int i) { return i2f(i); }
template <> __device__ __forceinline__ double small_to<double>(int i) { return (double)i; }

// coordinate c + dc (|dc| <= 1) wrapped into [0, E)
__device__ __forceinline__ int wrap1(int c, int E) { return c < 0 ? c + E : (c >= E ? c - E : c); }


// diagnostic: the bounded wait against a phase that never completes (16
// bytes expected on the barrier, nothing copied)
__global__ void k_wait_probe(uint64_t limit_ns, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) *flag = KMC_DERR_TIMEOUT;
}

int kmc_wait_probe(double limit_seconds, cudaStream_t s) {
  if (!(limit_seconds >= 0.001)) limit_seconds = 0.001;
  if (limit_seconds > 2.0) limit_seconds = 2.0;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return -1;
  int host = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_probe<<<1, 32, 0, s>>>((uint64_t)(limit_seconds * 1e9), flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  return e == cudaSuccess ? host : -1;
}


// partial near-field sum (already scaled) into a fixed-point accumulator in
// shared memory, rounded to nearest
__device__ __forceinline__ void fixed_add(int* a, float v) { atomicAdd(a, __float2int_rn(v)); }
__device__ __forceinline__ void fixed_add(long long* a, double v) {
  atomicAdd((unsigned long long*)a, (unsigned long long)__double2ll_rn(v));
}


// Evaluation is per distinct site of the leaf: the potential at a site is
// needed once even when several charges propose to hop there, and at an own
// charge's site it is that charge's old-position potential (the pair at
// distance 0 is skipped).  Phases: (0) the 27 neighbour leaves (slot base,
// count) and the source passes; in the FP32 form the first pass's slot
// positions are copied into shared memory by bulk asynchronous copies that
// run while phases 1-3 proceed; (1) occupancy bits; (2) needed-site bits,
// masked hops written; (3) compact site list; (4) near-field sums (sources
// split between the warps, fixed-point reduction) + L2P; (5) write-out by
// re-enumerating the same hops.  Site coordinates come from the slot
// positions (coalesced), user indices only where an output is written.
// mode: PROP_SUM (the pair sums of this step), PROP_FILL (pair sums at every
// site of the leaf into the near-field cache d.nearfx; no hops, no L2P, no
// outputs) or PROP_CACHED (the near-field sums read from the cache, no pairs).
// The cached form holds no source chunk in shared memory and runs twelve CTAs
// per SM (more resident leaves hide its load and barrier latency; sixteen
// spilled too much of the L2P).
enum { PROP_SUM = 0, PROP_FILL = 1, PROP_CACHED = 2 };

// Outputs of a leaf recorded by the site phases for the write-out: (output
// index, local site) pairs, nhop u + k for hop k of charge u (unmasked, target
// in this leaf) and -1 - u for the old position of an own charge u.  A leaf with
// more entries (a dense leaf) re-enumerates its hops instead.
template <int NH> __host__ __device__ constexpr int wlist_cap() { return NH == KMC_NHOP ? 384 : 768; }

// shared-memory layout of one leaf (byte count: propose_smem)
template <typename T> struct LeafSmem {
  typedef typename cplx<T>::type C;
  unsigned char* src;  // sources of the current pass (FP32: staged records; FP64: NearField<double>::Src)
  C* Lc;               // [P] the leaf's local expansion, 16-byte aligned
  int64_t* nb_base;    // [27] slot base: own leaf, then the 26 others
  uint64_t* bar;       // [1] copy barrier (FP32 form)
  int* nb_off;         // [28] first source of each leaf in the pass layout
  int* nb_cnt;         // [27] charges per leaf
  int* nb_leaf;        // [27] leaf index
  int* pq;             // [28] first leaf of each source pass; pq[npass] = 27
  int* misc;           // [4] number of passes, fixed-point exponent, number of sites, write-list entries
  T* phis;             // [W3] potential per local site (fixed-point near-field sums before the L2P)
  uint32_t* bits;      // [nbw] occupied sites
  uint32_t* need;      // [nbw] sites where a potential is needed
  int* woff;           // [nbw + 1] prefix of needed sites per word
  uint16_t* sites;     // [W3] needed local sites (x | y << 4 | z << 8), compacted
  double* isq;         // FP64 form: 1/sqrt(n) for the squared lattice distances n <= 3 (2W - 1)^2
  int2* wl;            // [wlist_cap] recorded outputs (output index, local site)
  __device__ __forceinline__ LeafSmem(unsigned char* sm, const Geo& g, int chunk) {
    constexpr bool F32 = sizeof(T) == 4;
    const int W3 = g.W * g.W * g.W, nbw = (W3 + 31) / 32;
    src = sm;
    Lc = (C*)(sm + (F32 ? nfmma::bytes(chunk) : NearField<double>::bytes(chunk)));
    nb_base = (int64_t*)(Lc + g.P);
    bar = (uint64_t*)(nb_base + 27);
    nb_off = (int*)(bar + 1);
    nb_cnt = nb_off + 28;
    nb_leaf = nb_cnt + 27;
    pq = nb_leaf + 27;
    misc = pq + 28;
    phis = (T*)(misc + 4);
    bits = (uint32_t*)(phis + W3);
    need = bits + nbw;
    woff = (int*)(need + nbw);
    sites = (uint16_t*)(woff + nbw + 1);
    isq = (double*)(((uintptr_t)(sites + ((W3 + 1) & ~1)) + 7) & ~(uintptr_t)7);
    wl = (int2*)(isq + (F32 ? 0 : 3 * (2 * g.W - 1) * (2 * g.W - 1) + 1));
  }
};

// the leaf of a CTA and the thread's indices
struct LeafCtx {
  int64_t leaf;
  int lx, ly, lz, gx0, gy0, gz0;
  int tid, lane, warp;  // thread (0..127), lane, warp (0..3)
};
__device__ __forceinline__ LeafCtx leaf_ctx(const Geo& g, int64_t leaf, int tid) {
  LeafCtx x;
  const int nL = g.nL, lsh = g.L - 1;  // nL = 2^(L-1)
  x.leaf = leaf;
  x.lx = (int)(leaf & (nL - 1));
  x.ly = (int)((leaf >> lsh) & (nL - 1));
  x.lz = (int)(leaf >> (2 * lsh));
  x.gx0 = x.lx * g.W;
  x.gy0 = x.ly * g.W;
  x.gz0 = x.lz * g.W;
  x.tid = tid;
  x.lane = tid & 31;
  x.warp = tid >> 5;
  return x;
}

// Setup of a leaf: its local expansion, cleared site bitmaps and (warp 0) the
// 27 neighbour leaves (slot base, count), the split of their sources into
// passes of at most `chunk` (whole leaves), the fixed-point exponent and, in
// the FP32 form, the bulk copies of the first pass's slot positions, which
// land while the site phases run.
template <typename T, int mode>
__device__ __forceinline__ void leaf_setup(const Geo& g, const Dev& d, const LeafSmem<T>& S, const LeafCtx& x, int chunk) {
  typedef typename cplx<T>::type C;
  constexpr bool F32 = sizeof(T) == 4;
  const int W3 = g.W * g.W * g.W, nbw = (W3 + 31) / 32, nL = g.nL;
  const int nisq = 3 * (2 * g.W - 1) * (2 * g.W - 1) + 1;
  const int tid = x.tid, lane = x.lane;
  const C* Pe = (const C*)d.Peff + (g.cell_off[g.L] + x.leaf) * g.P;
  for (int c = tid; c < g.P; c += 128) S.Lc[c] = Pe[c];
  if (!F32 && mode != PROP_CACHED)
    for (int c = tid; c < nisq; c += 128) S.isq[c] = d.isq[c];
  for (int c = tid; c < nbw; c += 128) {
    S.bits[c] = 0u;
    S.need[c] = 0u;
  }
  // list entry 0 is this leaf, entries 1..26 the other neighbours in
  // 27-neighbourhood order (x fastest), centre skipped
  if (F32 && tid == 0) mbar_init(S.bar, 1);
  if (x.warp == 0) {
    int u = 0;
    if (lane < 27) {
      const int qq = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
      const int ux = x.lx + qq % 3 - 1, uy = x.ly + (qq / 3) % 3 - 1, uz = x.lz + qq / 9 - 1;
      const int sx = wrap1(ux, nL), sy = wrap1(uy, nL), sz = wrap1(uz, nL);
      const int nleaf = sx + nL * (sy + nL * sz);
      S.nb_leaf[lane] = nleaf;
      S.nb_base[lane] = (int64_t)nleaf * g.cap;
      // free space: a neighbour beyond the box does not exist (no images)
      const bool exists = !g.bc || (ux >= 0 && ux < nL && uy >= 0 && uy < nL && uz >= 0 && uz < nL);
      const int c = exists ? d.cnt[nleaf] : 0;
      S.nb_cnt[lane] = c;
      u = c;
    }
    // offsets of the leaves' sources: warp scan
    int incl = u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t2 = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t2;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 26);
    if (lane < 27) S.nb_off[lane] = incl - u;
    if (lane == 0) S.nb_off[27] = total;
    __syncwarp();
    if (lane == 0) {
      // the split into passes at leaf boundaries (one pass unless the
      // neighbourhood is dense); one leaf always fits (chunk >= capacity)
      int np = 0;
      S.pq[0] = 0;
      if (mode != PROP_CACHED && total > chunk) {
        int start = 0;
        for (int q = 0; q < 27; q++) {
          if (S.nb_off[q] + S.nb_cnt[q] - start > chunk) {
            S.pq[++np] = q;
            start = S.nb_off[q];
          }
        }
      }
      S.pq[++np] = 27;
      S.misc[0] = np;
      S.misc[3] = 0;  // write-list entries
      {  // fixed-point exponent of the near-field sums: 2^ks * bound < 2^(bits - 2)
        const double bound = g.qmax * (double)max(total, 1);  // lattice units
        S.misc[1] = (F32 ? 30 : 62) - (ilogb(bound) + 1);
      }
    }
    __syncwarp();
    if (F32 && mode != PROP_CACHED) {  // first pass: one bulk copy per leaf (one lane each)
      const int q1 = S.pq[1];
      if (lane == 0) mbar_expect_tx(S.bar, (uint32_t)(S.nb_off[q1] * 16));
      __syncwarp();
      if (lane < q1 && S.nb_cnt[lane])
        bulk_copy_g2s(S.src + 16 * S.nb_off[lane], d.spos32 + S.nb_base[lane], (uint32_t)(16 * S.nb_cnt[lane]), S.bar);
    }
  }
  __syncthreads();
}

// The sites of a leaf: (1) occupancy bits; (2) needed-site bits, masked hops
// written; (3) the compacted list of needed sites; their fixed-point sums
// cleared.  Returns the number of sites (also in S.misc[2]).
template <typename T, int NH, int mode>
__device__ __forceinline__ int leaf_sites(const Geo& g, const Dev& d, const LeafSmem<T>& S, const LeafCtx& x) {
  typedef typename vec4<T>::type V4;
  constexpr bool F32 = sizeof(T) == 4;
  const int W = g.W, W3 = W * W * W, nbw = (W3 + 31) / 32, E = g.E;
  const int rW = (65536 + W - 1) / W;
  const int tid = x.tid, lane = x.lane, warp = x.warp;
  const T ih = (T)(1.0 / g.h);
  const V4* spos = (const V4*)(F32 ? (const void*)d.spos32 : (const void*)d.spos64);
  T* out_new = (T*)(F32 ? (void*)d.phi_new32 : (void*)d.phi_new);
  // warp w handles the leaves f = w and w + 4 of {own leaf (f = 0), the
  // neighbour across face f - 1 (f = 1..6)}; the first 32 charges of each
  // are loaded at once, before the occupancy barrier
  constexpr int hs = NH == KMC_NHOP ? 0 : 1, ne = hs ? 27 : 1 + KMC_NHOP, nhop = NH;
  const int cnt_own = S.nb_cnt[0];
  const int64_t base_own = S.nb_base[0];
  V4 pv[2];
  int32_t pu[2];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const int e = warp + 4 * i;
    if (e < ne) {
      const int li = c_ent_leaf[hs][e];
      if (lane < S.nb_cnt[li]) {
        pv[i] = spos[S.nb_base[li] + lane];
        pu[i] = d.uid[S.nb_base[li] + lane];
      }
    }
  }
  // (1) occupancy bitmap of this leaf's sites (warp 0)
  constexpr int wcap = wlist_cap<NH>();
  if (warp == 0)
    for (int j = lane; j < cnt_own; j += 32) {
      const V4 v = j < 32 ? pv[0] : spos[base_own + j];
      const int ls = (lattice_coord(v.x, ih) - x.gx0) +
                     W * (lattice_coord(v.y, ih) - x.gy0 + W * (lattice_coord(v.z, ih) - x.gz0));
      if (KMC_IN(ls >= 0 && ls < W3, d.err)) {
        atomicOr(&S.bits[ls >> 5], 1u << (ls & 31));
        atomicOr(&S.need[ls >> 5], 1u << (ls & 31));
        if (mode != PROP_FILL) {  // the old-position potential of this charge
          const int32_t u = j < 32 ? pu[0] : d.uid[base_own + j];
          const int w = atomicAdd(&S.misc[3], 1);
          if (w < wcap) S.wl[w] = make_int2(-1 - u, ls);
        }
      }
    }
  __syncthreads();
  // (2) hop targets inside this leaf: the leaf's own hops and the hops that
  // enter it from the neighbours of its entry list
  // not unrolled: with the 14-hop set (27 entries, seven per warp) unrolled
  // copies of this loop and of the write-out's made the launch twice as slow
  // (larger code, more register spills)
#pragma unroll 1
  for (int i = 0; i < (mode == PROP_FILL ? 0 : (ne + 3) / 4); i++) {
    const int e = warp + 4 * i;
    if (e >= ne) break;
    const int li = c_ent_leaf[hs][e];
    const uint32_t hm = c_ent_hops[hs][e];
    const int64_t mb = S.nb_base[li];
    const int cm = S.nb_cnt[li];
    for (int j = lane; j < cm; j += 32) {
      const bool pre = j < 32 && i < 2;
      const V4 v = pre ? (i == 0 ? pv[0] : pv[1]) : spos[mb + j];
      const int32_t u = pre ? (i == 0 ? pu[0] : pu[1]) : d.uid[mb + j];
      const bool uok = KMC_IN(u >= 0 && u < g.n, d.err);
      const int gx = lattice_coord(v.x, ih), gy = lattice_coord(v.y, ih), gz = lattice_coord(v.z, ih);
      for (uint32_t hb = hm; hb; hb &= hb - 1) {
        const int k = __ffs(hb) - 1;
        const int rx = gx + hop_c(k, 0), ry = gy + hop_c(k, 1), rz = gz + hop_c(k, 2);
        if (g.bc && (rx < 0 || rx >= E || ry < 0 || ry >= E || rz < 0 || rz >= E)) {
          if (e == 0 && uok) {  // free space: a hop out of the box is not a move
            d.mask[(int64_t)nhop * u + k] = 0;
            out_new[(int64_t)nhop * u + k] = qnan<T>();
          }
          continue;
        }
        const int tx = wrap1(rx, E), ty = wrap1(ry, E), tz = wrap1(rz, E);
        const int ux = tx - x.gx0, uy = ty - x.gy0, uz = tz - x.gz0;
        if (ux < 0 || ux >= W || uy < 0 || uy >= W || uz < 0 || uz >= W) continue;  // another leaf's CTA
        const int lt = ux + W * (uy + W * uz);
        if (!KMC_IN(lt >= 0 && lt < W3, d.err)) continue;
        if (S.bits[lt >> 5] & (1u << (lt & 31))) {
          if (uok) {
            d.mask[(int64_t)nhop * u + k] = 0;
            out_new[(int64_t)nhop * u + k] = qnan<T>();
          }
        } else {
          atomicOr(&S.need[lt >> 5], 1u << (lt & 31));
          if (uok) {  // the write-out's entry for this hop
            const int w = atomicAdd(&S.misc[3], 1);
            if (w < wcap) S.wl[w] = make_int2(nhop * u + k, lt);
          }
        }
      }
    }
  }
  if (mode == PROP_FILL)  // every site of the leaf
    for (int c = tid; c < nbw; c += 128) S.need[c] = 32 * c + 32 <= W3 ? 0xffffffffu : (1u << (W3 - 32 * c)) - 1u;
  __syncthreads();
  // (3) compact the needed sites (ascending local index); word offsets by a
  // warp scan
  if (warp == 0) {
    int base = 0;
    for (int w0 = 0; w0 < nbw; w0 += 32) {
      const int w2 = w0 + lane;
      const int c = w2 < nbw ? __popc(S.need[w2]) : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t2 = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t2;
      }
      if (w2 < nbw) S.woff[w2] = base + incl - c;
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      S.woff[nbw] = base;
      S.misc[2] = base;
    }
  }
  __syncthreads();
  // one thread per local site: a needed site's place is its word's offset plus
  // the needed sites below it in the word
  for (int l = tid; l < W3; l += 128) {
    const uint32_t m = S.need[l >> 5], bit = 1u << (l & 31);
    if (m & bit) {
      const int o = S.woff[l >> 5] + __popc(m & (bit - 1u));
      // l = x + W (y + W z) by reciprocal multiplication: floor(l rW / 2^16)
      // = floor(l / W) for l < 2^16 / W (W <= 12, l < 1728)
      const int q1 = (l * rW) >> 16, z = (q1 * rW) >> 16;
      if (KMC_IN(o < W3, d.err)) S.sites[o] = (uint16_t)((l - q1 * W) | ((q1 - z * W) << 4) | (z << 8));
    }
  }
  __syncthreads();
  const int nsites = S.woff[nbw];
  // fixed-point sums of the needed sites cleared (integer view of phis)
  typedef typename std::conditional<F32, int, long long>::type Acc;
  Acc* acc = (Acc*)S.phis;
  for (int b = tid; b < nsites; b += 128) {
    const int sv = S.sites[b];
    acc[(sv & 15) + W * (((sv >> 4) & 15) + W * (sv >> 8))] = 0;
  }
  return nsites;
}

// Staging of source pass [q0, q1) into S.src.  FP32: waits (bounded) for the
// pass's bulk copies (barrier phase `parity`), then turns the copied slot
// positions into staged records in this leaf's frame (a warp per leaf, a lane
// per source) and pads the last tile of eight.  FP64: loads the pass from the
// slot arrays.  Returns false for the whole CTA when the copies did not
// arrive (flagged; the copies drained); the caller then leaves the leaf.
template <typename T>
__device__ __forceinline__ bool leaf_stage(const Geo& g, const Dev& d, const LeafSmem<T>& S, const LeafCtx& x, int q0,
                                           int q1, uint32_t parity) {
  typedef typename vec4<T>::type V4;
  constexpr bool F32 = sizeof(T) == 4;
  const int W = g.W, nL = g.nL;
  const T ih = (T)(1.0 / g.h);
  if constexpr (F32) {
    const bool ok = mbar_wait_bounded(S.bar, parity, KMC_WAIT_NS);
    if (__syncthreads_or(!ok)) {
      if (x.tid == 0) {
        atomicOr(&d.err[0], KMC_DERR_TIMEOUT);
        mbar_wait_bounded(S.bar, parity, KMC_WAIT_NS);
      }
      __syncthreads();
      return false;
    }
    for (int q = q0 + x.warp; q < q1; q += 4) {
      const int qq = q == 0 ? 13 : (q <= 13 ? q - 1 : q);
      const int ux = x.lx + qq % 3 - 1, uy = x.ly + (qq / 3) % 3 - 1, uz = x.lz + qq / 9 - 1;
      const int ox = (ux - wrap1(ux, nL)) * W - x.gx0, oy = (uy - wrap1(uy, nL)) * W - x.gy0;
      const int oz = (uz - wrap1(uz, nL)) * W - x.gz0;
      float4* Sr = (float4*)S.src + (S.nb_off[q] - S.nb_off[q0]);
      for (int j = x.lane; j < S.nb_cnt[q]; j += 32) {
        const float4 v = Sr[j];
        Sr[j] = nfmma::record(lattice_coord(v.x, ih) + ox, lattice_coord(v.y, ih) + oy, lattice_coord(v.z, ih) + oz, v.w);
      }
    }
    const int ns = S.nb_off[q1] - S.nb_off[q0];
    if (x.tid < ((8 - (ns & 7)) & 7)) ((float4*)S.src)[ns + x.tid] = nfmma::pad_record();
  } else {
    const V4* spos = (const V4*)d.spos64;
    for (int q = q0 + x.warp; q < q1; q += 4) {
      const int qq = q == 0 ? 13 : (q <= 13 ? q - 1 : q);
      const int ux = x.lx + qq % 3 - 1, uy = x.ly + (qq / 3) % 3 - 1, uz = x.lz + qq / 9 - 1;
      const int shx = ux - wrap1(ux, nL), shy = uy - wrap1(uy, nL), shz = uz - wrap1(uz, nL);
      const int e0 = S.nb_off[q] - S.nb_off[q0];
      for (int j = x.lane; j < S.nb_cnt[q]; j += 32) {  // lattice coordinates in this leaf's frame
        const V4 v = spos[S.nb_base[q] + j];
        NearField<T>::stage(S.src, e0 + j, lattice_coord(v.x, ih) - x.gx0 + shx * W,
                            lattice_coord(v.y, ih) - x.gy0 + shy * W, lattice_coord(v.z, ih) - x.gz0 + shz * W, v.w);
      }
    }
  }
  return true;
}

// Pair sums of the staged pass [q0, q1) for warp `warp` of the four that share
// it: the pass's sources (FP32: tiles of eight) are split evenly between the
// warps, and every warp evaluates all needed sites against its share; the
// partial sums meet in fixed point (integer adds are associative, so the
// potentials do not depend on the order in which the warps arrive).  Scale
// 2^ks with 2^ks * bound < 2^(bits - 2), bound = max|q| times the number of
// sources over the smallest separation (1 site).
template <typename T>
__device__ __forceinline__ void leaf_pairs(const Geo& g, const Dev& d, const LeafSmem<T>& S, int nsites, int q0, int q1,
                                           T scale, int warp, int lane) {
  constexpr bool F32 = sizeof(T) == 4;
  const int W = g.W, W3 = W * W * W;
  const int ns = S.nb_off[q1] - S.nb_off[q0];
  const int nu = F32 ? (ns + 7) >> 3 : ns;
  const int u0 = (nu * warp) >> 2, u1 = (nu * (warp + 1)) >> 2;
  if (u1 <= u0) return;
  if constexpr (F32) {
    const int jg = min(max(q0 == 0 ? (S.nb_cnt[0] + 7) >> 3 : 0, u0), u1);  // own-leaf tiles lead pass 0
    const int nts = (nsites + 15) >> 4;
    const uint32_t* R = (const uint32_t*)S.src;
    int* acc = (int*)S.phis;
    for (int t0 = 0; t0 < nts; t0 += nfmma::TMAX) {
      const int nt = min(nfmma::TMAX, nts - t0);
      if (nt == 2) nfmma::round<2>(R, S.sites, nsites, W, t0, u0, jg, u1, acc, scale, lane, d.err);
      else nfmma::round<1>(R, S.sites, nsites, W, t0, u0, jg, u1, acc, scale, lane, d.err);
    }
  } else {
    const int nisq = 3 * (2 * W - 1) * (2 * W - 1) + 1;
    long long* acc = (long long*)S.phis;
    for (int rb = 0; rb < nsites; rb += 64) {
      const int b0 = rb + lane, b1 = b0 + 32;
      const bool two = rb + 32 < nsites;  // warp-uniform
      const int sv0 = b0 < nsites ? S.sites[b0] : 0, sv1 = b1 < nsites ? S.sites[b1] : 0;
      const int ix0 = sv0 & 15, iy0 = (sv0 >> 4) & 15, iz0 = sv0 >> 8;
      const int ix1 = sv1 & 15, iy1 = (sv1 >> 4) & 15, iz1 = sv1 >> 8;
      const int l0 = ix0 + W * (iy0 + W * iz0), l1 = ix1 + W * (iy1 + W * iz1);
      NearField<T> nf;
      nf.reset();
      nf.run2(S.src, S.isq, u0, u1, two, ix0, iy0, iz0, ix1, iy1, iz1, nisq, d.err);
      if (b0 < nsites && KMC_IN(l0 >= 0 && l0 < W3, d.err)) fixed_add(&acc[l0], nf.sum(0) * scale);
      if (two && b1 < nsites && KMC_IN(l1 >= 0 && l1 < W3, d.err)) fixed_add(&acc[l1], nf.sum(1) * scale);
    }
  }
}

// Finish of a leaf whose fixed-point near-field sums are complete: PROP_FILL
// writes them to the near-field cache; otherwise (4) near field back to
// floating point plus the L2P of the leaf's local expansion at every needed
// site, then (5) the write-out of old-position potentials and unmasked hop
// potentials by re-enumerating the hops of phase 2.  Potentials are written
// in precision T (FP32 arrays in the mixed form, FP64 arrays in the FP64 form).
template <typename T, int NH, int mode>
__device__ __forceinline__ void leaf_finish(const Geo& g, const Dev& d, const LeafSmem<T>& S, const LeafCtx& x,
                                            int nsites) {
  typedef typename cplx<T>::type C;
  typedef typename vec4<T>::type V4;
  constexpr bool F32 = sizeof(T) == 4;
  typedef typename std::conditional<F32, int, long long>::type Acc;
  const int W = g.W, W3 = W * W * W, nbw = (W3 + 31) / 32, E = g.E;
  const int tid = x.tid, lane = x.lane, warp = x.warp;
  const T h = (T)g.h, ih = (T)(1.0 / g.h);
  const V4* spos = (const V4*)(F32 ? (const void*)d.spos32 : (const void*)d.spos64);
  T* out_old = (T*)(F32 ? (void*)d.phi_old32 : (void*)d.phi_old);
  T* out_new = (T*)(F32 ? (void*)d.phi_new32 : (void*)d.phi_new);
  const Acc* acc = (const Acc*)S.phis;
  const int ks = S.misc[1];
  constexpr int hs = NH == KMC_NHOP ? 0 : 1, ne = hs ? 27 : 1 + KMC_NHOP, nhop = NH;
  (void)nbw;
  if (mode == PROP_FILL) {  // the sums at every site into the cache, rescaled to 2^-near_ks
    __syncthreads();
    const int sh = g.near_ks - ks;
    long long* dst = d.nearfx + x.leaf * (int64_t)g.cap;
    for (int b = tid; b < nsites; b += 128) {
      const int sv = S.sites[b];
      const int l = (sv & 15) + W * (((sv >> 4) & 15) + W * (sv >> 8));
      if (!KMC_IN(l >= 0 && l < W3 && W3 <= g.cap, d.err)) continue;
      const long long a = (long long)acc[l];
      dst[l] = sh >= 0 ? a * (1LL << sh) : (a + (1LL << (-sh - 1))) >> -sh;
    }
    return;
  }
  // the outputs were recorded by the site phases unless the leaf had more than
  // wlist_cap of them; then its hops are enumerated again, and the inputs of
  // that (first 32 charges of this warp's first two entries) are loaded now,
  // so that their latency passes during the L2P
  const int nw = S.misc[3];
  const bool listed = nw <= wlist_cap<NH>();
  V4 wv[2];
  int32_t wu[2];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const int e = warp + 4 * i;
    if (!listed && e < ne) {
      const int li = c_ent_leaf[hs][e];
      if (lane < S.nb_cnt[li]) {
        wu[i] = d.uid[S.nb_base[li] + lane];
        wv[i] = spos[S.nb_base[li] + lane];
      }
    }
  }
  __syncthreads();
  {
    const T hw = (T)(0.5 * W);
    const T back = (T)ldexp(1.0, -ks) * ih;  // lattice units to physical
    const T cback = (T)ldexp(1.0, -g.near_ks) * ih;
    const long long* cache = mode == PROP_CACHED ? d.nearfx + x.leaf * (int64_t)g.cap : nullptr;
    for (int b = tid; b < nsites; b += 128) {
      const int sv = S.sites[b];
      const int ix = sv & 15, iy = (sv >> 4) & 15, iz = sv >> 8;
      const int l = ix + W * (iy + W * iz);
      if (!KMC_IN(l >= 0 && l < W3, d.err)) continue;
      const T near = cache ? (T)cache[l] * cback : (T)acc[l] * back;
      S.phis[l] = near + l2p_point<T, C>(S.Lc, g.p, (small_to<T>(ix) + (T)0.5 - hw) * h,
                                         (small_to<T>(iy) + (T)0.5 - hw) * h, (small_to<T>(iz) + (T)0.5 - hw) * h);
    }
  }
  __syncthreads();
  if (listed) {  // (5) write-out from the recorded list
    for (int i = tid; i < nw; i += 128) {
      const int2 w = S.wl[i];
      if (!KMC_IN(w.y >= 0 && w.y < W3, d.err)) continue;
      const T v = S.phis[w.y];
      if (w.x < 0) {
        out_old[-1 - w.x] = v;
      } else {
        out_new[w.x] = v;
        d.mask[w.x] = 1;
      }
    }
    return;
  }
#pragma unroll 1
  for (int i = 0; i < (ne + 3) / 4; i++) {
    const int e = warp + 4 * i;
    if (e >= ne) break;
    const int li = c_ent_leaf[hs][e];
    const uint32_t hm = c_ent_hops[hs][e];
    const int64_t mb = S.nb_base[li];
    const int cm = S.nb_cnt[li];
    for (int j = lane; j < cm; j += 32) {
      const bool pre = j < 32 && i < 2;
      const int32_t u = pre ? (i == 0 ? wu[0] : wu[1]) : d.uid[mb + j];
      const V4 v = pre ? (i == 0 ? wv[0] : wv[1]) : spos[mb + j];
      const int gx = lattice_coord(v.x, ih), gy = lattice_coord(v.y, ih), gz = lattice_coord(v.z, ih);
      if (!KMC_IN(u >= 0 && u < g.n, d.err)) continue;
      if (e == 0) {
        const int lo = (gx - x.gx0) + W * ((gy - x.gy0) + W * (gz - x.gz0));
        if (KMC_IN(lo >= 0 && lo < W3, d.err)) out_old[u] = S.phis[lo];
      }
      for (uint32_t hb = hm; hb; hb &= hb - 1) {
        const int k = __ffs(hb) - 1;
        const int rx = gx + hop_c(k, 0), ry = gy + hop_c(k, 1), rz = gz + hop_c(k, 2);
        if (g.bc && (rx < 0 || rx >= E || ry < 0 || ry >= E || rz < 0 || rz >= E)) continue;  // phase 2
        const int tx = wrap1(rx, E), ty = wrap1(ry, E), tz = wrap1(rz, E);
        const int ux = tx - x.gx0, uy = ty - x.gy0, uz = tz - x.gz0;
        if (ux < 0 || ux >= W || uy < 0 || uy >= W || uz < 0 || uz >= W) continue;
        const int lt = ux + W * (uy + W * uz);
        if (S.bits[lt >> 5] & (1u << (lt & 31))) continue;  // masked: written in phase 2
        out_new[(int64_t)nhop * u + k] = S.phis[lt];
        d.mask[(int64_t)nhop * u + k] = 1;
      }
    }
  }
}

// One leaf by one CTA of four warps (the per-leaf kernels: FP64 form, the
// near-field cache modes, replica batches): setup, sites, then the source
// passes (staged, summed) and the finish.
// mode: PROP_SUM (the pair sums of this step), PROP_FILL (pair sums at every
// site of the leaf into the near-field cache d.nearfx; no hops, no L2P, no
// outputs) or PROP_CACHED (the near-field sums read from the cache, no pairs).
template <typename T, int NH, int mode>
__device__ __forceinline__ void propose_leaf(const Geo& g, const Dev& d, const int chunk, const int64_t leaf) {
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(128) unsigned char sm[];
  const LeafSmem<T> S(sm, g, chunk);
  const LeafCtx x = leaf_ctx(g, leaf, threadIdx.x);
  leaf_setup<T, mode>(g, d, S, x, chunk);
  const int nsites = leaf_sites<T, NH, mode>(g, d, S, x);
  // no sites: only the first pass's copies to drain; cached sums: no pairs (and no copies)
  const int npass = mode == PROP_CACHED ? 0 : (nsites ? S.misc[0] : 1);
  for (int pass = 0; pass < npass; pass++)
    (void)KMC_IN(S.nb_off[S.pq[pass + 1]] - S.nb_off[S.pq[pass]] <= chunk, d.err);
  const T scale = (T)ldexp(1.0, S.misc[1]);
  for (int pass = 0; pass < npass; pass++) {
    const int q0 = S.pq[pass], q1 = S.pq[pass + 1];
    if (pass > 0) {
      __syncthreads();  // everyone is done with the previous pass's sources
      if (F32 && x.tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(S.bar, (uint32_t)(16 * (S.nb_off[q1] - S.nb_off[q0])));
        for (int q = q0; q < q1; q++)
          if (S.nb_cnt[q])
            bulk_copy_g2s(S.src + 16 * (S.nb_off[q] - S.nb_off[q0]), d.spos32 + S.nb_base[q],
                          (uint32_t)(16 * S.nb_cnt[q]), S.bar);
      }
    }
    if (!leaf_stage<T>(g, d, S, x, q0, q1, pass & 1)) return;
    __syncthreads();
    leaf_pairs<T>(g, d, S, nsites, q0, q1, scale, x.warp, x.lane);
  }
  leaf_finish<T, NH, mode>(g, d, S, x, nsites);
}

// one CTA per leaf of one system
template <typename T, int NH, int mode>
__global__ void __launch_bounds__(PROP_THREADS, mode == PROP_CACHED ? 12 : 9)
    k_propose_lattice(const Geo g, const Dev d, int chunk) {
  propose_leaf<T, NH, mode>(g, d, chunk, (int64_t)blockIdx.x);
}

// one CTA per leaf of every replica of a batch (blocks [off[r], off[r + 1]) are replica r's leaves)
template <typename T, int NH, int mode>
__global__ void __launch_bounds__(PROP_THREADS, mode == PROP_CACHED ? 12 : 9)
    k_propose_batch(const BatchRep* reps, const int* off, int R, int chunk) {
  const int r = batch_find(off, R, blockIdx.x);
  propose_leaf<T, NH, mode>(reps[r].g, reps[r].d, chunk, (int64_t)blockIdx.x - off[r]);
}

static size_t propose_smem(const Geo& g, int prec, int chunk) {
  const size_t ts = prec == 0 ? 8 : 4;
  const int W3 = g.W * g.W * g.W;
  const int nbw = (W3 + 31) / 32;
  const size_t srcb = prec == 0 ? NearField<double>::bytes(chunk) : nfmma::bytes(chunk);
  const size_t isqb = prec == 0 ? 8 + 8 * (size_t)(3 * (2 * g.W - 1) * (2 * g.W - 1) + 1) : 0;
  const size_t wlb = 8 + 8 * (size_t)(g.nhop == KMC_MAXHOP ? wlist_cap<KMC_MAXHOP>() : wlist_cap<KMC_NHOP>());
  return srcb + 2 * ts * (size_t)g.P + 27 * 8 + 8 + (28 + 27 + 27 + 28 + 4) * 4 + ts * (size_t)W3 +
         4 * (size_t)(3 * nbw + 1) + 2 * (size_t)((W3 + 1) & ~1) + isqb + wlb;
}

// sources are streamed in chunks of at least 960 (every neighbour leaf's
// charges in one pass unless the neighbourhood is dense: 27 x 32 = 864 on
// average at 1/16 occupancy and 8^3-site leaves), small enough for nine
// 128-thread CTAs per SM
static int propose_chunk(const Geo& g) {
  int c = 960 > g.cap ? 960 : g.cap;
  return (c + 1) & ~1;
}

static void kmc_preload();

template <int MODE>
static void prepare_m(const Geo& g, int prec, size_t sm) {
  if (g.nhop == KMC_MAXHOP) {
    if (prec == 0) raise_dynamic_smem((const void*)k_propose_lattice<double, KMC_MAXHOP, MODE>, sm);
    else raise_dynamic_smem((const void*)k_propose_lattice<float, KMC_MAXHOP, MODE>, sm);
  } else {
    if (prec == 0) raise_dynamic_smem((const void*)k_propose_lattice<double, KMC_NHOP, MODE>, sm);
    else raise_dynamic_smem((const void*)k_propose_lattice<float, KMC_NHOP, MODE>, sm);
  }
}

void kmc_prepare(const Geo& g, int prec) {
  kmc_preload();
  if (g.E <= 0) return;
  const int chunk = propose_chunk(g);
  const size_t sm = propose_smem(g, prec, chunk);
  prepare_m<PROP_SUM>(g, prec, sm);
  if (g.near_cache) {
    prepare_m<PROP_FILL>(g, prec, sm);
    prepare_m<PROP_CACHED>(g, prec, propose_smem(g, prec, 0));
  }
}

template <int MODE>
static void propose_launch_m(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  const int chunk = MODE == PROP_CACHED ? 0 : propose_chunk(g);  // cached sums: no source staging
  const size_t sm = propose_smem(g, prec, chunk);
  const unsigned nb = (unsigned)g.ML;
  if (g.nhop == KMC_MAXHOP) {
    if (prec == 0) k_propose_lattice<double, KMC_MAXHOP, MODE><<<nb, PROP_THREADS, sm, s>>>(g, d, chunk);
    else k_propose_lattice<float, KMC_MAXHOP, MODE><<<nb, PROP_THREADS, sm, s>>>(g, d, chunk);
  } else {
    if (prec == 0) k_propose_lattice<double, KMC_NHOP, MODE><<<nb, PROP_THREADS, sm, s>>>(g, d, chunk);
    else k_propose_lattice<float, KMC_NHOP, MODE><<<nb, PROP_THREADS, sm, s>>>(g, d, chunk);
  }
}

static void propose_launch(const Geo& g, const Dev& d, int prec, int mode, cudaStream_t s) {
  if (mode == PROP_CACHED) propose_launch_m<PROP_CACHED>(g, d, prec, s);
  else if (mode == PROP_FILL) propose_launch_m<PROP_FILL>(g, d, prec, s);
  else propose_launch_m<PROP_SUM>(g, d, prec, s);
}

void kmc_propose_lattice(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  propose_launch(g, d, prec, g.near_cache ? PROP_CACHED : PROP_SUM, s);
}

// near-field cache: the pair sums at every site of every leaf
void kmc_near_fill(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  if (g.near_cache) propose_launch(g, d, prec, PROP_FILL, s);
}

// ------------------------------------------------------------------ dU, rates, block sums
// thread per particle; FP64 assembly.  Block sums are sequential over the
// block's threads so that the selection walk reproduces them exactly.
#define FIN_THREADS KMC_FIN_PARTICLES
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exact FP32 -> FP64 widening of a non-negative normal or zero value by
// moving the IEEE-754 fields (integer pipe; on this GPU a converting
// instruction costs as much as FP64 arithmetic)
__device__ __forceinline__ double widen_nonneg(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t e = b >> 23;
  if (e == 0) return 0.0;
  const uint64_t bits = ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// Inclusive scan of one value per thread over the first n threads of the block
// (n a power of two, 32..1024; every thread of the block calls it, the others'
// results are meaningless): Kogge-Stone by shuffles within each warp, then over
// the warp totals; the last lane of warp w takes the warp-total scan's own
// entry.  The total (element n - 1) is then the sum over aligned blocks level
// by level -- the same additions, bit for bit, as block_total and as the last
// element of a Hillis-Steele scan -- with two barriers in all.
// wt: 32 doubles of shared memory.
__device__ __forceinline__ double block_scan_shfl(double x, int n, double* wt) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = n >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31 && w < nw) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? wt[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o && o < nw) t += y;
    }
    if (lane < nw) wt[lane] = t;
  }
  __syncthreads();
  if (w >= nw) return 0.0;
  if (lane == 31) return wt[w];
  return w > 0 ? x + wt[w - 1] : x;
}

// the block total of one value per thread (blockDim.x == n, a power of two) as
// adjacent aligned blocks added level by level (v: n doubles of shared memory)
__device__ __forceinline__ double block_total(double* v, int n) {
  for (int off = 1; off < n; off <<= 1) {
    if ((threadIdx.x & (2 * off - 1)) == 0) v[threadIdx.x] += v[threadIdx.x + off];
    __syncthreads();
  }
  return v[0];
}


// rate = m 2^-e for m in (0.5, 1] and 0 <= e <= 1021, formed by moving the
// IEEE-754 fields (exact; no FP64 arithmetic)
__device__ __forceinline__ double scale_pow2(float m, int e) {
  const uint32_t b = __float_as_uint(m);
  const uint64_t bits = ((uint64_t)((b >> 23) + 896u - (uint32_t)e) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// One thread per particle i and its 6 events j = 6 i + k: phi_new and mask
// read and dU and rate written as 8- and 16-byte vectors.  The per-particle
// sum of the 6 rates is sequential in k and the block sum equals the last
// element of the same fixed-order scan the selection walk takes, so both see
// the same cumulative sums.
// MIXED: the assembly in FP32 (the dU tolerance of the mixed form is far
// above FP32 rounding); rate = exp(-x) = 2^-y, y = x log2(e) = n + f, with
// 2^-f from the MUFU ex2 and 2^-n put into the FP64 exponent, so rates keep
// FP64 range down to 2^-1021 (an FP64 exp below that).  FP64: every
// operation in FP64.
template <bool MIXED, int NH>
__device__ __forceinline__ void finalize_blk(const Geo& g, const Dev& d, const int blk0) {
  __shared__ double ts[FIN_THREADS];
  const int64_t blk = (int64_t)blockIdx.x - blk0;
  const int64_t i = blk * FIN_THREADS + threadIdx.x;
  double tsum = 0.0;
  if (i < g.n) {
    const int E = g.E;
    const int s = d.site[i];
    const int cc[3] = {s % E, (s / E) % E, s / (E * E)};
    const uint16_t* mk = (const uint16_t*)(d.mask + NH * i);
    double r6[NH];
    // Dirichlet walls: the mirrors propose nothing, hops through a wall are
    // masked, and a hop moves the charge with its mirror:
    //   dU = dU_1 - q^2/2 [C(r' - r'_m) - 2 C(r' - r_m) + C(r - r_m)] - q E_z dz
    const bool dirw = g.dirichlet != 0, mirror = dirw && i >= g.nphys;
    const int half = E >> 1;
    if (MIXED) {
      const float q = d.q32[i], po = d.phi_old32[i], ikT = (float)(1.0 / g.kT);
      const float2* pn = (const float2*)(d.phi_new32 + NH * i);
      float du[NH];
#pragma unroll
      for (int k2 = 0; k2 < NH / 2; k2++) {
        const float2 v = pn[k2];
        const uint32_t mb = mk[k2];
#pragma unroll
        for (int o = 0; o < 2; o++) {
          const int k = 2 * k2 + o;
          // the dipole change of the wrapped hop vector (components of the
          // hop, minus the box edge where it crosses the periodic boundary)
          float qd = 0.f;
#pragma unroll
          for (int ax = 0; ax < 3; ax++) {
            const int hc = hop_c(k, ax);
            if (hc == 0) continue;
            float dw = hc > 0 ? (float)g.h : -(float)g.h;
            if (hc > 0 && cc[ax] == E - 1) dw -= (float)g.a;
            if (hc < 0 && cc[ax] == 0) dw += (float)g.a;
            qd += q * d.fdip[ax] * dw;
          }
          const float pv = o ? v.y : v.x;
          float duf = __int_as_float(0x7fc00000);
          double r = 0.0;
          bool on = o ? (mb >> 8) : (mb & 0xff);
          const int zn = cc[2] + hop_c(k, 2);
          if (dirw && (mirror || zn < 0 || zn >= half)) {
            if (on) d.mask[NH * i + k] = 0;
            on = false;
          }
          if (on) {
            duf = q * (pv - po) - qd - q * q * d.selfc32[k];
            if (dirw)
              duf -= 0.5f * q * q * (d.dirA32[zn] - 2.f * d.dirB32[k * half + cc[2]] + d.dirA32[cc[2]]) +
                     q * (float)(g.field_z * g.h) * (float)hop_c(k, 2);
            const float y = fmaxf(duf, 0.f) * ikT * 1.4426950408889634f;
            const float n = floorf(y);
            const int e = __float_as_int(n + 12582912.0f) - 0x4B400000;  // exact integer value of n
            r = e <= 1021 ? scale_pow2(ex2_approx(n - y), e) : exp(-(double)fmaxf(duf, 0.f) / g.kT);
          }
          du[k] = duf;
          r6[k] = r;
        }
      }
      float2* dout = (float2*)(d.dU32 + NH * i);
#pragma unroll
      for (int k2 = 0; k2 < NH / 2; k2++) dout[k2] = make_float2(du[2 * k2], du[2 * k2 + 1]);
    } else {
      const double q = d.q[i], po = d.phi_old[i];
      const double2* pn = (const double2*)(d.phi_new + NH * i);
      const double cdip = g.dipc;
      double du[NH];
#pragma unroll
      for (int k2 = 0; k2 < NH / 2; k2++) {
        const double2 v = pn[k2];
        const uint32_t mb = mk[k2];
#pragma unroll
        for (int o = 0; o < 2; o++) {
          const int k = 2 * k2 + o;
          double qd = 0.0;
#pragma unroll
          for (int ax = 0; ax < 3; ax++) {
            const int hc = hop_c(k, ax);
            if (hc == 0) continue;
            double dw = hc > 0 ? g.h : -g.h;
            if (hc > 0 && cc[ax] == E - 1) dw -= g.a;
            if (hc < 0 && cc[ax] == 0) dw += g.a;
            qd += q * (cdip * d.dip[ax]) * dw;
          }
          double dd = __longlong_as_double(0x7ff8000000000000LL), r = 0.0;
          bool on = o ? (mb >> 8) : (mb & 0xff);
          const int zn = cc[2] + hop_c(k, 2);
          if (dirw && (mirror || zn < 0 || zn >= half)) {
            if (on) d.mask[NH * i + k] = 0;
            on = false;
          }
          if (on) {
            dd = q * ((o ? v.y : v.x) - po) - qd - q * q * d.selfc[k];
            if (dirw)
              dd -= 0.5 * q * q * (d.dirA[zn] - 2.0 * d.dirB[k * half + cc[2]] + d.dirA[cc[2]]) +
                    q * g.field_z * g.h * hop_c(k, 2);
            r = exp(-fmax(dd, 0.0) / g.kT);
          }
          du[k] = dd;
          r6[k] = r;
        }
      }
      double2* dout = (double2*)(d.dU + NH * i);
#pragma unroll
      for (int k2 = 0; k2 < NH / 2; k2++) dout[k2] = make_double2(du[2 * k2], du[2 * k2 + 1]);
    }
    double2* rout = (double2*)(d.rate + NH * i);
#pragma unroll
    for (int k2 = 0; k2 < NH / 2; k2++) rout[k2] = make_double2(r6[2 * k2], r6[2 * k2 + 1]);
#pragma unroll
    for (int k = 0; k < NH; k++) tsum += r6[k];
  }
  ts[threadIdx.x] = tsum;
  __syncthreads();
  // the block sum as the selection's scan forms its last element (the same additions, bit for
  // bit), with a seventh of a scan's FP64 adds
  static_assert((FIN_THREADS & (FIN_THREADS - 1)) == 0, "aligned pairs need a power of two");
  const double tot = block_total(ts, FIN_THREADS);
  if (threadIdx.x == 0) d.bsum[blk] = tot;
}

template <bool MIXED, int NH>
__global__ void __launch_bounds__(FIN_THREADS) k_finalize(const Geo g, const Dev d) {
  finalize_blk<MIXED, NH>(g, d, 0);
}

template <bool MIXED, int NH>
__global__ void __launch_bounds__(FIN_THREADS) k_finalize_batch(const BatchRep* reps, const int* off, int R) {
  const int r = batch_find(off, R, blockIdx.x);
  finalize_blk<MIXED, NH>(reps[r].g, reps[r].d, off[r]);
}

// block sums of caller-provided rates (same block structure as k_finalize)
__global__ void __launch_bounds__(FIN_THREADS) k_rate_bsum(const Geo g, const Dev d) {
  __shared__ double ts[FIN_THREADS];
  int64_t i = blockIdx.x * (int64_t)FIN_THREADS + threadIdx.x;
  double tsum = 0.0;
  if (i < g.n)
    for (int k = 0; k < g.nhop; k++) tsum += d.rate[(int64_t)g.nhop * i + k];
  ts[threadIdx.x] = tsum;
  __syncthreads();
  const double tot = block_total(ts, FIN_THREADS);
  if (threadIdx.x == 0) d.bsum[blockIdx.x] = tot;
}

void kmc_finalize_rates(const Geo& g, const Dev& d, int prec, cudaStream_t s) {
  unsigned nb = (unsigned)((g.n + FIN_THREADS - 1) / FIN_THREADS);
  if (g.nhop == KMC_MAXHOP) {
    if (prec == 0) k_finalize<false, KMC_MAXHOP><<<nb, FIN_THREADS, 0, s>>>(g, d);
    else k_finalize<true, KMC_MAXHOP><<<nb, FIN_THREADS, 0, s>>>(g, d);
  } else {
    if (prec == 0) k_finalize<false, KMC_NHOP><<<nb, FIN_THREADS, 0, s>>>(g, d);
    else k_finalize<true, KMC_NHOP><<<nb, FIN_THREADS, 0, s>>>(g, d);
  }
}

// ------------------------------------------------------------------ selection
// Q = sum of all rates; event j with R_{j-1} < Q zeta <= R_j (Algorithm 1),
// where R is the cumulative sum taken block by block (block sums from the
// finalize kernel, chunks of block sums per thread here); dt = -ln(xi)/Q.
#define SEL_THREADS 1024

__device__ __forceinline__ void select_one(const Geo& g, const Dev& d, const int use_counter) {
  __shared__ double cs[SEL_THREADS];
  __shared__ double ts[FIN_THREADS];
  __shared__ double wt[32];
  __shared__ double sh_target, sh_prev;
  __shared__ int sh_t;
  __shared__ int64_t sh_blk;
  const int tid = threadIdx.x;
  const int64_t nb = (g.n + FIN_THREADS - 1) / FIN_THREADS;
  const int64_t per = (nb + SEL_THREADS - 1) / SEL_THREADS;
  const double* uni = use_counter ? d.uni_run + 2 * (int64_t)(*d.stepc) : d.uni_small;
  const double zeta = uni[0], xi = uni[1];
  double c = 0.0;
  for (int64_t b = tid * per; b < min(nb, (tid + 1) * per); b++) c += d.bsum[b];
  if (tid == 0) { sh_t = -1; sh_blk = -1; }
  cs[tid] = block_scan_shfl(c, SEL_THREADS, wt);
  __syncthreads();
  const double Q = cs[SEL_THREADS - 1];
  const double target = Q * zeta;
  if (Q > 0.0) {
    double prev = tid ? cs[tid - 1] : 0.0;
    if (prev < target && target <= cs[tid]) { sh_t = tid; sh_prev = prev; }
  }
  __syncthreads();
  if (tid == 0) {
    d.dtq[1] = Q;
    d.dtq[0] = (Q > 0.0) ? -log(xi) / Q : __longlong_as_double(0x7ff0000000000000LL);
    int t = sh_t;
    if (Q > 0.0 && t < 0) {  // rounding: last chunk with weight
      for (int u = SEL_THREADS - 1; u >= 0; u--)
        if (cs[u] > (u ? cs[u - 1] : 0.0)) { t = u; break; }
      sh_prev = t ? cs[t - 1] : 0.0;
    }
    if (t >= 0) {
      double run = sh_prev;
      int64_t blk = -1, bend = min(nb, (t + 1) * per);
      for (int64_t b = t * per; b < bend; b++) {
        double bs = d.bsum[b];
        if (bs > 0.0 && run + bs >= target) { blk = b; break; }
        run += bs;
      }
      if (blk < 0)
        for (int64_t b = bend - 1; b >= t * per; b--)
          if (d.bsum[b] > 0.0) { blk = b; break; }
      sh_blk = blk;
      sh_target = target - run;
    }
  }
  __syncthreads();
  const int64_t blk = sh_blk;
  if (blk < 0) {
    if (tid == 0) *d.event = -1;
    return;
  }
  double t = 0.0;
  if (tid < FIN_THREADS) {
    int64_t i = blk * FIN_THREADS + tid;
    if (i < g.n)
      for (int k = 0; k < g.nhop; k++) t += d.rate[(int64_t)g.nhop * i + k];
  }
  if (tid == 0) sh_t = -1;
  t = block_scan_shfl(t, FIN_THREADS, wt);
  if (tid < FIN_THREADS) ts[tid] = t;
  __syncthreads();
  const double res = sh_target;
  if (tid < FIN_THREADS) {
    double prev = tid ? ts[tid - 1] : 0.0;
    if (prev < res && res <= ts[tid]) { sh_t = tid; sh_prev = prev; }
  }
  __syncthreads();
  if (tid == 0) {
    int t = sh_t;
    double run = sh_prev, rr = res;
    if (t < 0) {  // rounding between the block sum and its scan
      for (int u = FIN_THREADS - 1; u >= 0; u--)
        if (ts[u] > (u ? ts[u - 1] : 0.0)) { t = u; break; }
      run = t ? ts[t - 1] : 0.0;
      rr = ts[t];
    }
    int64_t i = blk * FIN_THREADS + t;
    int ksel = -1;
    for (int k = 0; k < g.nhop; k++) {
      double r = d.rate[(int64_t)g.nhop * i + k];
      if (r > 0.0 && run + r >= rr) { ksel = k; break; }
      run += r;
    }
    if (ksel < 0)
      for (int k = g.nhop - 1; k >= 0; k--)
        if (d.rate[(int64_t)g.nhop * i + k] > 0.0) { ksel = k; break; }
    *d.event = (int64_t)g.nhop * i + ksel;
  }
}

__global__ void __launch_bounds__(SEL_THREADS) k_select(const Geo g, const Dev d, int use_counter) {
  select_one(g, d, use_counter);
}

// one CTA per member of a batch (the device step counter of each member)
__global__ void __launch_bounds__(SEL_THREADS) k_select_batch(const BatchRep* reps) {
  select_one(reps[blockIdx.x].g, reps[blockIdx.x].d, 1);
}

void kmc_rate_bsum(const Geo& g, const Dev& d, cudaStream_t s) {
  unsigned nb = (unsigned)((g.n + FIN_THREADS - 1) / FIN_THREADS);
  k_rate_bsum<<<nb, FIN_THREADS, 0, s>>>(g, d);
}

void kmc_select(const Geo& g, const Dev& d, int use_counter, cudaStream_t s) {
  k_select<<<1, SEL_THREADS, 0, s>>>(g, d, use_counter);
}

// store the step's event and dt, advance the device step counter
__device__ __forceinline__ void record_one(const Dev& d) {
  int st = *d.stepc;
  d.ev_hist[st] = *d.event;
  d.dt_hist[st] = d.dtq[0];
  *d.stepc = st + 1;
}

__global__ void k_record(const Dev d) { record_one(d); }

void kmc_record(const Geo& g, const Dev& d, cudaStream_t s) {
  (void)g;
  k_record<<<1, 1, 0, s>>>(d);
}

// ------------------------------------------------------------------ accept
// Move record from a lattice event index (device resident, no host sync).
__device__ __forceinline__ void move_from_event_one(const Geo& g, const Dev& d) {
  MoveRec mv;
  int64_t j = *d.event;
  mv.valid = 0;
  if (j >= 0 && KMC_IN(j < (int64_t)g.nhop * g.n, d.err)) {
    int64_t i = j / g.nhop;
    int k = (int)(j - (int64_t)g.nhop * i);
    int E = g.E;
    int s = d.site[i];
    int gx = s % E, gy = (s / E) % E, gz = s / (E * E);
    int tx = (gx + hop_c(k, 0) + E) % E, ty = (gy + hop_c(k, 1) + E) % E, tz = (gz + hop_c(k, 2) + E) % E;
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
    mv.dU = g.prec ? (double)d.dU32[j] : d.dU[j];
  }
  *d.move = mv;
}

__global__ void k_move_from_event(const Geo g, const Dev d) { move_from_event_one(g, d); }

// thread per member of a batch: record the step's event, then its move record
__global__ void k_record_move_batch(const BatchRep* reps, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  record_one(reps[r].d);
  move_from_event_one(reps[r].g, reps[r].d);
}

void kmc_accept_from_event(const Geo& g, const Dev& d, cudaStream_t s) { k_move_from_event<<<1, 1, 0, s>>>(g, d); }

// Dirichlet walls: the accepted hop's mirror move -- charge i + nphys from
// (x, y, a - z) to (x', y', a - z') with charge -q -- for a second accept
// update; its energy change is already in the first record (dU = 0 here).
__device__ __forceinline__ int mirror_site(int s, int E) {
  const int x = s % E, y = (s / E) % E, z = s / (E * E);
  return x + E * (y + E * (E - 1 - z));
}
__global__ void k_mirror_move(const Geo g, const Dev d) {
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  mv.i += (int32_t)g.nphys;
  mv.site_old = mirror_site(mv.site_old, g.E);
  mv.site_new = mirror_site(mv.site_new, g.E);
  mv.q = -mv.q;
  mv.r[2] = g.a - mv.r[2];
  mv.rn[2] = g.a - mv.rn[2];
  mv.dU = 0.0;
  *d.move = mv;
}

void kmc_mirror_move(const Geo& g, const Dev& d, cudaStream_t s) { k_mirror_move<<<1, 1, 0, s>>>(g, d); }

// Dirichlet walls: U = 1/2 U_mirrored - E_z sum_phys q z (fixed-order reduction)
__global__ void k_dirichlet_energy(const Geo g, const Dev d) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < g.nphys; i += blockDim.x) a += d.q[i] * d.pos[3 * i + 2];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.U[0] = 0.5 * d.U[0] - g.field_z * sh[0];
}

void kmc_dirichlet_energy(const Geo& g, const Dev& d, cudaStream_t s) { k_dirichlet_energy<<<1, 256, 0, s>>>(g, d); }

// multipoles of the ancestors of the old and new positions, all levels:
// Mt_l[anc(r)] -= q R(r - c), Mt_l[anc(r')] += q R(r' - c).  thread per
// (level, coefficient); each value from the regular-harmonic recurrences.
// multipole_delta gives the change of coefficient ci on level l for both ends
// of the move (val[0]: -q at r, val[1]: +q at r'), and the two cells
__device__ __forceinline__ void multipole_delta(const Geo& g, const MoveRec& mv, int l, int ci, double2* val,
                                                int64_t* cell) {
  int n = 0;
  while (tri(n + 1, 0) <= ci) n++;
  const int m = ci - tri(n, 0);
  const int nl = 1 << (l - 1);
  const double wl = g.a / nl;
  for (int side = 0; side < 2; side++) {
    const double* x = side ? mv.rn : mv.r;
    const double q = side ? mv.q : -mv.q;
    const int cx = cell_at(x[0], nl, g.inv_a), cy = cell_at(x[1], nl, g.inv_a), cz = cell_at(x[2], nl, g.inv_a);
    cell[side] = cx + (int64_t)nl * (cy + (int64_t)nl * cz);
    const double dx = x[0] - (cx + 0.5) * wl, dy = x[1] - (cy + 0.5) * wl, dz = x[2] - (cz + 0.5) * wl;
    const double r2 = dx * dx + dy * dy + dz * dz;
    double2 mm = make_double2(1.0, 0.0);
    for (int j = 1; j <= m; j++) {
      const double sc = c_halfm_d[j];
      mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
    }
    double2 a1 = mm, a2 = make_double2(0.0, 0.0);
    for (int nn = m + 1; nn <= n; nn++) {
      const double cc = c_inv_d[tri(nn, m)];
      const double zz = (2 * nn - 1) * dz;
      const double2 v = make_double2((zz * a1.x - r2 * a2.x) * cc, (zz * a1.y - r2 * a2.y) * cc);
      a2 = a1;
      a1 = v;
    }
    val[side] = make_double2(q * a1.x, q * a1.y);
  }
}

__device__ __forceinline__ void acc_multipole_role(const Geo& g, const Dev& d, const MoveRec& mv, int t) {
  const int l = 1 + t / g.P, ci = t % g.P;
  if (l > g.L) return;
  double2 val[2];
  int64_t cell[2];
  multipole_delta(g, mv, l, ci, val, cell);
  if (cell[0] == cell[1]) {
    val[0].x += val[1].x;
    val[0].y += val[1].y;
  }
  const int nside = cell[0] == cell[1] ? 1 : 2;
  for (int side = 0; side < nside; side++) {
    double2* out = d.Mt + (g.cell_off[l] + cell[side]) * g.P + ci;
    double2 v = *out;
    v.x += val[side].x;
    v.y += val[side].y;
    *out = v;
  }
}

// far field: H += R dK with dK the level-1 multipole change (about the domain
// centre), computed by the block into shared memory; one warp per output
// coefficient, lanes split the (k, l) sum; fixed-order warp reduction.
__device__ __forceinline__ void acc_far_role(const Geo& g, const Dev& d, const MoveRec& mv, double2* dks, int blk) {
  for (int c = threadIdx.x; c < g.P; c += blockDim.x) {
    double2 val[2];
    int64_t cell[2];
    multipole_delta(g, mv, 1, c, val, cell);
    dks[c] = make_double2(val[0].x + val[1].x, val[0].y + val[1].y);
  }
  __syncthreads();
  const int ci = blk * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (ci >= g.P) return;
  int n = 0;
  while (tri(n + 1, 0) <= ci) n++;
  const int m = ci - tri(n, 0);
  const int nkl = (g.p + 1) * (g.p + 1);  // (k, l) pairs with l in [-k, k]
  double ax = 0.0, ay = 0.0;
  for (int t = lane; t < nkl; t += 32) {
    int k = 0;
    while ((k + 1) * (k + 1) <= t) k++;
    int ll = t - k * k - k;
    double2 a = tab_get(dks, k, ll), b = tab_get(d.S, n + k, m + ll);
    double sx = a.x * b.x + a.y * b.y, sy = a.y * b.x - a.x * b.y;
    if (k & 1) { ax -= sx; ay -= sy; }
    else { ax += sx; ay += sy; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  if (lane == 0) {
    double2* H = d.Psi + g.cell_off[1] * g.P;
    double2 v = H[ci];
    v.x += ax;
    v.y += ay;
    H[ci] = v;
    if (d.Psi32) d.Psi32[g.cell_off[1] * g.P + ci] = make_float2((float)v.x, (float)v.y);
  }
}

// P2L of a point charge q at offset (dx,dy,dz) from a cell centre, all (n, m):
// out[tri(n,m)] (+)= q conj(I_n^m(d)).
// column m of the P2L table of charge q at offset (dx, dy, dz) from the
// expansion centre: out[tri(n, m)] = q conj(I_n^m(d)) for n = m .. p
__device__ void p2l_column(double2* out, double q, double dx, double dy, double dz, int p, int m) {
  const double r2 = dx * dx + dy * dy + dz * dz, inv = 1.0 / r2;
  double2 mm = make_double2(1.0 / sqrt(r2), 0.0);
  for (int j = 1; j <= m; j++) {
    const double sc = -(2.0 * j - 1.0) * inv;
    mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
  }
  double2 a1 = mm, a2 = make_double2(0.0, 0.0), v = mm;
  for (int n = m; n <= p; n++) {
    if (n > m) {
      const double zz = (2 * n - 1) * dz;
      const double c2 = (double)((n - 1) * (n - 1) - m * m);
      v = make_double2((zz * a1.x - c2 * a2.x) * inv, (zz * a1.y - c2 * a2.y) * inv);
      a2 = a1;
      a1 = v;
    }
    out[tri(n, m)] = make_double2(q * v.x, -q * v.y);
  }
}

// The same columns from a group of 16 lanes (p <= 15): lane m of the group
// computes column m.  1/|d| and 1/|d|^2 are computed once (lane 0) and
// broadcast, and the sectoral values I_m^m(d) = prod_{j <= m} f_j with f_0 =
// 1/|d|, f_j = -(2j - 1) (dx + i dy) / |d|^2 come from an inclusive prefix
// product over the lanes (four shuffle steps), instead of every thread
// recomputing the square root, the division and its O(m) chain.  gmask: the
// group's 16 lanes; every lane of the group calls this (lanes m > p only take
// part in the shuffles).  T: the arithmetic of the column (FP64; FP32 in the
// mixed form: 0.101 -> 0.069 ms of the accept on the 1M-charge workload); the
// terms are added in FP64 into the FP64 expansions.
#define P2L_GROUP 16
template <typename T> __device__ __forceinline__ T p2l_rsqrt(T x);
template <> __device__ __forceinline__ float p2l_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double p2l_rsqrt<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ void p2l_group_column(double q, double dx_, double dy_, double dz_, int p, int m,
                                                 unsigned gmask, double2* acc_out, bool accumulate) {
  const T dx = (T)dx_, dy = (T)dy_, dz = (T)dz_;
  const T r2 = dx * dx + dy * dy + dz * dz;
  T inv = 0, rinv = 0;
  if (m == 0) {
    inv = (T)1 / r2;
    rinv = p2l_rsqrt<T>(r2);
  }
  inv = __shfl_sync(gmask, inv, 0, P2L_GROUP);
  rinv = __shfl_sync(gmask, rinv, 0, P2L_GROUP);
  T fx = m == 0 ? rinv : -((T)2 * m - (T)1) * inv * dx, fy = m == 0 ? (T)0 : -((T)2 * m - (T)1) * inv * dy;
#pragma unroll
  for (int o = 1; o < P2L_GROUP; o <<= 1) {
    const T tx = __shfl_up_sync(gmask, fx, o, P2L_GROUP), ty = __shfl_up_sync(gmask, fy, o, P2L_GROUP);
    if (m >= o) {
      const T nx = tx * fx - ty * fy, ny = tx * fy + ty * fx;
      fx = nx;
      fy = ny;
    }
  }
  if (m > p) return;
  T a1x = fx, a1y = fy, a2x = 0, a2y = 0, vx = fx, vy = fy;
  for (int n = m; n <= p; n++) {
    if (n > m) {
      const T zz = (T)(2 * n - 1) * dz;
      const T c2 = (T)((n - 1) * (n - 1) - m * m);
      vx = (zz * a1x - c2 * a2x) * inv;
      vy = (zz * a1y - c2 * a2y) * inv;
      a2x = a1x;
      a2y = a1y;
      a1x = vx;
      a1y = vy;
    }
    if (accumulate) {
      acc_out[n].x += q * (double)vx;
      acc_out[n].y -= q * (double)vy;
    } else {
      acc_out[tri(n, m)] = make_double2(q * (double)vx, -q * (double)vy);
    }
  }
}

// the image nu (0..26) of position x, seen from cell b on level l: true when
// its cell u = cell(x) + n_l nu lies in the interaction list of b, i.e.
// |floor(u/2) - floor(b/2)|_inf <= 1 and |u - b|_inf >= 2.
__device__ __forceinline__ int fdiv2(int u) { return (u >= 0) ? (u >> 1) : -((1 - u) >> 1); }
__device__ __forceinline__ bool image_in_il(const int u0[3], int nl, int nu, const int b[3]) {
  int nv[3] = {nu % 3 - 1, (nu / 3) % 3 - 1, nu / 9 - 1};
  bool in = true, far = false;
  for (int c = 0; c < 3; c++) {
    int u = u0[c] + nl * nv[c];
    if (abs(fdiv2(u) - (b[c] >> 1)) > 1) in = false;
    if (abs(u - b[c]) >= 2) far = true;
  }
  return in && far;
}

// coarse levels 2 and 3: thread per (cell, image of either position, m); the
// P2L tables go to a scratch area and are summed over the images in fixed order by
// k_acc_coarse_reduce.  Level 2 (8 cells) sees every image nu with
// |nu|_inf <= KMC_TOP (the block its interaction list covers) that is not one
// of the cell's 27 neighbours; level 3 (64 cells) the 27 nearest images under
// the usual interaction-list rule.  Slots: level-2 cell c, image i at
// c * 2 KMC_TOP_NIMG + i; level-3 cell c at the level-2 slots' end + c * 54 + i.
#define KMC_L2_SLOTS (8 * 2 * KMC_TOP_NIMG)
#define KMC_COARSE_SLOTS (KMC_L2_SLOTS + 64 * 54)
#define KMC_COARSE_CELLS 72

// lanes per P2L column set: a 16-lane group (p <= 15) or p + 1 threads (p > 15)
__host__ __device__ __forceinline__ int p2l_lanes(int p) { return p < P2L_GROUP ? P2L_GROUP : p + 1; }

__device__ __forceinline__ void acc_coarse_role(const Geo& g, const MoveRec& mv, double2* scratch, int t) {
  // t = (slot, m); with p <= 15 the 16 lanes of a slot form a shuffle group (slot uniform in it)
  const int lanes = p2l_lanes(g.p);
  const int slot = t / lanes, m = t - slot * lanes;
  if (slot >= KMC_COARSE_SLOTS) return;
  int l, cell, im, nimg1, span;
  if (slot < KMC_L2_SLOTS) {
    l = 2; cell = slot / (2 * KMC_TOP_NIMG); im = slot % (2 * KMC_TOP_NIMG); nimg1 = KMC_TOP_NIMG; span = KMC_TOP;
  } else {
    l = 3; cell = (slot - KMC_L2_SLOTS) / 54; im = (slot - KMC_L2_SLOTS) % 54; nimg1 = 27; span = 1;
  }
  const int nl = 1 << (l - 1);
  const int b[3] = {cell % nl, (cell / nl) % nl, cell / (nl * nl)};
  const double wl = g.a / nl;
  const int side = im / nimg1, nu = im % nimg1, w = 2 * span + 1;
  const int nv[3] = {nu % w - span, (nu / w) % w - span, nu / (w * w) - span};
  const double* x = side ? mv.rn : mv.r;
  const double q = side ? mv.q : -mv.q;
  int u0[3];
  for (int c = 0; c < 3; c++) u0[c] = cell_at(x[c], nl, g.inv_a);
  bool in_il;
  if (l == 2) {  // any image of the block that is not a neighbour of b
    bool far = false;
    for (int c = 0; c < 3; c++)
      if (abs(u0[c] + nl * nv[c] - b[c]) >= 2) far = true;
    in_il = far;
  } else {
    int nu27 = (nv[0] + 1) + 3 * ((nv[1] + 1) + 3 * (nv[2] + 1));
    in_il = image_in_il(u0, nl, nu27, b);
  }
  // free space: no images, and the level-2 interaction list is empty
  if (g.bc && (l == 2 || nv[0] || nv[1] || nv[2])) in_il = false;
  double2* out = scratch + (int64_t)slot * g.P;
  if (!in_il) {
    for (int n = m; n <= g.p; n++) out[tri(n, m)] = make_double2(0.0, 0.0);
    return;
  }
  double dx = x[0] + g.a * nv[0] - (b[0] + 0.5) * wl, dy = x[1] + g.a * nv[1] - (b[1] + 0.5) * wl,
         dz = x[2] + g.a * nv[2] - (b[2] + 0.5) * wl;
  if (g.p < P2L_GROUP) {
    if (g.prec == 1) p2l_group_column<float>(q, dx, dy, dz, g.p, m, 0xffffu << (threadIdx.x & 16), out, false);
    else p2l_group_column<double>(q, dx, dy, dz, g.p, m, 0xffffu << (threadIdx.x & 16), out, false);
  } else {
    p2l_column(out, q, dx, dy, dz, g.p, m);
  }
}

// one CTA (8 warps) per coarse cell: warp w sums the slots w, w + 8, ... of
// the cell (lanes over coefficients, coalesced rows), then the eight warp
// partials are added in warp order
#define ACR_WARPS 8
__device__ __forceinline__ void acc_coarse_reduce_blk(const Geo& g, const Dev& d, const double2* scratch, const int blk0) {
  extern __shared__ double2 acr[];  // [ACR_WARPS][P]
  MoveRec mv = *d.move;
  if (!mv.valid) return;
  const int cc = blockIdx.x - blk0, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int l, cell, first, nslot;
  if (cc < 8) { l = 2; cell = cc; first = cc * 2 * KMC_TOP_NIMG; nslot = 2 * KMC_TOP_NIMG; }
  else { l = 3; cell = cc - 8; first = KMC_L2_SLOTS + cell * 54; nslot = 54; }
  // eight slots in flight per lane (independent partial sums, combined in a fixed order)
  constexpr int ILP = 8;
  for (int c0 = 0; c0 < g.P; c0 += 32) {
    const int c = c0 + lane;
    if (c >= g.P) continue;
    double2 ps[ILP];
#pragma unroll
    for (int k = 0; k < ILP; k++) ps[k] = make_double2(0.0, 0.0);
    int s2 = warp;
    for (; s2 + (ILP - 1) * ACR_WARPS < nslot; s2 += ILP * ACR_WARPS) {
      double2 v[ILP];
#pragma unroll
      for (int k = 0; k < ILP; k++) v[k] = scratch[((int64_t)first + s2 + k * ACR_WARPS) * g.P + c];
#pragma unroll
      for (int k = 0; k < ILP; k++) {
        ps[k].x += v[k].x;
        ps[k].y += v[k].y;
      }
    }
    for (; s2 < nslot; s2 += ACR_WARPS) {
      const double2 v = scratch[((int64_t)first + s2) * g.P + c];
      ps[0].x += v.x;
      ps[0].y += v.y;
    }
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int k = 0; k < ILP; k++) {
      ax += ps[k].x;
      ay += ps[k].y;
    }
    acr[warp * g.P + c] = make_double2(ax, ay);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < g.P; c += blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int w = 0; w < ACR_WARPS; w++) {
      ax += acr[w * g.P + c].x;
      ay += acr[w * g.P + c].y;
    }
    const int64_t at = (g.cell_off[l] + cell) * g.P + c;
    double2 v = d.Psi[at];
    v.x += ax;
    v.y += ay;
    d.Psi[at] = v;
    if (d.Psi32) d.Psi32[at] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void __launch_bounds__(32 * ACR_WARPS) k_acc_coarse_reduce(const Geo g, const Dev d, const double2* scratch) {
  acc_coarse_reduce_blk(g, d, scratch, 0);
}

__global__ void __launch_bounds__(32 * ACR_WARPS) k_acc_coarse_reduce_batch(const BatchRep* reps, const int* off, int R) {
  const int r = batch_find(off, R, blockIdx.x);
  acc_coarse_reduce_blk(reps[r].g, reps[r].d, reps[r].d.acc_scratch, off[r]);
}

int kmc_coarse_slots() { return KMC_COARSE_SLOTS; }

// fine levels (n_l >= 8): the candidate cells are the children of the
// (wrapped) 3x3x3 parent neighbourhoods of the old and new positions' parent
// cells, each candidate handled by one thread that loops over the 54 images
// and accumulates the P2L of those in its interaction list.
__device__ __forceinline__ int wdist(int a, int b, int n) {
  int t = ((a - b) % n + n) % n;
  return min(t, n - t);
}

__device__ __forceinline__ void acc_fine_role(const Geo& g, const Dev& d, const MoveRec& mv, int l, int t) {
  // t = (candidate, m); with p <= 15 the 16 lanes of a candidate form a shuffle group
  const int lanes = p2l_lanes(g.p);
  int cand = t / lanes, m = t % lanes;
  if (cand >= 432) return;
  const int nl = 1 << (l - 1), np = nl >> 1;
  const double wl = g.a / nl;
  int side0 = cand / 216, rem = cand % 216;
  int di = rem >> 3, o = rem & 7;
  int dlt[3] = {di % 3 - 1, (di / 3) % 3 - 1, di / 9 - 1};
  const double* x0 = side0 ? mv.rn : mv.r;
  int P0[3], Pold[3];
  for (int c = 0; c < 3; c++) {
    P0[c] = cell_at(x0[c], np, g.inv_a);
    Pold[c] = cell_at(mv.r[c], np, g.inv_a);
  }
  int b[3];
  for (int c = 0; c < 3; c++) {
    if (g.bc && (P0[c] + dlt[c] < 0 || P0[c] + dlt[c] >= np)) return;  // free space: beyond the box
    b[c] = 2 * (((P0[c] + dlt[c]) % np + np) % np) + ((o >> c) & 1);
  }
  if (side0 == 1) {  // already covered by the old position's list?
    bool in_old = true;
    for (int c = 0; c < 3; c++)
      if ((g.bc ? abs((b[c] >> 1) - Pold[c]) : wdist(b[c] >> 1, Pold[c], np)) > 1) in_old = false;
    if (in_old) return;
  }
  double2 acc[KMC_MAXP + 1];
  for (int n = 0; n <= g.p; n++) acc[n] = make_double2(0.0, 0.0);
  bool any = false;
  for (int side = 0; side < 2; side++) {
    const double* x = side ? mv.rn : mv.r;
    double q = side ? mv.q : -mv.q;
    // n_l >= 8: the only image of the position's cell within three cells of b
    // is the minimum image; it contributes when it is in b's interaction list
    int nv[3];
    bool in = true, far = false;
    for (int c = 0; c < 3; c++) {
      const int u = cell_at(x[c], nl, g.inv_a);
      int du = b[c] - u;
      nv[c] = 0;
      if (!g.bc && 2 * du > nl) nv[c] = 1;  // periodic: the minimum image (free space: none)
      else if (!g.bc && 2 * du < -nl) nv[c] = -1;
      const int ui = u + nl * nv[c];
      if (abs(fdiv2(ui) - (b[c] >> 1)) > 1) in = false;
      if (abs(ui - b[c]) >= 2) far = true;
    }
    if (!(in && far)) continue;
    any = true;
    const double dx = x[0] + g.a * nv[0] - (b[0] + 0.5) * wl, dy = x[1] + g.a * nv[1] - (b[1] + 0.5) * wl,
                 dz = x[2] + g.a * nv[2] - (b[2] + 0.5) * wl;
    if (g.p < P2L_GROUP) {
      if (g.prec == 1) p2l_group_column<float>(q, dx, dy, dz, g.p, m, 0xffffu << (threadIdx.x & 16), acc, true);
      else p2l_group_column<double>(q, dx, dy, dz, g.p, m, 0xffffu << (threadIdx.x & 16), acc, true);
      continue;
    }
    const double r2 = dx * dx + dy * dy + dz * dz, inv = 1.0 / r2;
    double2 mm = make_double2(1.0 / sqrt(r2), 0.0);
    for (int j = 1; j <= m; j++) {
      const double sc = -(2.0 * j - 1.0) * inv;
      mm = make_double2(sc * (dx * mm.x - dy * mm.y), sc * (dx * mm.y + dy * mm.x));
    }
    double2 a1 = mm, a2 = make_double2(0.0, 0.0);
    acc[m].x += q * mm.x;
    acc[m].y -= q * mm.y;
    for (int n = m + 1; n <= g.p; n++) {
      const double zz = (2 * n - 1) * dz;
      const double c2 = (double)((n - 1) * (n - 1) - m * m);
      const double2 v = make_double2((zz * a1.x - c2 * a2.x) * inv, (zz * a1.y - c2 * a2.y) * inv);
      acc[n].x += q * v.x;
      acc[n].y -= q * v.y;
      a2 = a1;
      a1 = v;
    }
  }
  if (!any) return;
  const int64_t base = (g.cell_off[l] + b[0] + (int64_t)nl * (b[1] + (int64_t)nl * b[2])) * g.P;
  double2* out = d.Psi + base;
  // all loads first, then all stores (the row's coefficients are independent)
  for (int n = m; n <= g.p; n++) {
    double2 v = out[tri(n, m)];
    acc[n].x += v.x;
    acc[n].y += v.y;
  }
  for (int n = m; n <= g.p; n++) out[tri(n, m)] = acc[n];
  if (d.Psi32)
    for (int n = m; n <= g.p; n++) d.Psi32[base + tri(n, m)] = make_float2((float)acc[n].x, (float)acc[n].y);
}

// move the charge between leaf slots; dipole, energy and bookkeeping
__device__ __forceinline__ void acc_move_role(const Geo& g, const Dev& d, const MoveRec& mv) {
  int32_t i = mv.i;
  if (!KMC_IN(i >= 0 && i < g.n, d.err)) return;
  int32_t so = d.slot_of[i];
  int64_t lo = so / g.cap;
  int ln = 0;
  {
    int cx = cell_at(mv.rn[0], g.nL, g.inv_a), cy = cell_at(mv.rn[1], g.nL, g.inv_a), cz = cell_at(mv.rn[2], g.nL, g.inv_a);
    ln = cx + g.nL * (cy + g.nL * cz);
  }
  if (!KMC_IN(so >= 0 && lo < g.ML && so - lo * g.cap < d.cnt[lo] && ln >= 0 && ln < g.ML, d.err)) return;
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
  const double cdip = g.dipc;
  for (int c3 = 0; c3 < 3; c3++) {
    double m3 = d.dip[c3] + mv.q * (mv.rn[c3] - mv.r[c3]);
    d.dip[c3] = m3;
    d.fdip[c3] = (float)(cdip * m3);
  }
  d.U[0] += mv.dU;
}

// The independent parts of an accept in one launch, blocks taking roles by
// range: multipole changes of all levels, the far field, the coarse P2L
// columns (into scratch), the fine-level P2L updates (levels >= 4, each cell
// written by one thread) and the slot move.  They read only the move record
// and write disjoint data; the coarse columns are then summed per cell.
struct AccPlan {
  int nmp, nfar, ncoarse, nfine, fine_per_level;
};
#define ACC_THREADS 128
// the block ranges of the roles for a system of L levels and order p
__host__ __device__ __forceinline__ AccPlan acc_plan(const Geo& g) {
  AccPlan ap;
  ap.nmp = (g.L * g.P + ACC_THREADS - 1) / ACC_THREADS;
  ap.nfar = (g.P + ACC_THREADS / 32 - 1) / (ACC_THREADS / 32);
  // coarse levels 2 and 3 (8 + 64 cells, L >= 3 always): all cells x all images
  ap.ncoarse = (KMC_COARSE_SLOTS * p2l_lanes(g.p) + ACC_THREADS - 1) / ACC_THREADS;
  ap.fine_per_level = 432 * p2l_lanes(g.p);
  ap.nfine = g.L >= 4 ? (ap.fine_per_level * (g.L - 3) + ACC_THREADS - 1) / ACC_THREADS : 0;
  return ap;
}
__host__ __device__ __forceinline__ int acc_blocks(const AccPlan& ap) { return ap.nmp + ap.nfar + ap.ncoarse + ap.nfine + 1; }

__device__ __forceinline__ void acc_fused_blk(const Geo& g, const Dev& d, double2* scratch, const AccPlan& ap,
                                              const int blk0) {
  __shared__ double2 dks[ncoef(KMC_MAXP)];
  const MoveRec mv = *d.move;
  if (!mv.valid) return;
  int b = blockIdx.x - blk0;
  if (b < ap.nmp) {
    acc_multipole_role(g, d, mv, b * ACC_THREADS + threadIdx.x);
    return;
  }
  b -= ap.nmp;
  if (b < ap.nfar) {
    acc_far_role(g, d, mv, dks, b);
    return;
  }
  b -= ap.nfar;
  if (b < ap.ncoarse) {
    acc_coarse_role(g, mv, scratch, b * ACC_THREADS + threadIdx.x);
    return;
  }
  b -= ap.ncoarse;
  if (b < ap.nfine) {
    const int tf = b * ACC_THREADS + threadIdx.x;
    if (tf < ap.fine_per_level * (g.L - 3)) acc_fine_role(g, d, mv, 4 + tf / ap.fine_per_level, tf % ap.fine_per_level);
    return;
  }
  if (threadIdx.x == 0) acc_move_role(g, d, mv);
}

__global__ void __launch_bounds__(ACC_THREADS) k_acc_fused(const Geo g, const Dev d, double2* scratch, AccPlan ap) {
  acc_fused_blk(g, d, scratch, ap, 0);
}

__global__ void __launch_bounds__(ACC_THREADS) k_acc_fused_batch(const BatchRep* reps, const int* off, int R) {
  const int r = batch_find(off, R, blockIdx.x);
  const AccPlan ap = acc_plan(reps[r].g);
  acc_fused_blk(reps[r].g, reps[r].d, reps[r].d.acc_scratch, ap, off[r]);
}

// Near-field cache update for an accepted move of charge q from site r to site
// r'.  Block (side, o): the leaf T = S - o around the source leaf S of r (side
// 0, -q) or r' (side 1, +q); in T's frame the source sits at its position in
// S plus o W sites, as in T's propose CTA, so every site t of T gets
// +-q / |t - r_T| (lattice units), except
// the pair at distance 0.  Free space: leaves beyond the box do not exist.
__device__ __forceinline__ void near_update_blk(const Geo& g, const Dev& d, const int blk0) {
  const MoveRec mv = *d.move;
  if (!mv.valid || mv.site_old < 0 || mv.site_new < 0) return;
  const int bb = blockIdx.x - blk0;
  const int side = bb / 27, o = bb % 27;
  const int site = side ? mv.site_new : mv.site_old;
  const int E = g.E, W = g.W, nL = g.nL;
  if (!KMC_IN(site < E * E * E && W * W * W <= g.cap, d.err)) return;
  const int sx = site % E, sy = (site / E) % E, sz = site / (E * E);
  const int Sx = sx / W, Sy = sy / W, Sz = sz / W;
  const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
  int Tx = Sx - ox, Ty = Sy - oy, Tz = Sz - oz;
  if (g.bc) {
    if (Tx < 0 || Tx >= nL || Ty < 0 || Ty >= nL || Tz < 0 || Tz >= nL) return;
  } else {
    Tx = (Tx + nL) % nL;
    Ty = (Ty + nL) % nL;
    Tz = (Tz + nL) % nL;
  }
  const double rx = (double)(sx - Sx * W + ox * W), ry = (double)(sy - Sy * W + oy * W),
               rz = (double)(sz - Sz * W + oz * W);
  const double f = (side ? mv.q : -mv.q) * ldexp(1.0, g.near_ks);  // lattice units
  long long* dst = d.nearfx + ((int64_t)Tx + (int64_t)nL * (Ty + (int64_t)nL * Tz)) * g.cap;
  const int W3 = W * W * W;
  for (int l = threadIdx.x; l < W3; l += blockDim.x) {
    const int x = l % W, y = (l / W) % W, z = l / (W * W);
    const double dx = x - rx, dy = y - ry, dz = z - rz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) continue;
    atomicAdd((unsigned long long*)(dst + l), (unsigned long long)__double2ll_rn(f / sqrt(r2)));
  }
}

__global__ void __launch_bounds__(128) k_near_update(const Geo g, const Dev d) { near_update_blk(g, d, 0); }

__global__ void __launch_bounds__(128) k_near_update_batch(const BatchRep* reps, const int* off, int R) {
  const int r = batch_find(off, R, blockIdx.x);
  near_update_blk(reps[r].g, reps[r].d, off[r]);
}

void kmc_accept_apply(const Geo& g, const Dev& d, cudaStream_t s) {
  const AccPlan ap = acc_plan(g);
  k_acc_fused<<<acc_blocks(ap), ACC_THREADS, 0, s>>>(g, d, d.acc_scratch, ap);
  k_acc_coarse_reduce<<<KMC_COARSE_CELLS, 32 * ACR_WARPS, sizeof(double2) * ACR_WARPS * g.P, s>>>(g, d, d.acc_scratch);
  if (g.near_cache) k_near_update<<<2 * 27, 128, 0, s>>>(g, d);
}

// ------------------------------------------------------------------ batched step
// One KMC step of every member of a batch, each launch covering all members
// (propose over all members' leaves, rates over all members' charges, one
// selection CTA per member, the members' move records, then the accept
// updates of all members).  The members share precision, hop set and
// near-field mode; their sizes, levels and orders may differ.
int kmc_propose_chunk_min(const Geo& g) { return propose_chunk(g); }
size_t kmc_propose_smem_for(const Geo& g, int prec, int chunk, int cached) {
  return propose_smem(g, prec, cached ? 0 : chunk);
}
int kmc_acc_blocks_for(const Geo& g) { return acc_blocks(acc_plan(g)); }
int kmc_acr_blocks() { return KMC_COARSE_CELLS; }
size_t kmc_acr_smem_for(const Geo& g) { return sizeof(double2) * ACR_WARPS * g.P; }

// the propose launches of a batch step (one per class of pass capacity)
template <typename T, int NH>
static void propose_batch_t(const BatchPlan& bp, cudaStream_t s) {
  for (int c = 0; c < bp.nprop; c++) {
    if (bp.nblk_prop[c] <= 0) continue;
    if (bp.near_cache)
      k_propose_batch<T, NH, PROP_CACHED><<<bp.nblk_prop[c], PROP_THREADS, bp.smem_prop[c], s>>>(bp.reps, bp.off_prop[c],
                                                                                                 bp.R, 0);
    else
      k_propose_batch<T, NH, PROP_SUM><<<bp.nblk_prop[c], PROP_THREADS, bp.smem_prop[c], s>>>(bp.reps, bp.off_prop[c],
                                                                                              bp.R, bp.chunk_c[c]);
  }
}

void kmc_propose_batch(const BatchPlan& bp, cudaStream_t s) {
  if (bp.nhop == KMC_MAXHOP) {
    if (bp.prec == 0) propose_batch_t<double, KMC_MAXHOP>(bp, s);
    else propose_batch_t<float, KMC_MAXHOP>(bp, s);
  } else {
    if (bp.prec == 0) propose_batch_t<double, KMC_NHOP>(bp, s);
    else propose_batch_t<float, KMC_NHOP>(bp, s);
  }
}

template <typename T, int NH>
static void step_batch_t(const BatchPlan& bp, cudaStream_t s) {
  constexpr bool MIXED = sizeof(T) == 4;
  propose_batch_t<T, NH>(bp, s);
  k_finalize_batch<MIXED, NH><<<bp.nblk_fin, FIN_THREADS, 0, s>>>(bp.reps, bp.off_fin, bp.R);
  k_select_batch<<<bp.R, SEL_THREADS, 0, s>>>(bp.reps);
  k_record_move_batch<<<(bp.R + 127) / 128, 128, 0, s>>>(bp.reps, bp.R);
  k_acc_fused_batch<<<bp.nblk_acc, ACC_THREADS, 0, s>>>(bp.reps, bp.off_acc, bp.R);
  k_acc_coarse_reduce_batch<<<bp.nblk_acr, 32 * ACR_WARPS, bp.smem_acr, s>>>(bp.reps, bp.off_acr, bp.R);
  if (bp.near_cache && bp.nblk_nu > 0) k_near_update_batch<<<bp.nblk_nu, 128, 0, s>>>(bp.reps, bp.off_nu, bp.R);
}

void kmc_step_batch(const BatchPlan& bp, cudaStream_t s) {
  if (bp.nhop == KMC_MAXHOP) {
    if (bp.prec == 0) step_batch_t<double, KMC_MAXHOP>(bp, s);
    else step_batch_t<float, KMC_MAXHOP>(bp, s);
  } else {
    if (bp.prec == 0) step_batch_t<double, KMC_NHOP>(bp, s);
    else step_batch_t<float, KMC_NHOP>(bp, s);
  }
}

template <typename T, int NH>
static void prepare_batch_t(const BatchPlan& bp) {
  constexpr bool MIXED = sizeof(T) == 4;
  cudaFuncAttributes fa;
  for (int c = 0; c < bp.nprop; c++) {
    if (bp.near_cache) raise_dynamic_smem((const void*)k_propose_batch<T, NH, PROP_CACHED>, bp.smem_prop[c]);
    else raise_dynamic_smem((const void*)k_propose_batch<T, NH, PROP_SUM>, bp.smem_prop[c]);
  }
  cudaFuncGetAttributes(&fa, k_finalize_batch<MIXED, NH>);
  cudaFuncGetAttributes(&fa, k_select_batch);
  cudaFuncGetAttributes(&fa, k_record_move_batch);
  cudaFuncGetAttributes(&fa, k_acc_fused_batch);
  raise_dynamic_smem((const void*)k_acc_coarse_reduce_batch, bp.smem_acr);
  cudaFuncGetAttributes(&fa, k_near_update_batch);
}

void kmc_batch_prepare(const BatchPlan& bp) {
  if (bp.nhop == KMC_MAXHOP) {
    if (bp.prec == 0) prepare_batch_t<double, KMC_MAXHOP>(bp);
    else prepare_batch_t<float, KMC_MAXHOP>(bp);
  } else {
    if (bp.prec == 0) prepare_batch_t<double, KMC_NHOP>(bp);
    else prepare_batch_t<float, KMC_NHOP>(bp);
  }
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
  int cx = cell_at(X, g.nL, g.inv_a), cy = cell_at(Y, g.nL, g.inv_a), cz = cell_at(Z, g.nL, g.inv_a);
  int64_t leaf = cx + (int64_t)g.nL * (cy + (int64_t)g.nL * cz);
  const V4* spos = (const V4*)((sizeof(T) == 4) ? (const void*)d.spos32 : (const void*)d.spos64);
  T x = (T)X, y = (T)Y, z = (T)Z;
  T s = 0;
  int sing = 0;
  for (int o = 0; o < 27; o++) {
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    int ux = cx + ox, uy = cy + oy, uz = cz + oz;
    if (g.bc && (ux < 0 || ux >= g.nL || uy < 0 || uy >= g.nL || uz < 0 || uz >= g.nL)) continue;  // free space
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
  double cself = dU[t];
  double v = q * (phi_new[t] - phi_old[t]) - g.dipc * q * (d.dip[0] * dx + d.dip[1] * dy + d.dip[2] * dz) -
             q * q * cself;
  double dmx = dx, dmy = dy, dmz = dz;
  if (!g.bc) {  // periodic: the minimum image
    dmx -= g.a * rint(dx / g.a);
    dmy -= g.a * rint(dy / g.a);
    dmz -= g.a * rint(dz / g.a);
  }
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

// FP32 -> FP64 copy (API outputs and energy of the mixed form; not per step)
__global__ void k_widen(const float* src, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

void kmc_widen(const float* src, double* dst, int64_t n, cudaStream_t s) {
  if (n > 0) k_widen<<<1024, 256, 0, s>>>(src, dst, n);
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
    double M2 = d.dip[0] * d.dip[0] + d.dip[1] * d.dip[1] + d.dip[2] * d.dip[2];
    d.U[0] = 0.5 * sh[0] - 0.5 * g.dipc * M2;
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
    if (g.bc) {  // free space: targets must lie in the box
      if (!(x >= 0.0 && x < g.a)) {
        atomicOr(&d.err[0], KMC_DERR_BADPOS);
        x = 0.0;
        mout[t] = 0;
      }
    } else {
      x -= g.a * floor(x / g.a);
      if (x >= g.a) x -= g.a;
    }
    double o = ok ? d.pos[3 * (int64_t)i + k] : 0.0;
    tout[3 * t + k] = x;
    old[3 * t + k] = o;
    double dd = x - o;
    dv[3 * t + k] = g.bc ? dd : dd - g.a * rint(dd / g.a);
  }
}

void kmc_stage_general(const Geo& g, const Dev& d, int64_t m, const int32_t* part, const double* tin,
                       const uint8_t* min_, double* tout, double* old, double* dv, uint8_t* mout, cudaStream_t s) {
  if (m <= 0) return;
  k_stage_general<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(g, d, m, part, tin, min_, tout, old, dv, mout);
}

// load every per-step kernel up front: with lazy module loading a first
// launch inside a stream capture would invalidate the capture
static void kmc_preload() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, k_propose_lattice<float, KMC_NHOP, PROP_SUM>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<double, KMC_NHOP, PROP_SUM>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<float, KMC_MAXHOP, PROP_SUM>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<double, KMC_MAXHOP, PROP_SUM>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<float, KMC_NHOP, PROP_CACHED>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<double, KMC_NHOP, PROP_CACHED>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<float, KMC_MAXHOP, PROP_CACHED>);
  cudaFuncGetAttributes(&fa, k_propose_lattice<double, KMC_MAXHOP, PROP_CACHED>);
  cudaFuncGetAttributes(&fa, k_near_update);
  cudaFuncGetAttributes(&fa, k_finalize<true, KMC_NHOP>);
  cudaFuncGetAttributes(&fa, k_finalize<false, KMC_NHOP>);
  cudaFuncGetAttributes(&fa, k_finalize<true, KMC_MAXHOP>);
  cudaFuncGetAttributes(&fa, k_finalize<false, KMC_MAXHOP>);
  cudaFuncGetAttributes(&fa, k_rate_bsum);
  cudaFuncGetAttributes(&fa, k_select);
  cudaFuncGetAttributes(&fa, k_record);
  cudaFuncGetAttributes(&fa, k_move_from_event);
  cudaFuncGetAttributes(&fa, k_acc_fused);
  cudaFuncGetAttributes(&fa, k_mirror_move);
  cudaFuncGetAttributes(&fa, k_acc_coarse_reduce);
}
