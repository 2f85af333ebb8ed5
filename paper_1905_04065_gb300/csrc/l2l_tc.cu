// Per-step downward pass of the mixed form's finest level (when it has at
// least 4096 parents) on the fifth-generation tensor cores: the L2L
// translation of every parent's accumulated local expansion to its 8 children
// (the downward pass of Algorithm 2, translation by the child-offset regular
// harmonics).
//
// For one child position o the translation is a fixed real linear map of the
// parent's stored coefficients (P complex values, m >= 0; the m < 0 terms
// enter through the conjugate symmetry L_n^{-m} = (-1)^m conj(L_n^m)) to the
// child's: y = T_o x, T_o a real 2P x 2P matrix built once per level from the
// FP64 child tables.  So a level's pass is, per child position, one dense
// product Y_o = X T_o^T over all parents X (rows: parents, columns: the 2P
// real coefficients interleaved as stored).  It runs as tcgen05 kind::tf32
// MMAs, M = 128 parents, N = 16 ceil(2P / 16) outputs, K = 8 per MMA, FP32
// accumulation in tensor memory, with the FP32 operands split as
// x = hi + lo + r (hi = x rounded to the nearest TF32 value, lo = x - hi
// rounded to the nearest TF32 value, |r| <= 2^-22 |x|) and the products
// hi hi + hi lo + lo hi (the 3xTF32 scheme; the dropped lo lo and the
// residuals r leave about 3 2^-22 relative error per product).
//
// One CTA per (tile of 128 parents, child position): thread 0 issues the TMA
// loads of one K chunk of 32 values (hi and lo of the parents' tile, written
// by the level above's per-parent kernel with its outputs, and of T_o, each
// one contiguous block already in the 128-byte swizzle: 512-byte rows for the
// TMA), thread 32 issues the twelve MMAs of the chunk, and
// all four warps read the accumulator out (tcgen05.ld), add the child's own
// interaction-list expansion and write its accumulated expansion.  Every wait
// is bounded (KMC_WAIT_NS); on a timeout the CTA flags KMC_DERR_TIMEOUT, drains
// and frees its TMEM.
#include "common.cuh"
#include "kmcfmm.h"
#include "tc.cuh"

#include <stdlib.h>
#include <string.h>

#define LT_M 128          // parents per tile (MMA M)
#define LT_KC 32          // K values per chunk: one 128-byte swizzled row of FP32
#define LT_THREADS 128
#define LT_TMEM_COLS 256
#define LT_ATILE (LT_M * 128)  // one plane of the parents' tile per chunk

static int lt_K(const Geo& g) { return l2l_K(g.P); }
static int lt_nc8(const Geo& g) {
  const int c = (2 * g.P + 15) / 16;
  return c <= 6 ? 6 : c <= 9 ? 9 : c <= 12 ? 12 : c <= 15 ? 15 : 0;
}
static int64_t lt_npad(const Geo& g, int l) { return (void)g, l2l_npad(l); }  // parents of level l, whole tiles
// first level on the tensor cores, 0: none.  Only the finest level with at least 4096
// parents (256 CTAs of 128 parents x 8 children, two per SM): a level with fewer parents
// has too few CTAs to hide the per-CTA chain of K chunks, and runs faster on the CUDA cores.
int fmm_l2l_tc_first(const Geo& g) {
  if (g.prec != 1 || g.l2l != KMC_L2L_TENSOR || lt_nc8(g) == 0 || g.L < KMC_DOWN_COARSE + 1) return 0;
  if (((int64_t)1 << (3 * (g.L - 2))) < 4096 || tc_encode() == nullptr) return 0;
  return g.L;
}
size_t fmm_l2l_tc_table_floats(const Geo& g) { return (size_t)2 * 8 * 2 * (16 * lt_nc8(g)) * lt_K(g); }
size_t fmm_l2l_tc_split_floats(const Geo& g) { return (size_t)2 * lt_npad(g, g.L) * lt_K(g); }

// x = tf32(x) + r with |r| <= 2^-11 |x|, r exact in FP32
__device__ __forceinline__ float lt_tf32(float x) { return l2l_tf32(x); }

// degree and order of the stored coefficient c (c = n (n + 1) / 2 + m, 0 <= m <= n)
__device__ __forceinline__ void lt_nm(int c, int& n, int& m) {
  n = 0;
  while ((n + 1) * (n + 2) / 2 <= c) n++;
  m = c - n * (n + 1) / 2;
}

// T_o of level l into table slot ts: planes hi / lo of [N rows][K] (row = output real
// index 2 ci + (0 re, 1 im), column = input real index 2 cj + part), zero padding
__global__ void k_l2l_tables(const Geo g, const Dev d, int l, int ts, int N, int K, float* T) {
  const int o = blockIdx.y, row = blockIdx.x;
  const int ci = row >> 1, oc = row & 1;
  float* hi = T + ((size_t)(ts * 8 + o) * 2 + 0) * N * K;  // the table's blocks, one per K chunk
  float* lo = T + ((size_t)(ts * 8 + o) * 2 + 1) * N * K;
  const double2* Rt = d.Rch + ((int64_t)l * 8 + o) * g.P;
  int kk = 0, lo_m = 0;
  if (ci < g.P) lt_nm(ci, kk, lo_m);
  for (int col = threadIdx.x; col < K; col += blockDim.x) {
    const int cj = col >> 1, ic = col & 1;
    double v = 0.0;
    if (ci < g.P && cj < g.P) {
      int nn, mm;
      lt_nm(cj, nn, mm);
      const int j = nn - kk;
      if (j >= 0) {
        // y += L R (term m = +mm), y += (-1)^mm conj(L) R (term m = -mm, mm > 0), R = R_j^{m - lo}
        if (abs(mm - lo_m) <= j) {
          const double2 R = tab_get(Rt, j, mm - lo_m);
          v += oc == 0 ? (ic == 0 ? R.x : -R.y) : (ic == 0 ? R.y : R.x);
        }
        if (mm > 0 && abs(-mm - lo_m) <= j) {
          const double2 R = tab_get(Rt, j, -mm - lo_m);
          const double s = (mm & 1) ? -1.0 : 1.0;
          v += s * (oc == 0 ? (ic == 0 ? R.x : R.y) : (ic == 0 ? R.y : -R.x));
        }
      }
    }
    const float f = (float)v, h = lt_tf32(f);
    const int64_t at = l2l_sw_off(row, col, N, K / LT_KC);
    hi[at] = h;
    lo[at] = lt_tf32(f - h);
  }
}

// the parents' accumulated expansions of level l - 1, split into planes hi / lo of [npad][K]
__global__ void k_l2l_split(const Geo g, const Dev d, int l, int64_t npad, int K, float* A) {
  const int64_t np = (int64_t)1 << (3 * (l - 2));
  const int n2 = 2 * g.P;
  const float* Pe = (const float*)d.Peff + g.cell_off[l - 1] * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad * K; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t par = e / K;
    const int k = (int)(e % K);
    const float x = (par < np && k < n2) ? Pe[par * n2 + k] : 0.f;
    const float h = lt_tf32(x);
    const int64_t at = l2l_sw_off(par, k, LT_M, K / LT_KC);
    A[at] = h;
    A[npad * K + at] = lt_tf32(x - h);
  }
}

template <int NC8>
__global__ void __launch_bounds__(LT_THREADS, 2)
    k_l2l_tc(const Geo g, const Dev d, int l, int ts, int npad, const __grid_constant__ CUtensorMap amap,
             const __grid_constant__ CUtensorMap bmap) {
  constexpr int N = 16 * NC8;
  constexpr uint32_t IDESC = tc_idesc_tf32(LT_M, N);
  constexpr int BTILE = N * 128;
  extern __shared__ __align__(1024) unsigned char lt_sm[];
  __shared__ uint64_t full, empty, accf, fin_bar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_abort, s_used;
  volatile int* abortv = &s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x, o = blockIdx.y;
  const int K = LT_KC * ((2 * g.P + LT_KC - 1) / LT_KC), nkc = K / LT_KC;
  if (tid == 0) {
    mbar_init(&full, 1);
    mbar_init(&empty, 1);
    mbar_init(&accf, 1);
    mbar_init(&fin_bar, 1);
    s_abort = 0;
    s_used = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)),
                 "n"(LT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_taddr;
  const uint32_t sm0 = (smem_addr(lt_sm) + 1023u) & ~1023u;
  const uint32_t sAh = sm0, sAl = sm0 + LT_ATILE, sBh = sm0 + 2 * LT_ATILE, sBl = sBh + BTILE;
  int loaded = 0, used = 0;
  (void)used;
  // the loading and the issuing lane each run their loop while the rest of their warp waits at
  // __syncwarp, not in an mbarrier wait beside them
  if (tid == 0) {  // ---- loads: one K chunk at a time into the single stage
    for (int kc = 0; kc < nkc; kc++) {
      if (kc > 0 && !tc_wait(&empty, (uint32_t)((kc - 1) & 1), abortv)) break;
      mbar_expect_tx(&full, (uint32_t)(2 * LT_ATILE + 2 * BTILE));
      // one contiguous pre-swizzled block per operand plane (rows of 128 values in the maps)
      const int ya = (tile * nkc + kc) * (LT_M * LT_KC / 128), yl = npad * K / 128;
      const int yb = ((ts * 8 + o) * 2 * N * K + kc * N * LT_KC) / 128, ybl = N * K / 128;
      tma_load_2d(sAh, &amap, 0, ya, &full);
      tma_load_2d(sAl, &amap, 0, yl + ya, &full);
      tma_load_2d(sBh, &bmap, 0, yb, &full);
      tma_load_2d(sBl, &bmap, 0, yb + ybl, &full);
      loaded = kc + 1;
    }
  } else if (tid == 32) {  // ---- MMAs: hi hi + hi lo + lo hi per chunk
    for (int kc = 0; kc < nkc; kc++) {
      if (!tc_wait(&full, (uint32_t)(kc & 1), abortv)) break;
      tc_fence_after();
#pragma unroll
      for (int pr = 0; pr < 3; pr++) {
        const uint32_t a = pr == 2 ? sAl : sAh, b = pr == 1 ? sBl : sBh;
#pragma unroll
        for (int k8 = 0; k8 < 4; k8++)
          tc_mma_tf32(tbase, tc_sdesc_sw128(a + 32 * k8), tc_sdesc_sw128(b + 32 * k8), IDESC,
                      (kc == 0 && pr == 0 && k8 == 0) ? 0u : 1u);
      }
      tc_commit(&empty);
      used = kc + 1;
    }
    if (used == nkc) tc_commit(&accf);
    s_used = used;
  }
  if (warp < 2) __syncwarp();
  // ---- every warp: its 32 parents' rows of the accumulator, through shared memory (the stage is
  // free once the last MMA has completed) so that the children's rows are read and written by
  // whole warps, plus the children's own expansions
  bool ok = tc_wait(&accf, 0, abortv);
  ok = __all_sync(0xffffffffu, ok);
  ok = __syncthreads_and(ok);
  if (ok) {
    tc_fence_after();
    constexpr int NHALF = N / 2, LD = NHALF + 1;  // columns per pass; padded row stride (floats)
    static_assert(NHALF % 8 == 0, "whole x8 groups per pass");
    float* T = (float*)(lt_sm + (sm0 - smem_addr(lt_sm)));  // 128 x LD floats <= the stage
    const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16);
    const int r = 32 * warp + lane;
    const int64_t np = (int64_t)1 << (3 * (l - 2));
    const int nl = 1 << (l - 1), sh = l - 2, npl = nl >> 1, n2 = 2 * g.P;
    for (int hf = 0; hf < 2; hf++) {
#pragma unroll
      for (int gq = 0; gq < NHALF / 8; gq++) {
        uint32_t v[8];
        tc_ld8(ta + hf * NHALF + 8 * gq, v);
        tc_wait_ld(v);
#pragma unroll
        for (int q = 0; q < 8; q++) T[r * LD + 8 * gq + q] = __uint_as_float(v[q]);
      }
      __syncthreads();
      // a warp per row, four rows at a time: their own coefficients all in flight before the stores
      constexpr int NCI = (NHALF + 31) / 32;
      for (int r0 = 4 * warp; r0 < LT_M; r0 += 4 * (LT_THREADS / 32)) {
        int64_t cb[4];
        float w[4][NCI];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int64_t par = (int64_t)tile * LT_M + r0 + u;
          cb[u] = -1;
          if (par < np) {
            const int px = (int)(par & (npl - 1)), py = (int)((par >> sh) & (npl - 1)), pz = (int)(par >> (2 * sh));
            const int64_t child = (2 * px + (o & 1)) +
                                  (int64_t)nl * ((2 * py + ((o >> 1) & 1)) + (int64_t)nl * (2 * pz + (o >> 2)));
            cb[u] = (g.cell_off[l] + child) * n2;
          }
#pragma unroll
          for (int j = 0; j < NCI; j++) {
            const int col = hf * NHALF + lane + 32 * j;
            w[u][j] = (cb[u] >= 0 && lane + 32 * j < NHALF && col < n2) ? __ldg((const float*)d.Psi32 + cb[u] + col) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (cb[u] < 0) continue;
#pragma unroll
          for (int j = 0; j < NCI; j++) {
            const int c = lane + 32 * j, col = hf * NHALF + c;
            if (c < NHALF && col < n2) ((float*)d.Peff)[cb[u] + col] = T[(r0 + u) * LD + c] + w[u][j];
          }
        }
      }
      __syncthreads();
    }
  } else if (lane == 0) {
    *abortv = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0)  // drain: a load issued after the MMA side gave up
    for (int j = s_used; j < loaded; j++) (void)mbar_wait_bounded(&full, (uint32_t)(j & 1), KMC_WAIT_NS);
  if (tid == 32) {
    tc_commit(&fin_bar);
    if (!mbar_wait_bounded(&fin_bar, 0, KMC_WAIT_NS)) *abortv = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *abortv) atomicOr(&d.err[0], KMC_DERR_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(LT_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ host side
template <int NC8>
static cudaError_t lt_launch(dim3 grid, size_t dyn, cudaStream_t s, const Geo& g, const Dev& d, int l, int ts, int npad,
                             const CUtensorMap& amap, const CUtensorMap& bmap) {
  cudaError_t e = cudaFuncSetAttribute(k_l2l_tc<NC8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  k_l2l_tc<NC8><<<grid, LT_THREADS, dyn, s>>>(g, d, l, ts, npad, amap, bmap);
  return cudaGetLastError();
}

// rows x cols FP32 values, boxes of box_rows x box_cols; swizzled: the TMA writes the 128-byte swizzle
static bool lt_map(CUtensorMap* map, float* base, int cols, int64_t rows, int box_cols, int box_rows, bool swizzled) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return tc_encode()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzled ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void fmm_l2l_tc_tables(const Geo& g, const Dev& d, cudaStream_t s) {
  const int first = fmm_l2l_tc_first(g);
  if (!first || !d.l2lT) return;
  const int N = 16 * lt_nc8(g), K = lt_K(g);
  for (int l = first; l <= g.L; l++) k_l2l_tables<<<dim3((unsigned)N, 8), 128, 0, s>>>(g, d, l, l - first, N, K, d.l2lT);
}

bool fmm_l2l_tc(const Geo& g, const Dev& d, int l, cudaStream_t s) {
  const int first = fmm_l2l_tc_first(g);
  if (!first || l < first || l > g.L || !d.l2lT || !d.l2lA) return false;
  const int nc8 = lt_nc8(g), N = 16 * nc8, K = lt_K(g), ts = l - first;
  const int64_t npad = lt_npad(g, l);
  CUtensorMap amap, bmap;
  // the pre-swizzled blocks as rows of 128 values: a parents' block is 32 rows, a table block N / 4
  if (!lt_map(&amap, d.l2lA, 128, 2 * npad * K / 128, 128, LT_M * LT_KC / 128, false) ||
      !lt_map(&bmap, d.l2lT, 128, (int64_t)2 * 8 * 2 * N * K / 128, 128, N * LT_KC / 128, false))
    return false;
  if (l - 1 <= KMC_DOWN_COARSE) {  // the parents' level ran in the coarse launch: split them here
    const int64_t nb = (npad * K + 255) / 256;
    k_l2l_split<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, s>>>(g, d, l, npad, K, d.l2lA);
  }  // else the per-parent kernel of level l - 1 wrote the split with its outputs
  const size_t dyn = 2 * (size_t)LT_ATILE + 2 * (size_t)N * 128 + 1024;
  const dim3 grid((unsigned)(npad / LT_M), 8);
  cudaError_t e;
  switch (nc8) {
    case 6: e = lt_launch<6>(grid, dyn, s, g, d, l, ts, (int)npad, amap, bmap); break;
    case 9: e = lt_launch<9>(grid, dyn, s, g, d, l, ts, (int)npad, amap, bmap); break;
    case 12: e = lt_launch<12>(grid, dyn, s, g, d, l, ts, (int)npad, amap, bmap); break;
    default: e = lt_launch<15>(grid, dyn, s, g, d, l, ts, (int)npad, amap, bmap); break;
  }
  return e == cudaSuccess;
}

// ------------------------------------------------------------------ self-check of the tf32 path
// Four kind::tf32 MMAs (M = 128, N = 192, K = 4 x 8) of small integers (exact in
// TF32), both operands staged as k_l2l_tc stages them (2D TMA boxes of 32 FP32
// values per row, 128-byte swizzle), read back from TMEM.
#define LT_PROBE_N 192
#define LT_PROBE_SMEM (160 * 1024)
#define LT_PROBE_BOFF (64 * 1024)

__global__ void __launch_bounds__(128, 1)
    k_tc_probe_tf32(float* __restrict__ out, int* flag, const __grid_constant__ CUtensorMap amap,
                    const __grid_constant__ CUtensorMap bmap) {
  extern __shared__ __align__(1024) unsigned char pr_sm[];
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t s_taddr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)), "n"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_taddr, sm0 = (smem_addr(pr_sm) + 1023u) & ~1023u;
  bool bad = false;
  if (tid == 0) {
    mbar_expect_tx(&bar_tma, (LT_M + LT_PROBE_N) * 128);
    tma_load_2d(sm0, &amap, 0, 0, &bar_tma);
    tma_load_2d(sm0 + LT_PROBE_BOFF, &bmap, 0, 0, &bar_tma);
    if (!mbar_wait_bounded(&bar_tma, 0, KMC_WAIT_NS)) bad = true;
  }
  bad = __syncthreads_or(bad);
  if (!bad && tid == 0) {
    tc_fence_after();
    for (int k8 = 0; k8 < 4; k8++)
      tc_mma_tf32(tbase, tc_sdesc_sw128(sm0 + 32 * k8), tc_sdesc_sw128(sm0 + LT_PROBE_BOFF + 32 * k8),
                  tc_idesc_tf32(LT_M, LT_PROBE_N), k8 ? 1u : 0u);
    tc_commit(&bar_mma);
  }
  bool ok = !bad && mbar_wait_bounded(&bar_mma, 0, KMC_WAIT_NS);
  ok = __all_sync(0xffffffffu, ok);
  if (ok) {
    tc_fence_after();
    const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16);
    const int row = 32 * warp + lane;
    for (int c = 0; c < LT_PROBE_N / 8; c++) {
      uint32_t r[8];
      tc_ld8(ta + 8 * c, r);
      tc_wait_ld(r);
      for (int j = 0; j < 8; j++) out[row * LT_PROBE_N + 8 * c + j] = __uint_as_float(r[j]);
    }
  } else {
    atomicOr(flag, KMC_DERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && bad) tc_commit(&bar_mma);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(256) : "memory");
}

static int lt_probe_a(int r, int k) { return (r * 5 + k * 7) % 23 - 11; }
static int lt_probe_b(int n, int k) { return (n * 3 + k * 13) % 19 - 9; }

// 0 agreement, 1 mismatch, negative: unavailable or timed out; out: NULL or 128 x 192 floats
int tc_probe_tf32(float* out) {
  if (!tc_encode()) return -KMC_ERR_CUDA;
  static float hA[LT_M * 32], hB[LT_PROBE_N * 32];
  for (int r = 0; r < LT_M; r++)
    for (int k = 0; k < 32; k++) hA[r * 32 + k] = (float)lt_probe_a(r, k);
  for (int n = 0; n < LT_PROBE_N; n++)
    for (int k = 0; k < 32; k++) hB[n * 32 + k] = (float)lt_probe_b(n, k);
  float *dA = nullptr, *dB = nullptr, *dO = nullptr;
  int* dF = nullptr;
  int rc = -KMC_ERR_CUDA, hF = 0;
  const size_t nout = (size_t)LT_M * LT_PROBE_N;
  float* hO = (float*)malloc(nout * sizeof(float));
  CUtensorMap am, bm;
  if (!hO) return -KMC_ERR_OOM;
  if (cudaMalloc(&dA, sizeof hA) != cudaSuccess || cudaMalloc(&dB, sizeof hB) != cudaSuccess ||
      cudaMalloc(&dO, nout * sizeof(float)) != cudaSuccess || cudaMalloc(&dF, sizeof(int)) != cudaSuccess)
    goto done;
  if (cudaMemcpy(dA, hA, sizeof hA, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, hB, sizeof hB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dO, 0xff, nout * sizeof(float)) != cudaSuccess || cudaMemset(dF, 0, sizeof(int)) != cudaSuccess)
    goto done;
  if (!lt_map(&am, dA, 32, LT_M, 32, LT_M, true) || !lt_map(&bm, dB, 32, LT_PROBE_N, 32, LT_PROBE_N, true)) goto done;
  if (cudaFuncSetAttribute(k_tc_probe_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, LT_PROBE_SMEM) != cudaSuccess)
    goto done;
  k_tc_probe_tf32<<<1, 128, LT_PROBE_SMEM>>>(dO, dF, am, bm);
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  if (cudaMemcpy(hO, dO, nout * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&hF, dF, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    goto done;
  if (out) memcpy(out, hO, nout * sizeof(float));
  rc = hF ? -KMC_ERR_TIMEOUT : 0;
  for (int r = 0; r < LT_M && rc == 0; r++)
    for (int n = 0; n < LT_PROBE_N; n++) {
      int want = 0;
      for (int k = 0; k < 32; k++) want += lt_probe_a(r, k) * lt_probe_b(n, k);
      if (hO[(size_t)r * LT_PROBE_N + n] != (float)want) {
        rc = 1;
        break;
      }
    }
done:
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dO);
  cudaFree(dF);
  free(hO);
  return rc;
}
