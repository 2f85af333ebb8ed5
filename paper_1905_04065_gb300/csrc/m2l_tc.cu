// M2L of Algorithm 2 on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators, TMA operand staging).
//
// The arithmetic is the exact integer slicing of the FP64 operands described
// beside the slicing kernels (fmm_kernels.cu): every operand is cut into
// 7-bit integer slices held exactly in bf16, the slice products of one
// diagonal D (slice pairs (a, D - 2 - a)) are summed by the tensor core in
// FP32, which is exact on these integers while a sum stays below 2^24, the
// sums are converted to int32 per diagonal, and the diagonals are combined in
// FP64 with their power-of-two weights.  Every partial sum is an exact
// integer, so this kernel gives bit for bit the result of the mma.sync form.
//
// Mapping.  Out[b][i] = sum over far translations v of the parity class,
// sum_kk Mslice[src(b, v)][kk] * Rslice_v[i][kk]:
//   * MMA M = 128 target cells of one parity class (TMEM lane = cell row);
//   * MMA N = NN = 16 * NC8 >= 2P output coefficients (TMEM column = i);
//   * K = the 2P real input coefficients, in chunks of 64 (four MMAs of 16).
// Both operands sit in shared memory in the 128-byte-swizzled K-major layout
// (a row's 64 values in 128 bytes, its eight 16-byte pieces permuted by the
// row index mod 8, atoms of 8 rows x 128 bytes), which the tensor core reads a
// full bank width at a time, and both arrive by TMA: the target tile is a box
// of bx x by x bz <= 8 x 4 x 4 cells of one parity class, and the cells'
// slices sit in a ghost-padded per-class layout (k_oz_bslice_tc), so the
// source cells of the tile under one translation are one 5D box (the TMA
// applies the swizzle); the slicing kernel writes every (translation, slice,
// K chunk) of the R slices as one contiguous block already in the swizzled
// order, fetched as one 2D box of NN / 4 rows of 512 bytes.
//
// Exactness bound.  Per output entry and translation a diagonal sums at most
// K = 2P <= 240 terms, each at most 2*128*64 + (S - 2)*64*64 <= 32768 in
// magnitude (S = 6), i.e. < 7.9e6; two translations (TC_TP) stay below 2^24,
// so the FP32 accumulator in TMEM holds two translations' sums exactly before
// they are read out (tcgen05.ld), rounded to int32 (exact) and added into
// per-thread int32 registers (189 translations stay below 2^31).
//
// Work and roles.  A work item is (diagonal D, parity class, tile, split of
// the interaction list); persistent CTAs, one per SM, take items largest
// diagonal first.  Per item and far translation the ns = D - 1 slice pairs
// (a, D - 2 - a) and the K chunks of 64 are stages of one A tile and one B
// tile (four MMAs of K = 16 each).  Warp 0 lane 0 issues the TMA loads into
// NST rotating stages, warp 1 lane 0 issues the MMAs and commits each stage
// back to the loader, warps 2..13 read the accumulators out (two TMEM
// accumulators alternate between translation pairs, so the readout of one
// pair overlaps the MMAs of the next) and add every item's exact integer sums
// into acc64[D - 2][cell][i]; k_oz_finish combines the diagonals in FP64 in a
// fixed order, bit for bit as the mma.sync form does.  Only mbarriers order
// the roles; the CTA-wide barrier comes only before and after the loop.
//
// Every wait is bounded (KMC_WAIT_NS): on a timeout the CTA flags
// KMC_DERR_TIMEOUT, drains its own copies and MMAs (bounded again), frees its
// TMEM and returns.
#include "common.cuh"
#include "kmcfmm.h"
#include "tc.cuh"

#include <stdlib.h>
#include <string.h>

#define TC_M 128
#define TC_EPI_WARPS 12  // readout warps: 4 TMEM lane quarters x 3 column thirds
#define TC_THREADS (64 + 32 * TC_EPI_WARPS)  // load warp, MMA warp, readout warps
#define TC_TP 2             // translations per TMEM accumulation
#define TC_BUF_COL 256      // TMEM column of the second accumulator
#define TC_TMEM_COLS 512
#define TC_MAX_NC8 15       // NN <= 240: p <= 14
#define TC_MIN_SMEM (120 * 1024)  // one CTA per SM (its TMEM allocation is the whole SM's)
#define TC_ATILE (TC_M * 128)     // A tile: 128 rows x 64 values


// Geometry of one level's launch: target tiles are boxes of bx x by x bz
// cells of a parity class (at most 8 x 4 x 4 = 128, the MMA's M); the cells'
// slices sit in a ghost-padded per-class layout, so the source cells of a
// tile under one translation form one box of that layout (one TMA load).
struct TcLevel {
  int l, nl, h2;        // level, cells per side, class cells per side
  int bx, by, bz;       // tile box
  int tx_n, ty_n, tz_n; // tiles per class side
  int ntile, nsplit;    // tiles per class, interaction-list splits
  int S, nkc, nitem;    // slices, K chunks of 64, work items
};

// Work item w (largest diagonals first): diagonal D, parity class, tile, split.
struct TcItem {
  int D, cls, tile, split;
};
__device__ __forceinline__ TcItem tc_item(const TcLevel& L, int w) {
  TcItem it;
  it.split = w % L.nsplit;
  w /= L.nsplit;
  it.tile = w % L.ntile;
  w /= L.ntile;
  it.cls = w & 7;
  it.D = L.S + 1 - (w >> 3);
  return it;
}
// far translation q of the item's interaction-list range (q counts all 216 entries); false if near
__device__ __forceinline__ bool tc_trans(int cls, int qo, int& tx, int& ty, int& tz) {
  const int ox = cls & 1, oy = (cls >> 1) & 1, oz = cls >> 2;
  const int c8 = qo & 7, dl = qo >> 3;
  tx = 2 * (dl % 3 - 1) + (c8 & 1) - ox;
  ty = 2 * ((dl / 3) % 3 - 1) + ((c8 >> 1) & 1) - oy;
  tz = 2 * (dl / 9 - 1) + (c8 >> 2) - oz;
  return !(abs(tx) <= 1 && abs(ty) <= 1 && abs(tz) <= 1);
}
__device__ __forceinline__ int tc_q0(const TcLevel& L, int split) { return 216 * split / L.nsplit; }
__device__ __forceinline__ int tc_nfar(const TcLevel& L, const TcItem& it) {
  int n = 0, tx, ty, tz;
  for (int q = tc_q0(L, it.split); q < tc_q0(L, it.split + 1); q++) n += tc_trans(it.cls, q, tx, ty, tz);
  return n;
}

// Persistent CTAs (one per SM) over the level's work items, warp-specialised:
// warp 0 lane 0 loads (two TMA boxes per stage), warp 1 lane 0 issues the
// MMAs, warps 2..13 read the accumulators out of TMEM and add every item's
// exact per-diagonal integer sums into acc64[D - 2][cell][i] (integer
// atomics: the result does not depend on their order; k_oz_finish combines
// the diagonals in FP64 in a fixed order).
template <int NC8>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(const TcLevel L, const Geo g, const Dev d, long long* __restrict__ acc64,
             const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap cmap, int nst) {
  constexpr int NN = 16 * NC8, NH = NN / 3, NG = NH / 8;  // MMA N; columns, x8 groups per readout thread
  static_assert(NC8 % 3 == 0, "column thirds of whole x8 groups");
  constexpr uint32_t IDESC = tc_idesc(TC_M, NN);
  constexpr int STAGE = TC_ATILE + NN * 128;  // one A tile and one B tile of 64 K values
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ uint64_t full[8], empty[8], accf[2], acce[2], fin_bar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_abort, s_consumed;
  volatile int* abortv = &s_abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n2 = 2 * g.P;
  const int64_t ncell = (int64_t)L.nl * L.nl * L.nl;
  const uint32_t arows = (uint32_t)(L.bx * L.by * L.bz);
  if (tid == 0) {
    for (int s = 0; s < nst; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], TC_EPI_WARPS);
    }
    mbar_init(&fin_bar, 1);
    s_abort = 0;
    s_consumed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)),
                 "n"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_taddr;
  const uint32_t sm0 = (smem_addr(tc_sm) + 1023u) & ~1023u;  // swizzle atoms are 1024-byte aligned
  int produced = 0;

  if (warp == 0 && lane == 0) {  // ---- loads
    int j = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < L.nitem && ok; w += gridDim.x) {
      const TcItem it = tc_item(L, w);
      const int ns = it.D - 1;
      const int x0 = (it.tile % L.tx_n) * L.bx, y0 = ((it.tile / L.tx_n) % L.ty_n) * L.by,
                z0 = (it.tile / (L.tx_n * L.ty_n)) * L.bz;
      const int ox = it.cls & 1, oy = (it.cls >> 1) & 1, oz = it.cls >> 2;
      for (int q = tc_q0(L, it.split); q < tc_q0(L, it.split + 1) && ok; q++) {
        int tx, ty, tz;
        if (!tc_trans(it.cls, q, tx, ty, tz)) continue;
        const int v = (tx + 3) + 7 * ((ty + 3) + 7 * (tz + 3));
        // source cell 2 j + o + t = 2 (j + floor((o + t) / 2)) + ((o + t) & 1)
        const int ux = ox + tx, uy = oy + ty, uz = oz + tz;
        const int scls = (ux & 1) | ((uy & 1) << 1) | ((uz & 1) << 2);
        const int cx = x0 + (ux >> 1) + 2, cy = y0 + (uy >> 1) + 2, cz = z0 + (uz >> 1) + 2;
        for (int a = 0; a < ns && ok; a++)
          for (int kc = 0; kc < L.nkc; kc++, j++) {
            const int s = j % nst;
            if (j >= nst && !tc_wait(&empty[s], (uint32_t)((j / nst - 1) & 1), abortv)) {
              ok = false;
              break;
            }
            const uint32_t st = sm0 + (uint32_t)(s * STAGE);
            mbar_expect_tx(&full[s], arows * 128u + (uint32_t)(NN * 128));
            tma_load_5d(st, &cmap, kc * 64, cx, cy, cz, a * 8 + scls, &full[s]);
            tma_load_2d(st + TC_ATILE, &amap, 0, ((v * OZ_S + (ns - 1 - a)) * L.nkc + kc) * (NN / 4), &full[s]);
          }
      }
    }
    produced = j;
  } else if (warp == 1 && lane == 0) {  // ---- MMAs
    int k = 0, gidx = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < L.nitem && ok; w += gridDim.x) {
      const TcItem it = tc_item(L, w);
      const int ns = it.D - 1, nt = tc_nfar(L, it);
      for (int t = 0; t < nt && ok; t++) {
        const bool gstart = t % TC_TP == 0, gend = t % TC_TP == TC_TP - 1 || t == nt - 1;
        const int buf = gidx & 1;
        if (gstart && gidx >= 2 && !tc_wait(&acce[buf], (uint32_t)(((gidx >> 1) - 1) & 1), abortv)) {
          ok = false;
          break;
        }
        const uint32_t dt = tbase + (uint32_t)(buf * TC_BUF_COL);
        for (int a = 0; a < ns && ok; a++)
          for (int kc = 0; kc < L.nkc; kc++, k++) {
            const int s = k % nst;
            if (!tc_wait(&full[s], (uint32_t)((k / nst) & 1), abortv)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = sm0 + (uint32_t)(s * STAGE);
#pragma unroll
            for (int k16 = 0; k16 < 4; k16++)
              tc_mma(dt, tc_sdesc_sw128(st + 32 * k16), tc_sdesc_sw128(st + TC_ATILE + 32 * k16), IDESC,
                     (gstart && a == 0 && kc == 0 && k16 == 0) ? 0u : 1u);
            tc_commit(&empty[s]);
          }
        if (ok && gend) {
          tc_commit(&accf[buf]);
          gidx++;
        }
      }
    }
    s_consumed = k;
  } else if (warp >= 2) {  // ---- accumulators out of TMEM
    const int ew = warp - 2, eq = warp & 3, eh = ew >> 2, row = 32 * eq + lane;
    const uint32_t ta0 = tbase + ((uint32_t)(32 * eq) << 16) + (uint32_t)(eh * NH);
    int iacc[NH];
#pragma unroll
    for (int j = 0; j < NH; j++) iacc[j] = 0;
    int gidx = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < L.nitem && ok; w += gridDim.x) {
      const TcItem it = tc_item(L, w);
      const int ngrp = (tc_nfar(L, it) + TC_TP - 1) / TC_TP;
      int b = -1;  // this thread's target cell
      if (row < (int)arows) {
        const int x = row % L.bx, y = (row / L.bx) % L.by, z = row / (L.bx * L.by);
        const int jx = (it.tile % L.tx_n) * L.bx + x, jy = ((it.tile / L.tx_n) % L.ty_n) * L.by + y,
                  jz = (it.tile / (L.tx_n * L.ty_n)) * L.bz + z;
        b = (2 * jx + (it.cls & 1)) + L.nl * ((2 * jy + ((it.cls >> 1) & 1)) + L.nl * (2 * jz + (it.cls >> 2)));
      }
      for (int gi = 0; gi < ngrp; gi++, gidx++) {
        const int buf = gidx & 1;
        bool wok = tc_wait(&accf[buf], (uint32_t)((gidx >> 1) & 1), abortv);
        wok = __all_sync(0xffffffffu, wok);  // tcgen05.ld is warp-collective
        if (!wok) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = ta0 + (uint32_t)(buf * TC_BUF_COL);
#pragma unroll
        for (int cc = 0; cc < NG; cc += 2) {
          uint32_t r0[8], r1[8];
          tc_ld8(ta + 8 * cc, r0);
          if (cc + 1 < NG) tc_ld8(ta + 8 * (cc + 1), r1);
          tc_wait_ld(r0);
          if (cc + 1 < NG) tc_wait_ld(r1);
#pragma unroll
          for (int j = 0; j < 8; j++) iacc[8 * cc + j] += __float2int_rn(__uint_as_float(r0[j]));
          if (cc + 1 < NG) {
#pragma unroll
            for (int j = 0; j < 8; j++) iacc[8 * (cc + 1) + j] += __float2int_rn(__uint_as_float(r1[j]));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&acce[buf]);
      }
      if (!ok) break;
      // the item's diagonal: exact integer sums, added in any order
      {
        unsigned long long* dst = (unsigned long long*)(acc64 + ((int64_t)(it.D - 2) * ncell + (b >= 0 ? b : 0)) * n2 + eh * NH);
        const int lim = b >= 0 ? n2 - eh * NH : 0;
#pragma unroll
        for (int j = 0; j < NH; j++) {
          if (j < lim) atomicAdd(dst + j, (unsigned long long)(long long)iacc[j]);
          iacc[j] = 0;
        }
      }
    }
  }

  // drain: loads in flight after a timeout, then every MMA, then free the TMEM
  __syncthreads();
  if (warp == 0 && lane == 0)
    for (int j = s_consumed; j < produced; j++) (void)mbar_wait_bounded(&full[j % nst], (uint32_t)((j / nst) & 1), KMC_WAIT_NS);
  if (warp == 1 && lane == 0) {
    tc_commit(&fin_bar);
    if (!mbar_wait_bounded(&fin_bar, 0, KMC_WAIT_NS)) *abortv = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *abortv) atomicOr(&d.err[0], KMC_DERR_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TC_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ host side
// x8 column groups per thread half: NN = 16 * nc8 >= 2P (0: p too large for one MMA N)
static int tc_nc8(const Geo& g) {
  const int c = (2 * g.P + 15) / 16;
  return c <= 6 ? 6 : c <= 9 ? 9 : c <= 12 ? 12 : c <= TC_MAX_NC8 ? TC_MAX_NC8 : 0;
}

int fmm_m2l_tc_rows(const Geo& g) { return 16 * tc_nc8(g); }
int fmm_m2l_tc_kchunks(const Geo& g) { return (2 * g.P + 63) / 64; }

bool fmm_m2l_tc_ok(const Geo& g) { return g.m2l == KMC_M2L_TENSOR && tc_nc8(g) > 0 && tc_encode() != nullptr; }

template <int NC8>
static cudaError_t tc_launch(int grid, size_t dyn, cudaStream_t s, const TcLevel& L, const Geo& g, const Dev& d,
                             long long* acc64, const CUtensorMap& amap, const CUtensorMap& cmap, int nst) {
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<NC8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  k_m2l_tc<NC8><<<grid, TC_THREADS, dyn, s>>>(L, g, d, acc64, amap, cmap, nst);
  return cudaGetLastError();
}

bool fmm_m2l_tc(const Geo& g, const Dev& d, int l, const unsigned short* As, const unsigned short* Bp,
                long long* acc64, cudaStream_t s) {
  const int nc8 = tc_nc8(g);
  const TcEncodeTiled enc = tc_encode();
  if (!nc8 || !enc || (((uintptr_t)As) & 15) || (((uintptr_t)Bp) & 15)) return false;
  const int n2 = 2 * g.P, nc = oz_cols(n2), NN = 16 * nc8;
  TcLevel L;
  L.l = l;
  L.nl = 1 << (l - 1);
  L.h2 = L.nl >> 1;
  L.bx = L.h2 < 8 ? L.h2 : 8;
  L.by = L.h2 < 4 ? L.h2 : 4;
  L.bz = L.by;
  L.tx_n = L.h2 / L.bx;
  L.ty_n = L.h2 / L.by;
  L.tz_n = L.h2 / L.bz;
  L.ntile = L.tx_n * L.ty_n * L.tz_n;
  L.S = oz_slices(g);
  L.nkc = fmm_m2l_tc_kchunks(g);
  {  // interaction-list splits where a level has few items: about two items per SM
    const int per = L.S * 8 * L.ntile, want = (2 * 152 + per - 1) / per;
    L.nsplit = want < 1 ? 1 : (want > 24 ? 24 : want);
  }
  L.nitem = L.S * 8 * L.ntile * L.nsplit;
  // the translations' slices (k_oz_aslice_tc layout) as rows of 256 values; the block of one
  // translation, slice and K chunk (NN rows x 64 values, swizzled) is NN / 4 consecutive rows
  CUtensorMap amap, cmap;
  {
    const cuuint64_t dims[2] = {256, (cuuint64_t)343 * OZ_S * L.nkc * NN / 4};
    const cuuint64_t strides[1] = {256 * sizeof(unsigned short)};
    const cuuint32_t box[2] = {256, (cuuint32_t)(NN / 4)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)As, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  // the cells' slices (k_oz_bslice_tc layout) as [8 S][Xp][Xp][Xp][nc]; a box is 64 values of
  // bx x by x bz cells, written by the TMA in the 128-byte swizzle the MMA reads
  {
    const cuuint64_t xp = (cuuint64_t)L.h2 + 4, rb = (cuuint64_t)nc * sizeof(unsigned short);
    const cuuint64_t dims[5] = {(cuuint64_t)nc, xp, xp, xp, (cuuint64_t)8 * OZ_S};
    const cuuint64_t strides[4] = {rb, rb * xp, rb * xp * xp, rb * xp * xp * xp};
    const cuuint32_t box[5] = {64, (cuuint32_t)L.bx, (cuuint32_t)L.by, (cuuint32_t)L.bz, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (enc(&cmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 5, (void*)Bp, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  const int stage = TC_ATILE + NN * 128;
  int nst = (215 * 1024) / stage;
  nst = nst < 2 ? 2 : (nst > 8 ? 8 : nst);
  size_t dyn = (size_t)nst * stage + 1024;  // + alignment of the swizzle atoms
  if (dyn < TC_MIN_SMEM) dyn = TC_MIN_SMEM;
  const int grid = L.nitem < 152 ? L.nitem : 152;
  cudaError_t e;
  switch (nc8) {
    case 6: e = tc_launch<6>(grid, dyn, s, L, g, d, acc64, amap, cmap, nst); break;
    case 9: e = tc_launch<9>(grid, dyn, s, L, g, d, acc64, amap, cmap, nst); break;
    case 12: e = tc_launch<12>(grid, dyn, s, L, g, d, acc64, amap, cmap, nst); break;
    default: e = tc_launch<TC_MAX_NC8>(grid, dyn, s, L, g, d, acc64, amap, cmap, nst); break;
  }
  return e == cudaSuccess;
}

// ------------------------------------------------------------------ self-check of the MMA path
// Four tcgen05 MMAs (M = 128, N = TC_PROBE_N, K = 4 x 16) of small integer
// operands staged exactly as k_m2l_tc stages them (A by cp.async pieces into
// the 128-byte-swizzled positions, B as one swizzled contiguous block by one
// 2D TMA box), read back from TMEM; the operands sit at the start of a large
// shared allocation, so every access stays inside it.
#define TC_PROBE_N 192
#define TC_PROBE_SMEM (160 * 1024)
#define TC_PROBE_BOFF (64 * 1024)

__global__ void __launch_bounds__(128, 1)
    k_tc_probe(const unsigned short* __restrict__ A, float* __restrict__ out, int* flag,
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
  for (int c = 0; c < 8; c++)  // row tid of A: 64 values in eight 16-byte pieces
    cp_async16_tc(sm0 + tc_sw128(tid, 8 * c), A + tid * 64 + 8 * c);
  if (tid == 0) {
    mbar_expect_tx(&bar_tma, TC_PROBE_N * 128);
    tma_load_2d(sm0 + TC_PROBE_BOFF, &bmap, 0, 0, &bar_tma);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0 && !mbar_wait_bounded(&bar_tma, 0, KMC_WAIT_NS)) bad = true;
  bad = __syncthreads_or(bad);
  if (!bad && tid == 0) {
    tc_fence_after();
    for (int k16 = 0; k16 < 4; k16++)
      tc_mma(tbase, tc_sdesc_sw128(sm0 + 32 * k16), tc_sdesc_sw128(sm0 + TC_PROBE_BOFF + 32 * k16),
             tc_idesc(TC_M, TC_PROBE_N), k16 ? 1u : 0u);
    tc_commit(&bar_mma);
  }
  bool ok = !bad && mbar_wait_bounded(&bar_mma, 0, KMC_WAIT_NS);
  ok = __all_sync(0xffffffffu, ok);
  if (ok) {
    tc_fence_after();
    const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16);
    const int row = 32 * warp + lane;
    for (int c = 0; c < TC_PROBE_N / 8; c++) {
      uint32_t r[8];
      tc_ld8(ta + 8 * c, r);
      tc_wait_ld(r);
      for (int j = 0; j < 8; j++) out[row * TC_PROBE_N + 8 * c + j] = __uint_as_float(r[j]);
    }
  } else {
    atomicOr(flag, KMC_DERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && bad) {  // drain whatever was issued (bounded)
    (void)mbar_wait_bounded(&bar_tma, 0, KMC_WAIT_NS);
    tc_commit(&bar_mma);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(256) : "memory");
}

// small integer operands; bf16 holds them exactly (bits = the float's upper half)
static unsigned short tc_bf16_int(int v) {
  const float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  return (unsigned short)(u >> 16);
}
static int tc_probe_a(int r, int k) { return (r * 7 + k * 3) % 17 - 8; }
static int tc_probe_b(int n, int k) { return (n * 5 + k * 11) % 13 - 6; }

int kmc_check_tensor_mma(int device, int kind, float* out) {
  if (cudaSetDevice(device) != cudaSuccess) return -KMC_ERR_CUDA;
  if (kind == 1) return tc_probe_tf32(out);
  if (kind != 0) return -KMC_ERR_ARG;
  const TcEncodeTiled enc = tc_encode();
  if (!enc) return -KMC_ERR_CUDA;
  static unsigned short hA[TC_M * 64], hB[TC_PROBE_N * 64];
  for (int r = 0; r < TC_M; r++)
    for (int k = 0; k < 64; k++) hA[r * 64 + k] = tc_bf16_int(tc_probe_a(r, k));
  for (int n = 0; n < TC_PROBE_N; n++)  // the block order of k_oz_aslice_tc: swizzled rows of 64 values
    for (int k = 0; k < 64; k++) hB[tc_sw128(n, k) / 2] = tc_bf16_int(tc_probe_b(n, k));
  unsigned short *dA = nullptr, *dB = nullptr;
  float* dO = nullptr;
  int* dF = nullptr;
  int rc = -KMC_ERR_CUDA;
  const size_t nout = (size_t)TC_M * TC_PROBE_N;
  float* hO = (float*)malloc(nout * sizeof(float));
  CUtensorMap map;
  const cuuint64_t dims[2] = {256, TC_PROBE_N / 4};
  const cuuint64_t strides[1] = {256 * sizeof(unsigned short)};
  const cuuint32_t box[2] = {256, TC_PROBE_N / 4};
  const cuuint32_t estr[2] = {1, 1};
  int hF = 0;
  if (!hO) return -KMC_ERR_OOM;
  if (cudaMalloc(&dA, sizeof hA) != cudaSuccess || cudaMalloc(&dB, sizeof hB) != cudaSuccess ||
      cudaMalloc(&dO, nout * sizeof(float)) != cudaSuccess || cudaMalloc(&dF, sizeof(int)) != cudaSuccess)
    goto done;
  if (cudaMemcpy(dA, hA, sizeof hA, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, hB, sizeof hB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dO, 0xff, nout * sizeof(float)) != cudaSuccess || cudaMemset(dF, 0, sizeof(int)) != cudaSuccess)
    goto done;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)dB, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    goto done;
  if (cudaFuncSetAttribute(k_tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_PROBE_SMEM) != cudaSuccess)
    goto done;
  k_tc_probe<<<1, 128, TC_PROBE_SMEM>>>(dA, dO, dF, map);
  if (cudaDeviceSynchronize() != cudaSuccess) goto done;
  if (cudaMemcpy(hO, dO, nout * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&hF, dF, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    goto done;
  if (out) memcpy(out, hO, nout * sizeof(float));
  rc = hF ? -KMC_ERR_TIMEOUT : 0;
  for (int r = 0; r < TC_M && rc == 0; r++)
    for (int n = 0; n < TC_PROBE_N; n++) {
      int want = 0;
      for (int k = 0; k < 64; k++) want += tc_probe_a(r, k) * tc_probe_b(n, k);
      if (hO[(size_t)r * TC_PROBE_N + n] != (float)want) {
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
