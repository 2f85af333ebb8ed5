// common.cuh -- shared device types, state layout and solid-harmonic helpers.
//
// Solid harmonics (Eq. (multipole_local_expansion) up to normalisation, which
// the paper leaves open):
//   regular    R_n^m(x) = r^n P_n^m(cos t) e^{i m f} / (n+m)!
//   irregular  I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1}
// with the Condon-Shortley phase in P_n^m, and R_n^{-m} = (-1)^m conj(R_n^m),
// I_n^{-m} = (-1)^m conj(I_n^m).  They satisfy 1/|x-y| = sum conj(R(y)) I(x)
// for |y| < |x| and are generated by the Cartesian recurrences
//   R_m^m = -(x+iy)/(2m) R_{m-1}^{m-1},
//   (n^2-m^2) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m,
//   I_m^m = -(2m-1)(x+iy)/r^2 I_{m-1}^{m-1},
//   r^2 I_n^m = (2n-1) z I_{n-1}^m - ((n-1)^2-m^2) I_{n-2}^m.
// Expansion coefficients are stored for 0 <= m <= n <= p at tri(n,m).
//   multipole   Mt_n^m = sum q R_n^m(y - c)          phi(x) = Re sum conj(Mt) I(x - c)
//   local       L_n^m  = sum q conj(I_n^m(y - c))    phi(x) = Re sum L R(x - c)
// Translations (t = vector between centres):
//   M2M  Mt'(c2)_n^m = sum_{k,l} Mt_k^l(c1) R_{n-k}^{m-l}(c1 - c2)
//   M2L  L_n^m(c2)   = sum_{k,l} (-1)^k Mt_k^l(c1) conj(I_{n+k}^{m+l}(c1 - c2))
//   L2L  L'_k^l(c2)  = sum_{n,m} L_n^m(c1) R_{n-k}^{m-l}(c2 - c1)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define KMC_MAXL 10   // maximum number of levels
#ifndef KMC_MAXP
#define KMC_MAXP 24   // maximum expansion degree
#endif
#define KMC_NHOP 6    // lattice hop directions of the nearest-neighbour set (+x,-x,+y,-y,+z,-z)
#define KMC_ISQ_N (3 * 23 * 23 + 1)  // squared lattice distances within 27 leaves of <= 12 sites
#define KMC_MAXHOP 14 // with the 8 body diagonals (the hop set of the paper's Sec. 5.3 benchmark)

// component a (0 = x, 1 = y, 2 = z) of lattice hop k: k < 6 the faces
// (+x, -x, +y, -y, +z, -z), k = 6 + d the body diagonals with component a
// negative when bit a of d is set (x fastest: (+,+,+), (-,+,+), (+,-,+), ...)
__host__ __device__ __forceinline__ constexpr int hop_c(int k, int a) {
  return k < 6 ? ((k >> 1) == a ? ((k & 1) ? -1 : 1) : 0) : ((((k - 6) >> a) & 1) ? -1 : 1);
}
#define KMC_FIN_PARTICLES 128  // particles per block sum of the rates
#define KMC_DOWN_COARSE 4      // downward levels 2 .. 4 (fewer than 512 parents) share one launch
// R(c_b - c_a) for a cell b of level l <= KMC_DOWN_COARSE and its ancestor a of level la < l, one
// table per position of b inside a: 8^(l - la) tables for (l, la), in the order (2,1), (3,1),
// (3,2), (4,1), (4,2), (4,3): 8 + 64 + 8 + 512 + 64 + 8
#define KMC_COARSE_TABLES 664
__host__ __device__ __forceinline__ int coarse_table_base(int l, int la) {
  // first table of (l, la) in the order above
  return l == 2 ? 0 : l == 3 ? (la == 1 ? 8 : 72) : (la == 1 ? 80 : la == 2 ? 592 : 656);
}
// Periodic images nu with |nu|_inf <= KMC_TOP are handled by the tree (the
// level-2 interaction list covers the (2 KMC_TOP + 1)^3 block of domain copies);
// the rest are the far field V_inf of the lattice operator.
#ifndef KMC_TOP
#define KMC_TOP 2
#endif
#define KMC_TOP_SPAN (4 * KMC_TOP + 3)  // level-2 M2L offsets per axis: [-(2 KMC_TOP + 1), 2 KMC_TOP + 1]
#define KMC_TOP_NOFF (KMC_TOP_SPAN * KMC_TOP_SPAN * KMC_TOP_SPAN)
#define KMC_TOP_NIMG ((2 * KMC_TOP + 1) * (2 * KMC_TOP + 1) * (2 * KMC_TOP + 1))

__host__ __device__ __forceinline__ constexpr int tri(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ __forceinline__ constexpr int ncoef(int p) { return (p + 1) * (p + 2) / 2; }

// ---------------------------------------------------------------- complex helpers
template <typename T> struct cplx;
template <> struct cplx<float> { typedef float2 type; };
template <> struct cplx<double> { typedef double2 type; };
template <typename T> struct vec4;
template <> struct vec4<float> { typedef float4 type; };
template <> struct vec4<double> { typedef double4_32a type; };

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmk(double x, double y) {
  C r; r.x = x; r.y = y; return r;
}
// value at (n, m) for any sign of m from a table holding 0 <= m <= n
template <typename C> __device__ __forceinline__ C tab_get(const C* t, int n, int m) {
  if (m >= 0) return t[tri(n, m)];
  C v = t[tri(n, -m)];
  v.y = -v.y;
  if (m & 1) { v.x = -v.x; v.y = -v.y; }
  return v;
}

// ---------------------------------------------------------------- geometry
struct Geo {
  int L, p, P, P2;        // levels, order, ncoef(p), ncoef(2p)
  int nL;                 // leaves per side (2^(L-1))
  int cap;                // slots per leaf
  int64_t n;              // charges
  int64_t ML;             // number of leaves
  double a, w;            // box edge, leaf width
  int E;                  // lattice edge (0 = off-lattice)
  int W;                  // lattice sites per leaf side (E / nL)
  double h;               // lattice spacing
  int64_t cell_off[KMC_MAXL + 2];  // first cell of level l in per-level arrays (l = 1..L)
  int64_t ncell_total;
  double kT;
  double inv_a;           // 1 / a
  int prec;               // 0 = FP64 form, 1 = mixed form
  double qmax;            // largest |charge|
  int m2l;                // M2L arithmetic (kmc_m2l): 0 tensor cores (tcgen05, p <= 14; mma.sync to p = 16; else FP64),
                          // 1 FP64, 2 the mma.sync tensor-core form
  int nhop;               // lattice hops per charge: 6 (faces) or 14 (faces and body diagonals)
  int bc;                 // boundary conditions: 0 periodic (tinfoil), 1 free space
  double dipc;            // 4 pi / (3 V): the dipole (surface) term's factor; 0 in free space
  int dirichlet;          // 1: grounded walls at z = 0 and z = a/2 by mirror charges (lattice mode)
  int64_t nphys;          // charges below the mirror plane (the caller's); their mirrors follow
  double field_z;         // applied field along z (Dirichlet walls)
  int near_cache;         // 1: near-field sums of every site kept in d.nearfx (lattice mode)
  int near_ks;            // their fixed-point exponent: value = nearfx * 2^-near_ks
  int l2l;                // kmc_l2l: arithmetic of the mixed form's per-step downward pass
};

// cell coordinate of x on a level with n cells per side, floor(x n / a)
// clamped to [0, n); the one rule used by binning, accept and evaluation
__device__ __forceinline__ int cell_at(double x, int n, double inv_a) {
  int c = (int)floor(x * ((double)n * inv_a));
  return min(max(c, 0), n - 1);
}

struct MoveRec {
  int32_t valid;      // 1 if a move is to be applied
  int32_t i;          // particle (user index)
  int32_t site_old, site_new;   // lattice sites (or -1)
  double q;
  double r[3];        // old position (primary cell)
  double rn[3];       // new position (primary cell)
  double dU;          // energy change of this move
};

// All device buffers owned by a handle (plain pointers, passed by value).
#define KMC_DIP_BLOCKS 304  // blocks of the dipole reduction (two per SM)
struct Dev {
  // particles, user order
  double* q;          // [n]
  double* pos;        // [n*3]
  int32_t* site;      // [n] lattice site or -1
  int32_t* slot_of;   // [n]
  // leaf-sorted slots
  int32_t* cnt;       // [ML]
  int32_t* uid;       // [ML*cap]
  double4_32a* spos64;    // [ML*cap] (x,y,z,q)
  float4* spos32;     // [ML*cap]
  // expansions (all levels, cell-major, ncoef(p) per cell)
  double2* Mt;        // multipoles
  double2* Psi;       // per-level interaction-list local expansions; level 1 holds H
  void* Peff;         // downward-accumulated locals (T2), all levels
  double2* Itab;      // M2L irregular values [(L+1) * 343 * P2]
  double2* Itab2;     // level-2 M2L irregular values [KMC_TOP_NOFF * P2]
  double2* Rch;       // child-offset regular harmonics [(L+1) * 8 * P]
  double2* Rcoarse;   // ancestor-offset regular harmonics of levels 2..KMC_DOWN_COARSE [KMC_COARSE_TABLES * P]
  double2* S;         // lattice sums over the far images [P2]
  double* selfc;      // [KMC_MAXHOP] self-pair correction C(d) per hop direction
  // Dirichlet walls: C(d) of the charge-mirror displacements, FP64 and FP32
  double* dirA;       // [E/2]  C(0, 0, (2z + 1 - E) h): charge at z-site z and its mirror
  double* dirB;       // [nhop E/2]  C(hx h, hy h, (2z + hz + 1 - E) h): after hop k, to the old mirror
  float* dirA32;
  float* dirB32;
  long long* nearfx;  // [ML * cap] near-field sum at every site of every leaf (local site index
                      // x + W (y + W z)), fixed point, lattice units
  double* isq;        // [KMC_ISQ_N] 1/sqrt(n), n the squared lattice distance (entry 0 = 0)
  double* dip;        // [3] dipole moment M
  double* dip_part;   // [3 * KMC_DIP_BLOCKS] per-block partial sums of M
  float* fdip;        // [3] (4 pi / 3V) M in FP32 for the mixed rate assembly
  double* U;          // [1] total energy
  // FP32 copies used by the mixed form (NULL in the FP64 form)
  float* q32;         // [n] charges
  float* selfc32;     // [KMC_MAXHOP]
  float2* Psi32;      // per-level locals, all levels
  float2* Rch32;      // child-offset regular harmonics
  float2* Rcoarse32;  // ancestor-offset regular harmonics
  float* phi_old32;   // [n]
  float* phi_new32;   // [nhop n]
  float* dU32;        // [6n]
  float* l2lT;        // tensor-core downward pass: translation matrices (hi, lo planes), or NULL
  float* l2lA;        // its split parents' expansions (hi, lo planes)
  // per step
  double* phi_old;    // [n]
  double* phi_new;    // [nhop n]
  uint8_t* mask;      // [nhop n]
  double* dU;         // [nhop n]
  double* rate;       // [nhop n]
  double* bsum;       // [nblk]
  int64_t* event;     // [1]
  double* dtq;        // [2] (dt, Q)
  MoveRec* move;      // [1]
  double2* acc_scratch;  // coarse-level (2, 3) P2L terms of the accepted move
  int* err;           // [4] device error flags
  double* scratch;    // init-time scratch (lattice-sum terms)
  double* uni_small;  // [2] (zeta, xi) staged for a single kmc_step
  // device-driven step loop
  int* stepc;         // [1] step counter
  double* uni_run;    // [2*steps] uniforms
  int64_t* ev_hist;   // [steps] selected events
  double* dt_hist;    // [steps] time increments
};

// One member of a batch of independent systems advanced by the same kernels:
// its geometry and its device buffers.  A batched launch covers the blocks of
// every member; blocks [off[r], off[r + 1]) belong to member r.
struct BatchRep {
  Geo g;
  Dev d;
};

// member r of block b: the largest r with off[r] <= b (members without
// blocks in this launch have off[r] == off[r + 1] and are skipped); off[R] is
// the launch's block count
__device__ __forceinline__ int batch_find(const int* off, int R, int b) {
  int lo = 0, hi = R;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// device error codes (bit flags in err[0])
#define KMC_DERR_CAPACITY 1
#define KMC_DERR_SINGULAR 2
#define KMC_DERR_BADPOS 4
#define KMC_DERR_BADSITE 8
#define KMC_DERR_TIMEOUT 16
#define KMC_DERR_BOUNDS 32  // checked builds: an index failed its bounds check

// Bounds checks compiled into checked builds (-DKMC_CHECKS; compute-sanitizer is
// not available): KMC_IN(cond, err) is true in normal builds; in checked builds
// it sets KMC_DERR_BOUNDS in *err when cond fails, and the guarded access is
// skipped.  Usage: if (KMC_IN(i < n, d.err)) a[i] = v;
#ifdef KMC_CHECKS
__device__ __forceinline__ bool kmc_in(bool ok, int* err) {
  if (!ok) atomicOr(err, KMC_DERR_BOUNDS);
  return ok;
}
#define KMC_IN(cond, err) kmc_in((cond), (err))
#else
#define KMC_IN(cond, err) true
#endif


// 1/((n-m)(n+m)) for n > m, table built on the host into constant memory by each TU
#define KMC_NTRI (((2 * KMC_MAXP + 1) * (2 * KMC_MAXP + 2)) / 2)

// ---- bulk asynchronous copies (global -> shared) completed on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t gsrc;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(gsrc) : "l"(src));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// potentially blocking test: the thread is suspended until the phase completes
// or a time limit of the hardware runs out, so a waiting warp issues few
// instructions
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for phase `parity` of the barrier, at most ~limit_ns; false on timeout
// (the clock is read on every 32nd retry only: a read of %globaltimer costs more than a retry,
// and a thread that reads it right after the phase completes wakes late)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_test(bar, parity)) return true;
  uint64_t t0 = 0;
  for (uint32_t it = 1;; it++) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 31) == 0) {
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}
#define KMC_WAIT_NS 1000000000ull  // one second

// ---------------------------------------------------------------- M2L slicing (Algorithm 2 on the tensor cores)
// slice counts, tile paddings and the scaling exponent shared by the slicing
// kernels and both tensor-core M2L kernels
#define OZ_S 6
#define OZ_S_MIXED 4
static __host__ __device__ __forceinline__ int oz_slices(const Geo& g) { return g.prec == 1 ? OZ_S_MIXED : OZ_S; }
#define OZ_MT 64
#define OZ_NT 64
#define OZ_KC 32
#define OZ_LD (OZ_KC + 8)  // shared row stride (bf16): 80 B rows, conflict-free ldmatrix
#define OZ_MAXP 16
#define OZ_MAXP_P 153  // ncoef(OZ_MAXP)

static __host__ __device__ __forceinline__ int oz_rows(int n2) { return (n2 + OZ_MT - 1) / OZ_MT * OZ_MT; }
static __host__ __device__ __forceinline__ int oz_cols(int n2) { return (n2 + OZ_KC - 1) / OZ_KC * OZ_KC; }

// 2^e with e the smallest integer such that |x| < 2^e for every |x| <= m (0 if m = 0)
__device__ __forceinline__ int oz_exp(unsigned long long mbits) {
  const double m = __longlong_as_double((long long)mbits);
  return m > 0.0 ? ilogb(m) + 1 : 0;
}

// ---------------------------------------------------------------- launch wrappers
// (defined in the .cu files, called by the host runtime)
void fmm_upload_constants(int p);
void fmm_bin(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_p2m(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_m2m(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_itab(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_child_tables(const Geo& g, const Dev& d, cudaStream_t s);  // child and ancestor offset tables
size_t fmm_m2l_scratch_bytes(const Geo& g);
// ev: null, or 2 (KMC_MAXL + 1) events recorded around level l's M2L product kernel (2 l, 2 l + 1)
void fmm_m2l(const Geo& g, const Dev& d, void* scratch, cudaStream_t s, cudaEvent_t* ev = nullptr);
// per-step downward pass of the mixed form's finest level on tcgen05 (tf32 x 3)
// its operands (the split parents' expansions, planes hi / lo of l2l_npad(L) rows x l2l_K(P)
// values, and the translation tables) sit in blocks of `rows` rows x 32 values (block
// (r / rows) nkc + c / 32), each block in the order of the MMA's 128-byte-swizzled K-major
// shared-memory operand, so that one block is one contiguous TMA copy: the offset (in values)
// of row r, column c
__host__ __device__ __forceinline__ int64_t l2l_sw_off(int64_t r, int c, int rows, int nkc) {
  const int64_t blk = (r / rows) * nkc + (c >> 5);
  const int rr = (int)(r % rows), k = c & 31;
  return blk * rows * 32 + (((rr >> 3) * 1024 + (rr & 7) * 128 + ((((k >> 2) ^ rr) & 7) << 4)) >> 2) + (k & 3);
}
__host__ __device__ __forceinline__ int l2l_K(int P) { return 32 * ((2 * P + 31) / 32); }
__host__ __device__ __forceinline__ int64_t l2l_npad(int L) { return ((((int64_t)1 << (3 * (L - 2))) + 127) / 128) * 128; }
// x rounded to the nearest TF32 value (10 explicit mantissa bits; ties away from zero)
__device__ __forceinline__ float l2l_tf32(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }
int fmm_l2l_tc_first(const Geo& g);               // first level it covers, 0 if none
size_t fmm_l2l_tc_table_floats(const Geo& g);     // l2lT size
size_t fmm_l2l_tc_split_floats(const Geo& g);     // l2lA size
void fmm_l2l_tc_tables(const Geo& g, const Dev& d, cudaStream_t s);  // at init, after the child tables
bool fmm_l2l_tc(const Geo& g, const Dev& d, int l, cudaStream_t s);  // level l; false: not launched
int tc_probe_tf32(float* out);                    // self-check of the tf32 MMA path
bool fmm_m2l_tc_ok(const Geo& g);           // the tcgen05 M2L applies (KMC_M2L_TENSOR, p <= 14)
int fmm_m2l_tc_rows(const Geo& g);           // its MMA N (rows of its A-slice layout), 0 if p > 14
int fmm_m2l_tc_kchunks(const Geo& g);        // its K chunks of 64 values
// level l's M2L from the slices in the tcgen05 layouts (As: k_oz_aslice_tc, Bp:
// k_oz_bslice_tc) into acc64 (zeroed; k_oz_finish converts); false: not launched
bool fmm_m2l_tc(const Geo& g, const Dev& d, int l, const unsigned short* As, const unsigned short* Bp,
                long long* acc64, cudaStream_t s);
void fmm_dirichlet_tables(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_mirror_move(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_near_fill(const Geo& g, const Dev& d, int prec, cudaStream_t s);
void kmc_dirichlet_energy(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_lattice_sums(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_far_field(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_self_and_dipole(const Geo& g, const Dev& d, cudaStream_t s);
void fmm_prepare(const Geo& g, int prec);
void fmm_downward(const Geo& g, const Dev& d, int prec, cudaStream_t s);
void fmm_selfcorr_list(const Geo& g, const Dev& d, int64_t m, const double* dvec, double* out, cudaStream_t s);
void fmm_drift1(const double* a, const double* b, int64_t count, double* out2, cudaStream_t s);
void fmm_drift(const Geo& g, const double2* a, const double2* b, int64_t count, double* out2,
               cudaStream_t s);

void kmc_upload_constants(int p);
void kmc_propose_lattice(const Geo& g, const Dev& d, int prec, cudaStream_t s);
void kmc_finalize_rates(const Geo& g, const Dev& d, int prec, cudaStream_t s);
void kmc_prepare(const Geo& g, int prec);
int kmc_wait_probe(double limit_seconds, cudaStream_t s);  // flag bits, -1 on a CUDA error
void kmc_rate_bsum(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_select(const Geo& g, const Dev& d, int use_counter, cudaStream_t s);
void kmc_record(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_accept_from_event(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_accept_apply(const Geo& g, const Dev& d, cudaStream_t s);
void kmc_eval_points(const Geo& g, const Dev& d, int prec, int64_t m, const double* pts,
                     const int32_t* excl, double* out, cudaStream_t s);
void kmc_assemble_general(const Geo& g, const Dev& d, int64_t m, const int32_t* particle,
                          const double* tgt, const uint8_t* mask, const double* phi_new,
                          const double* phi_old, double* dU, cudaStream_t s);
void kmc_stage_general(const Geo& g, const Dev& d, int64_t m, const int32_t* part, const double* tin,
                       const uint8_t* min_, double* tout, double* old, double* dv, uint8_t* mout, cudaStream_t s);
void kmc_widen(const float* src, double* dst, int64_t n, cudaStream_t s);
void fmm_shadow_all(const Geo& g, const Dev& d, cudaStream_t s);
int kmc_coarse_slots();
void raise_dynamic_smem(const void* fn, size_t bytes);
void kmc_energy_reduce(const Geo& g, const Dev& d, cudaStream_t s);

// Launch plan of one batched KMC step: every launch covers all members of a
// batch (BatchRep), member r owning blocks [off[r], off[r + 1]) of it.  Host
// struct; the arrays it points to live on the device.
struct BatchPlan {
  int R;                      // members
  int prec, nhop, near_cache; // shared by all members
  int Lmax;                   // deepest tree among the members
  int chunk;                  // requested pass capacity (0: each member's smallest)
  const BatchRep* reps;       // [R]
  const int* off_down[KMC_MAXL + 1];  // level l >= 2: the parent cells of level l - 1 of members with L >= l
  int nblk_down[KMC_MAXL + 1];
  size_t smem_down;
  // propose: one launch per class of members with the same pass capacity (their leaves)
  int nprop;
  int chunk_c[KMC_MAXL];
  const int* off_prop[KMC_MAXL];
  int nblk_prop[KMC_MAXL];
  size_t smem_prop[KMC_MAXL];
  const int* off_fin;         // rate blocks of KMC_FIN_PARTICLES charges
  int nblk_fin;
  const int* off_acc;         // fused accept blocks
  int nblk_acc;
  const int* off_acr;         // coarse-cell reduction blocks (72 per member)
  int nblk_acr;
  size_t smem_acr;
  const int* off_nu;          // near-field cache update blocks (54 per member with the cache)
  int nblk_nu;
};
void fmm_downward_batch(const BatchPlan& bp, cudaStream_t s);
size_t fmm_coarse_smem(int p, int prec);  // dynamic shared memory of the coarse-level downward kernel
void kmc_propose_batch(const BatchPlan& bp, cudaStream_t s);
void kmc_step_batch(const BatchPlan& bp, cudaStream_t s);  // propose, rates, select, record, accept
void kmc_batch_prepare(const BatchPlan& bp);                // load the kernels, raise their smem limits
int kmc_propose_chunk_min(const Geo& g);                    // smallest pass capacity for g's leaves
size_t kmc_propose_smem_for(const Geo& g, int prec, int chunk, int cached);
int kmc_acc_blocks_for(const Geo& g);
int kmc_acr_blocks();
size_t kmc_acr_smem_for(const Geo& g);
void kmc_validate(const Geo& g, const Dev& d, cudaStream_t s);
