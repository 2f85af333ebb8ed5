/*
 * kmcfmm.h -- C ABI of the GB300 (sm_103a) FMM-for-KMC library.
 *
 * The library evaluates, for a neutral periodic system of point charges in a
 * cubic box of edge a, the electrostatic energy change dU of single-charge
 * hops ("propose", Sec. 3 Eq. (proposed_energy) and its periodic form
 * Eq. (proposed_energy_sr) plus the far field of Sec. 3.1), selects an event
 * with rejection-free KMC (Algorithm 1), and applies the incremental update
 * of the expansions when a hop is accepted (Sec. 3, "Accept move").  The
 * one-off full FMM (Algorithm 2: P2M, M2M, M2L over wrapped interaction
 * lists; the periodic lattice operator of Sec. 2.2.1) runs on the device.
 *
 * Energy convention: conducting ("tinfoil") boundary at infinity, i.e. the
 * cubic-order lattice sum with the surface term of Sec. 2.2.2 / App. B
 * removed.  This equals the Ewald energy with the k = 0 term omitted.
 *
 * Conventions common to every call
 * --------------------------------
 *  - Every function returns KMC_OK (0) or a KMC_ERR_* code; after an error
 *    kmc_last_error(h) returns a message.  Errors are sticky for a handle
 *    only when the device state may be inconsistent (KMC_ERR_CUDA,
 *    KMC_ERR_CAPACITY); then every later call returns KMC_ERR_STATE.
 *  - Array arguments live in host memory or in device memory of the
 *    handle's GPU, as kmc_opts.mem says (KMC_MEM_HOST / KMC_MEM_DEVICE).
 *    Scalar outputs (energy, event, dt, Q, drift) are always host pointers.
 *  - The caller owns every buffer it passes; the library copies inputs into
 *    its own device layout and never keeps or frees a caller pointer.
 *  - All device work is ordered on the stream given in kmc_opts.stream
 *    (a cudaStream_t; NULL = legacy default stream).  Calls that return a
 *    host scalar or write host arrays synchronise that stream.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Indices: particles are numbered 0..n-1 in the caller's order ("user
 *    order").  Lattice hop k of particle i is the event j = nh i + k, nh the
 *    number of hops of the handle's hop set (kmc_opts.hops): k = 0..5 for the
 *    faces (+x, -x, +y, -y, +z, -z) and, with KMC_HOPS_14, k = 6..13 for the
 *    body diagonals (+-1, +-1, +-1) with x fastest: (+,+,+), (-,+,+), (+,-,+),
 *    (-,-,+), (+,+,-), (-,+,-), (+,-,-), (-,-,-).  Targets wrap periodically.
 */
#ifndef KMCFMM_H
#define KMCFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum kmc_status {
  KMC_OK = 0,
  KMC_ERR_ARG = 1,         /* invalid argument (sizes, levels, order, positions, singular move) */
  KMC_ERR_NOT_NEUTRAL = 2, /* sum of charges != 0 (the periodic sums diverge, Sec. 2.2.1) */
  KMC_ERR_OOM = 3,         /* device allocation failed */
  KMC_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  KMC_ERR_CAPACITY = 5,    /* a leaf cell ran out of slots */
  KMC_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  KMC_ERR_STATE = 7        /* handle unusable after an earlier error, or wrong call order */
};

enum kmc_precision {
  KMC_PREC_FP64 = 0, /* every step in FP64 */
  KMC_PREC_MIXED = 1 /* L2P, the near-field pair sums and the dU assembly (q (phi' - phi) less
                        the dipole and self-image terms) in FP32 with FP32 accumulation, the
                        rates from an FP32 exponent kept in FP64 range; lattice sums, the
                        accept updates of the expansions and the cumulative rate sums in FP64;
                        the tensor-core M2L on four slices (29-bit operands, see kmc_m2l) */
};

enum kmc_mem { KMC_MEM_HOST = 0, KMC_MEM_DEVICE = 1 };

/* Boundary conditions (Sec. 2.2). */
enum kmc_bc {
  KMC_BC_PERIODIC = 0, /* the box replicated periodically, conducting boundary at infinity; the
                          system must be neutral */
  KMC_BC_FREE = 1,     /* free space: the charges of the box alone, no images (Eq. (proposed_energy)
                          as written); any net charge; lattice hops leaving the box are masked and
                          general targets outside [0, box) are rejected */
  KMC_BC_DIRICHLET_Z = 2 /* grounded walls (phi = 0) at z = 0 and z = box/2 with an applied field
                          field_z along z, periodic in x and y (the Dirichlet case of Sec. 2.2):
                          lattice mode only, even lattice edge, every charge below z = box/2.  The
                          library appends a mirror of opposite charge at (x, y, box - z) for every
                          charge and runs the periodic method on the mirrored cell; a hop moves a
                          charge and its mirror together, hops through a wall are masked,
                          U = U_mirrored / 2 - field_z sum q z and dU = U(after) - U(before).  The
                          outputs cover the caller's n charges only; general proposals and moves
                          (kmc_fmm_propose, kmc_fmm_accept) and caller rates in kmc_step return
                          KMC_ERR_STATE. */
};

/* Lattice hop set (the moves Algorithm 5 proposes for every charge). */
enum kmc_hops {
  KMC_HOPS_6 = 0, /* the 6 nearest-neighbour sites */
  KMC_HOPS_14 = 1 /* the 6 faces and the 8 body diagonals at distance sqrt(3) h: the hop set of the
                     paper's Sec. 5.3 scaling benchmark */
};

/* Arithmetic of the one-off M2L (Algorithm 2, translations grouped by vector
 * as dense real matrix products).  Both give FP64-accurate results in the FP64
 * form. */
enum kmc_m2l {
  KMC_M2L_TENSOR = 0,      /* bf16 tensor cores with exact integer slicing of the FP64 operands
                              (six 7-bit slices, 21 slice products, exact per-diagonal sums; the
                              mixed form four slices, 10 products, 29 significant bits), on the
                              fifth-generation MMA (tcgen05, TMEM accumulators, TMA staging) for
                              p <= 14, the mma.sync form for p = 15, 16; FP64 CUDA cores when p > 16 */
  KMC_M2L_FP64 = 1,        /* FP64 CUDA cores */
  KMC_M2L_TENSOR_SYNC = 2  /* the same slicing on the warp-level mma.sync form (p <= 16, else FP64):
                              bit for bit the result of KMC_M2L_TENSOR, kept as its cross-check */
};

/* Arithmetic of the mixed form's per-step downward pass (the L2L translations
 * of the accumulated local expansions, Algorithm 2's downward pass) on its two
 * finest levels; the FP64 form and the coarser levels always use CUDA cores. */
enum kmc_l2l {
  KMC_L2L_TENSOR = 0, /* tcgen05 kind::tf32 MMAs, each FP32 operand split into two TF32 parts
                         (hi hi + hi lo + lo hi, FP32 accumulation), p <= 14 */
  KMC_L2L_CUDA = 1    /* FP32 CUDA cores */
};

typedef struct kmc_opts {
  int precision;      /* kmc_precision */
  int lattice_edge;   /* E > 0: lattice mode, sites at ((i+1/2)h, (j+1/2)h, (k+1/2)h),
                         box = E*h, E must be a multiple of 2^(levels-1);
                         0: off-lattice (only kmc_fmm_propose / kmc_fmm_accept) */
  double lattice_h;   /* lattice spacing h (lattice mode) */
  double kT;          /* rate rule r = exp(-max(dU,0)/kT) used by kmc_step / kmc_run */
  void* stream;       /* cudaStream_t for all device work; NULL = default stream */
  int mem;            /* kmc_mem: where array arguments live */
  int device;         /* CUDA device ordinal */
  int leaf_capacity;  /* off-lattice slots per leaf (0 = automatic); lattice mode uses (E/2^(L-1))^3 */
  int m2l;            /* kmc_m2l: arithmetic of the M2L at init and recompute */
  int hops;           /* kmc_hops: lattice hop set (nh = 6 or 14 hops per charge) */
  int bc;             /* kmc_bc: boundary conditions */
  double field_z;     /* applied electric field along z with Dirichlet walls (energy -q field_z z) */
  int near_cache;     /* lattice mode: 1 = keep the near-field sum (the direct part of phi, Sec. 3,
                         Eq. (proposed_energy_sr): charges in the 27 leaves around the site's leaf) of
                         every site in device memory, 8 bytes per site, filled at init and recompute
                         and updated by every accepted move for the sites whose neighbourhood holds
                         the old or the new position; proposals then read it instead of summing the
                         pairs.  The values agree with the per-step sum to rounding (fixed point,
                         2^-k with 2^k |sum| < 2^62).  0 = sum every step (default). */
  int l2l;            /* kmc_l2l: arithmetic of the mixed form's per-step downward pass */
} kmc_opts;

typedef struct kmc_fmm* kmc_handle;

/* Fill opts with defaults: FP64, off-lattice, h = 1, kT = 1, NULL stream, host memory, device 0,
 * tensor-core M2L, 6 hops, periodic, no applied field, near field summed every step. */
void kmc_opts_default(kmc_opts* opts);

/*
 * Create a handle and run the one-off full FMM (Algorithm 2 with the periodic
 * modifications of Sec. 3.1: wrapped interaction lists, the lattice-sum far
 * field H = R K of Sec. 2.2.1, the dipole field of Sec. 2.2.2).
 *   positions: n x 3 doubles (row-major), each coordinate in [0, box).
 *   charges:   n doubles, sum must vanish (relative 1e-12 of sum |q|).
 *   levels:    L >= 3 (8^(l-1) cells on level l, Sec. 2.2); at most 10.
 *   order:     p, the largest expansion degree (Eq. (multipole_local_expansion)
 *              sums n = 0..p), 1 <= p <= 24.
 * Errors: KMC_ERR_ARG (n < 2, levels/order out of range, a position outside
 * [0, box) or not finite, lattice positions off the sites or two charges on
 * one site, box not divisible), KMC_ERR_NOT_NEUTRAL, KMC_ERR_OOM, KMC_ERR_CUDA.
 * On error *h is set to NULL unless the handle could be created, in which
 * case it holds the error message and must be destroyed.
 */
int kmc_fmm_init(kmc_handle* h, int64_t n, const double* positions, const double* charges, double box,
                 int levels, int order, const kmc_opts* opts);

/* Total energy U (Algorithm 3 plus the far field and the dipole term), host scalar. */
int kmc_fmm_energy(kmc_handle h, double* U);

/*
 * dU for m arbitrary proposals (the propose() / propose_with_dats() interface
 * of Sec. 4.2 and App. C, flattened): proposal t moves particle[t] to
 * target[3t..3t+2] (wrapped into the box).  mask may be NULL; where
 * mask[t] == 0 the proposal is skipped and dU[t] = NaN (the paper leaves such
 * entries undefined).  A target equal to the particle's own position, or
 * equal to another charge's position, is singular: dU[t] = NaN and the call
 * returns KMC_ERR_ARG after filling every other entry.
 */
int kmc_fmm_propose(kmc_handle h, int64_t m, const int32_t* particle, const double* target,
                    const uint8_t* mask, double* dU);

/*
 * Lattice mode: proposal generation (each charge to the nh sites of its hop
 * set, masked when occupied, as in Algorithm 5) and dU for every unmasked
 * hop.  mask and dU are n x nh (event order j = nh i + k); masked entries get
 * mask 0 and dU NaN.  Either output may be NULL.  The rates for kmc_step are
 * kept on the device.
 */
int kmc_fmm_propose_lattice(kmc_handle h, uint8_t* mask, double* dU);
/*
 * The same for the mixed-precision form, with dU in FP32: the form's own
 * result (its dU assembly is FP32), copied without widening, 4 bytes per hop
 * instead of 8.  KMC_ERR_STATE for an FP64-form handle.
 */
int kmc_fmm_propose_lattice_f32(kmc_handle h, uint8_t* mask, float* dU);
/*
 * The mixed-form FP32 call without waiting: the proposal, the rates and the
 * copies of mask and dU are enqueued and the call returns (kmc_step may follow
 * at once: it runs after the proposal); the copies into mask and dU (pinned
 * host or device memory, owned by the caller) run on a stream of their own,
 * overlapping the calls that follow.  Errors of the proposal's kernels are
 * reported by the next call that synchronises (kmc_step, kmc_fmm_outputs_wait).
 * kmc_step and kmc_fmm_accept_event run beside the copies; every other call
 * on the handle is ordered after them.  The outputs may be read, and their
 * memory reused or freed, after kmc_fmm_outputs_wait (which blocks until the
 * pending copies are done; KMC_OK when none is pending) or after the next
 * proposal call on the handle has returned (it is ordered after them and
 * waits for its own kernels).  KMC_ERR_STATE for an FP64-form handle.
 */
int kmc_fmm_propose_lattice_async(kmc_handle h, uint8_t* mask, float* dU);
int kmc_fmm_outputs_wait(kmc_handle h);

/*
 * Accept the move of particle to target (wrapped), whether proposed or not:
 * dU is recomputed (Sec. 3.1 footnote), the per-level local expansions, the
 * multipoles, the far-field coefficients, the dipole and the energy are
 * updated, and the charge changes leaf.  dU_accepted (host, may be NULL)
 * receives dU.  Errors: KMC_ERR_ARG (bad index, singular target, lattice
 * target off a site), KMC_ERR_CAPACITY.
 */
int kmc_fmm_accept(kmc_handle h, int32_t particle, const double target[3], double* dU_accepted);

/*
 * Lattice mode: accept event j = nh i + k (hop k of particle i), with the
 * updates of kmc_fmm_accept.  When the rates of the last kmc_fmm_propose_lattice
 * are still current (no accept since), the move is built on the device from the
 * event and dU_accepted receives that proposal's dU (FP32 in the mixed form);
 * otherwise the move goes through kmc_fmm_accept and dU is recomputed.  With
 * Dirichlet walls the charge's mirror moves with it.  Errors: KMC_ERR_ARG (index
 * out of range, a masked event: occupied target or, with walls, a wall).
 */
int kmc_fmm_accept_event(kmc_handle h, int64_t event, double* dU_accepted);

/*
 * Rejection-free selection (Algorithm 1): rates r_j (m = nh n entries in event
 * order, or NULL to use the rates of the last kmc_fmm_propose_lattice),
 * Q = sum r_j, event j with R_{j-1} < Q zeta <= R_j, dt = -ln(xi) / Q.
 * zeta, xi in (0, 1].  Outputs are host scalars; *event = -1 if Q == 0.
 * Does not accept the event.
 */
int kmc_step(kmc_handle h, const double* rates, double zeta, double xi, int64_t* event, double* dt,
             double* Q);

/*
 * Lattice mode: run `steps` full KMC steps on the device without host
 * synchronisation (propose -> rates -> select -> accept per step, replayed
 * from a CUDA graph).  uniforms: steps x 2 values (zeta_s, xi_s) in (0, 1].
 * events (int64, steps) and dts (double, steps) receive the selected events
 * and time increments; either may be NULL.
 */
int kmc_run(kmc_handle h, int steps, const double* uniforms, int64_t* events, double* dts);

/*
 * kmc_run without graph replay, with per-phase device timing: phase_ms
 * (host, KMC_NPHASE doubles, may be NULL) receives the summed duration of
 * each phase over all steps, measured with CUDA events on the handle's
 * stream: [0] downward pass, [1] propose kernel (near-field pairs + L2P),
 * [2] dU / rates, [3] selection, [4] accept updates.  Same results as
 * kmc_run.  Synchronises the stream.
 */
#define KMC_NPHASE 5
int kmc_run_profiled(kmc_handle h, int steps, const double* uniforms, int64_t* events, double* dts,
                     double* phase_ms);

/*
 * Full FP64 recompute of every expansion from the current positions
 * (Algorithm 2), replacing the incrementally updated ones; the energy is
 * recomputed.  drift (host, 3 doubles, may be NULL) receives the drift of the
 * incremental accept updates measured against the fresh expansions:
 *   [0] max_i |phi_incr(r_i) - phi_fresh(r_i)| / max_i |phi_fresh(r_i)|
 *       (potential at every charge, own term excluded),
 *   [1] max |Psi_incr - Psi_fresh| / max |Psi_fresh| over all coefficients
 *       of all levels (high-order coefficients of a local expansion carry the
 *       truncation error of the M2L, so this is an upper bound),
 *   [2] |U_tracked - U_fresh| / |U_fresh| (energy accumulated from the
 *       accepted dU against the recomputed energy).
 */
int kmc_fmm_recompute(kmc_handle h, double* drift);

/*
 * Leaf-cell index of every particle, user order: the finest-level cell of the
 * octree of Sec. 2.2 (8^(L-1) cells on level L) that holds it,
 * cx + n (cy + n cz) with n = 2^(L-1) and c = floor(x n / box) per axis.  An
 * inspection hook (tests compare it bit-exactly with integer arithmetic); the
 * binning it reports is the one every kernel uses.  leaf: n int32, in the
 * handle's memory kind.
 */
int kmc_fmm_leaf_index(kmc_handle h, int32_t* leaf);

/*
 * Current positions (n x 3 doubles, row-major, user order, wrapped into
 * [0, box)) after the accepted moves so far: the state Algorithm 1 advances.
 * An inspection and checkpoint hook; positions: in the handle's memory kind.
 */
int kmc_fmm_positions(kmc_handle h, double* positions);

/*
 * Allocation-free selection.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- a library running
 * inside a framework whose caching allocator owns the device memory, a host
 * loop that must not stall on the device synchronisation cudaMalloc/cudaFree
 * can cause, a plugin host that forbids its plugins to own device memory.  It
 * performs the selection of kmc_step (Q = sum r_j, event j with
 * R_{j-1} < Q zeta <= R_j, dt = -ln(xi)/Q) without a handle and without
 * allocating: its scratch is a file-scope device array of KMC_STATIC_MAX_N/128
 * block sums plus 8 doubles (about 1 MB), held by every GPU that loads the
 * library until the process exits.
 *   rates:  6 n doubles in DEVICE memory of the current device (event order
 *           j = 6 i + k), owned by the caller; 1 <= n <= KMC_STATIC_MAX_N,
 *           larger n returns KMC_ERR_ARG.  The library reads exactly 6 n
 *           entries and cannot check the buffer's length: the caller must.
 *   zeta, xi in (0, 1]; event, dt, Q: host scalars (event = -1 if Q == 0).
 *   stream: cudaStream_t (NULL = default stream); the call copies the two
 *           uniforms from the host and synchronises the stream.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array,
 * so calls whose GPU work overlaps (other streams, other host threads) race;
 * serialise them.  Nothing in the array has to start at zero: each call
 * writes every element it reads.
 */
#define KMC_STATIC_MAX_N 16777216
int kmc_select_static(const double* rates, int64_t n, double zeta, double xi, int64_t* event, double* dt,
                      double* Q, void* stream);

/*
 * Replica batches (many independent systems advanced together, the ensemble
 * parallelism of Sec. 5.4 on one GPU).  A batch holds `count` lattice-mode
 * handles on one device (not owned; they must outlive the batch).
 *   When the members share precision, hop set and near-field mode and have no
 *   Dirichlet walls, every launch of a batch step covers all members: the
 *   downward pass (one launch per level), the propose over the flattened list
 *   of all members' leaves, the rates over all members' charges, one
 *   selection CTA per member (the per-member segment of the cumulative rate
 *   sums), the members' move records and the accept updates -- L_max + 6
 *   launches per step whatever the number of members (one more per extra
 *   leaf-capacity class of the propose, one more with the near-field cache),
 *   replayed from a CUDA graph.  Members may differ in size, levels and order.
 *   Otherwise each member's own step is a parallel branch of one graph.
 *   kmc_batch_run: uniforms (HOST) steps x count x 2 values (zeta, xi) laid
 *   out [step][member][2]; events (int64) and dts (HOST, steps x count,
 *   [step][member], may be NULL).  The same events as kmc_run on each
 *   member (unless a uniform falls within rounding of a cumulative-rate
 *   boundary); with batched kernels the time increments agree to rounding
 *   (the batch translates the downward pass level by level, a single system
 *   sums the coarse levels' translations in one launch: the same expansions
 *   in another order).
 *   kmc_batch_run_timed: the same, and device_ms (host) receives the device
 *   time of the steps (CUDA events on the batch's stream around the step
 *   launches; staging of the uniforms and reading of the events excluded).
 *   kmc_batch_set_chunk: near-field sources staged in shared memory per pass
 *   of the batched propose (the P2P tile): 0 = each member the smallest that
 *   fits its leaves, members of equal capacity sharing one propose launch
 *   (the default); else one capacity for all members (even, at least every
 *   member's leaf capacity).  KMC_ERR_STATE for a batch of members' own
 *   kernels.  Errors of every call: KMC_ERR_ARG, KMC_ERR_CUDA,
 *   KMC_ERR_OOM, or a member's error (see kmc_batch_last_error).
 *   kmc_batch_info: fused (1 = batched kernels), the largest pass capacity in
 *   use, and the kernel launches of one batch step (host ints, each may be
 *   NULL).
 *   kmc_batch_propose_timed: a measurement hook with no counterpart in the
 *   paper: runs only the batch step's propose launches (Sec. 3, Eq.
 *   (proposed_energy_sr) for every member) `reps` times on the batch's stream and stores in
 *   device_ms (host) the mean device time of one set (CUDA events).  The
 *   members' state is not changed (the next run recomputes every potential
 *   it uses).  KMC_ERR_ARG if the batch is not on the batched kernels or has
 *   not run yet.
 */
typedef struct kmc_batch* kmc_batch_handle;
int kmc_batch_create(kmc_batch_handle* b, int count, const kmc_handle* handles);
int kmc_batch_run(kmc_batch_handle b, int steps, const double* uniforms, int64_t* events, double* dts);
int kmc_batch_run_timed(kmc_batch_handle b, int steps, const double* uniforms, int64_t* events, double* dts,
                        double* device_ms);
int kmc_batch_set_chunk(kmc_batch_handle b, int chunk);
int kmc_batch_info(kmc_batch_handle b, int* fused, int* chunk, int* launches_per_step);
int kmc_batch_propose_timed(kmc_batch_handle b, int reps, double* device_ms);
const char* kmc_batch_last_error(kmc_batch_handle b);
void kmc_batch_destroy(kmc_batch_handle b);

/*
 * Timing hook with no counterpart in the paper: runs the one-off M2L of the
 * handle's current multipole expansions (Algorithm 2, every level, in the
 * handle's M2L arithmetic, kmc_m2l) reps times into a scratch copy of the
 * local expansions, so the handle's state is unchanged, and reports the mean
 * device time per run of each level's product kernel (level_ms[l], l = 3 ..
 * levels; an array of 11 doubles, other entries 0) and of the whole M2L with
 * its operand slicing (total_ms), from CUDA events on the handle's stream.
 * Allocates the M2L scratch (as init does) for the duration of the call.
 * Errors: KMC_ERR_ARG (reps <= 0, null outputs), KMC_ERR_OOM, KMC_ERR_CUDA.
 */
int kmc_fmm_m2l_timed(kmc_handle h, int reps, double* level_ms, double* total_ms);

/*
 * Diagnostic with no counterpart in the paper: runs, on `device`, the bounded
 * device-side wait that the FP32 lattice propose uses for its bulk copies,
 * against a barrier phase that can never complete (bytes expected, nothing
 * copied), with a limit of limit_seconds (clamped to [0.001, 2]).  Returns
 * KMC_ERR_TIMEOUT when the wait gave up and the kernel returned as designed,
 * KMC_OK if it did not time out (a defect), KMC_ERR_CUDA on a CUDA error.
 * Allocates a 4-byte flag for the duration of the call; no handle needed.
 */
int kmc_check_bounded_wait(int device, double limit_seconds);

/*
 * Diagnostic with no counterpart in the paper: four fifth-generation
 * tensor-core MMAs of small integer operands, staged in shared memory exactly
 * as the library's tensor-core kernels stage theirs, read back from tensor
 * memory with tcgen05.ld and compared on the host with the exact integer
 * product.  kind 0: tcgen05.mma kind::f16, M = 128, N = 192, K = 4 x 16,
 * bf16 x bf16 -> FP32, staged as the M2L stages its operands (cp.async pieces
 * for A, one 2D TMA box of a contiguous block for B, 128-byte-swizzled K-major
 * tiles, the K step advanced inside the swizzle atom); kind 1: kind::tf32,
 * M = 128, N = 192, K = 4 x 8, staged as the downward pass stages its operands
 * (2D TMA boxes of 32 FP32 values per row, 128-byte swizzle).  Returns 0 when
 * every entry agrees, 1 on a mismatch, -KMC_ERR_TIMEOUT when a bounded wait
 * gave up, -KMC_ERR_ARG for an unknown kind, -KMC_ERR_CUDA / -KMC_ERR_OOM when
 * the device, the driver's tensor-map encoder or an allocation is unavailable.
 * out: NULL, or a host array of 128 * 192 floats that receives the product as
 * read from tensor memory (row-major, row = M index).  Allocates and frees
 * about 100 kB of device memory; no handle needed.
 */
int kmc_check_tensor_mma(int device, int kind, float* out);

/* Message of the last error on this handle (static string if h is NULL). */
const char* kmc_last_error(kmc_handle h);

/* Release the handle and all device memory it owns.  NULL is allowed. */
void kmc_fmm_destroy(kmc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* KMCFMM_H */
