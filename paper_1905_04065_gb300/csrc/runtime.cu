// runtime.cu -- host runtime and C ABI of the FMM-for-KMC library (see
// include/kmcfmm.h for the contract of every entry point).
//
// The runtime owns all device memory of a handle, orders every launch on
// the caller's stream, checks every CUDA call, reads the device error flags
// after each synchronising call, and replays the device-driven KMC step loop
// from CUDA graphs.  No arithmetic of the method runs on the host.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/kmcfmm.h"
#include "common.cuh"

// NVTX range of one C-ABI call (domain "kmcfmm"), visible in Nsight Systems and
// usable as an ncu --nvtx filter; without an attached tool the calls do nothing
static nvtxDomainHandle_t trace_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("kmcfmm");
  return d;
}
struct TraceRange {
  explicit TraceRange(const char* name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(trace_domain(), &a);
  }
  ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
};
#define KMC_TRACE(name) TraceRange trace_range_(name)

struct kmc_fmm {
  Geo g;
  Dev d;
  int prec;
  int mem;
  int device;
  cudaStream_t stream;
  char msg[512];
  bool broken;
  bool peff_valid;    // leaf expansions reflect the current expansions
  bool rates_valid;   // device rates belong to the current configuration
  // asynchronous output copies (kmc_fmm_propose_lattice_async): a copy stream,
  // the events that order it after the proposal and the next writers after it
  cudaStream_t cstream;
  cudaEvent_t ev_ready, ev_copied;
  bool copy_pending;
  std::vector<void*> allocs;
  // general-propose scratch
  size_t gen_cap;
  int32_t* gen_part;
  double* gen_tgt;
  double* gen_old;
  double* gen_pn;
  double* gen_po;
  double* gen_dv;
  double* gen_du;
  uint8_t* gen_mask;
  // step-loop capacity and graph
  int run_cap;
  int run_gen;  // bumped whenever the step-loop buffers are reallocated
  cudaGraphExec_t graph;
  int graph_steps;
  double* drift2;
  double* phi_save;
  int32_t* iota;
};

static const char* g_static_msg = "invalid handle";

static int fail(kmc_fmm* h, int code, const char* fmt, ...) {
  if (!h) return code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
  va_end(ap);
  if (code == KMC_ERR_CUDA || code == KMC_ERR_CAPACITY) h->broken = true;
  return code;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(h, KMC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKLAUNCH()                                                                                \
  do {                                                                                            \
    cudaError_t e_ = cudaGetLastError();                                                          \
    if (e_ != cudaSuccess) return fail(h, KMC_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
static int dalloc(kmc_fmm* h, P** ptr, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(h, KMC_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(p);
  *ptr = (P*)p;
  return KMC_OK;
}

#define ALLOC(ptr, bytes)                        \
  do {                                           \
    int r_ = dalloc(h, &(ptr), (size_t)(bytes)); \
    if (r_) return r_;                           \
  } while (0)

static cudaMemcpyKind in_kind(const kmc_fmm* h) {
  return h->mem == KMC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind out_kind(const kmc_fmm* h) {
  return h->mem == KMC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// read and clear the device error flags; map them to a status
static int check_flags(kmc_fmm* h, const char* where) {
  int e[4];
  CK(cudaMemcpyAsync(e, h->d.err, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e[0] == 0) return KMC_OK;
  CK(cudaMemsetAsync(h->d.err, 0, sizeof(e), h->stream));
  if (e[0] & KMC_DERR_CAPACITY) return fail(h, KMC_ERR_CAPACITY, "%s: a leaf cell ran out of slots", where);
  if (e[0] & KMC_DERR_BADPOS) return fail(h, KMC_ERR_ARG, "%s: a position is not finite or outside [0, box)", where);
  if (e[0] & KMC_DERR_BADSITE) return fail(h, KMC_ERR_ARG, "%s: a position is not on a lattice site", where);
  if (e[0] & KMC_DERR_SINGULAR)
    return fail(h, KMC_ERR_ARG, "%s: a target coincides with a charge (singular move)", where);
  if (e[0] & KMC_DERR_TIMEOUT) return fail(h, KMC_ERR_TIMEOUT, "%s: a device-side wait exceeded its limit", where);
  if (e[0] & KMC_DERR_BOUNDS) return fail(h, KMC_ERR_STATE, "%s: an index failed its bounds check (checked build)", where);
  return fail(h, KMC_ERR_STATE, "%s: device error flags 0x%x", where, e[0]);
}

// after_copies: order the call's work after a pending asynchronous output copy
// (every call but kmc_step and kmc_fmm_accept_event, which write neither the
// masks nor the dU the copy reads)
static int guard(kmc_fmm* h, bool after_copies = true) {
  if (!h) return KMC_ERR_ARG;
  if (h->broken) return fail(h, KMC_ERR_STATE, "handle unusable after an earlier error: %s", h->msg);
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(h, KMC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  if (after_copies && h->copy_pending) {
    e = cudaStreamWaitEvent(h->stream, h->ev_copied, 0);
    if (e != cudaSuccess) return fail(h, KMC_ERR_CUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
  }
  return KMC_OK;
}

// ------------------------------------------------------------------ full FMM
static int full_fmm(kmc_fmm* h) {
  const Geo& g = h->g;
  const Dev& d = h->d;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(d.Mt, 0, sizeof(double2) * g.ncell_total * g.P, s));
  fmm_p2m(g, d, s);
  fmm_m2m(g, d, s);
  {  // M2L scratch (per-level translation matrices), stream-ordered, released after use
    void* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, fmm_m2l_scratch_bytes(g), s));
    fmm_m2l(g, d, scratch, s);
    CK(cudaFreeAsync(scratch, s));
  }
  fmm_far_field(g, d, s);
  fmm_shadow_all(g, d, s);
  fmm_self_and_dipole(g, d, s);
  if (g.near_cache) kmc_near_fill(g, d, h->prec, s);  // near-field sums of every site, afresh
  CKLAUNCH();
  h->peff_valid = false;
  h->rates_valid = false;
  return KMC_OK;
}

static int refresh_peff(kmc_fmm* h) {
  if (h->peff_valid) return KMC_OK;
  fmm_downward(h->g, h->d, h->prec, h->stream);
  CKLAUNCH();
  h->peff_valid = true;
  return KMC_OK;
}

// potential at every charge (own term excluded) into d.phi_old
static int compute_phi_old(kmc_fmm* h) {
  int r = refresh_peff(h);
  if (r) return r;
  if (h->g.E > 0) {
    kmc_propose_lattice(h->g, h->d, h->prec, h->stream);
    kmc_finalize_rates(h->g, h->d, h->prec, h->stream);
    if (h->prec == 1) kmc_widen(h->d.phi_old32, h->d.phi_old, h->g.n, h->stream);
    h->rates_valid = true;
  } else {
    kmc_eval_points(h->g, h->d, h->prec, h->g.n, h->d.pos, h->iota, h->d.phi_old, h->stream);
  }
  CKLAUNCH();
  return KMC_OK;
}

static int compute_energy(kmc_fmm* h) {
  int r = compute_phi_old(h);
  if (r) return r;
  kmc_energy_reduce(h->g, h->d, h->stream);
  if (h->g.dirichlet) kmc_dirichlet_energy(h->g, h->d, h->stream);  // U = U_mirrored / 2 + field term
  CKLAUNCH();
  return KMC_OK;
}

// ------------------------------------------------------------------ C ABI
// The dynamic shared-memory limit of a kernel is a per-device attribute shared
// by every handle in the process.  Handles of different shapes need different
// sizes, so the limit only ever grows: a smaller later handle must not lower it
// below what an earlier one launches with (a launch above the limit fails, and
// inside a stream capture that failure invalidates the whole capture).
void raise_dynamic_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set[std::make_pair(fn, dev)];
  if (bytes <= cur) return;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess) cur = bytes;
}

extern "C" {

void kmc_opts_default(kmc_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = KMC_PREC_FP64;
  o->lattice_edge = 0;
  o->lattice_h = 1.0;
  o->kT = 1.0;
  o->stream = nullptr;
  o->mem = KMC_MEM_HOST;
  o->device = 0;
  o->leaf_capacity = 0;
  o->m2l = KMC_M2L_TENSOR;
  o->hops = KMC_HOPS_6;
  o->bc = KMC_BC_PERIODIC;
  o->field_z = 0.0;
  o->near_cache = 0;
  o->l2l = KMC_L2L_TENSOR;
}

const char* kmc_last_error(kmc_handle h) { return h ? h->msg : g_static_msg; }

void kmc_fmm_destroy(kmc_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->cstream) {
    cudaStreamSynchronize(h->cstream);
    cudaStreamDestroy(h->cstream);
    cudaEventDestroy(h->ev_ready);
    cudaEventDestroy(h->ev_copied);
  }
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

static int init_impl(kmc_fmm* h, int64_t n, const double* positions, const double* charges, double box, int levels,
                     int order) {
  Geo& g = h->g;
  Dev& d = h->d;
  memset(&g, 0, sizeof(g));
  memset(&d, 0, sizeof(d));
  g.L = levels;
  g.p = order;
  g.P = ncoef(order);
  g.P2 = ncoef(2 * order);
  g.nL = 1 << (levels - 1);
  g.n = n;
  g.ML = (int64_t)g.nL * g.nL * g.nL;
  g.a = box;
  g.w = box / g.nL;
  g.inv_a = 1.0 / box;
  g.kT = 1.0;
  g.prec = h->prec;
  int64_t off = 0;
  for (int l = 1; l <= levels; l++) {
    g.cell_off[l] = off;
    off += (int64_t)1 << (3 * (l - 1));
  }
  g.cell_off[levels + 1] = off;
  g.ncell_total = off;
  return KMC_OK;
}

int kmc_fmm_init(kmc_handle* out, int64_t n, const double* positions, const double* charges, double box, int levels,
                 int order, const kmc_opts* opts) {
  KMC_TRACE("kmc_fmm_init");
  if (!out) return KMC_ERR_ARG;
  *out = nullptr;
  kmc_opts o;
  if (opts) o = *opts;
  else kmc_opts_default(&o);
  kmc_fmm* h = new kmc_fmm();
  memset(h->msg, 0, sizeof(h->msg));
  h->broken = false;
  h->prec = o.precision == KMC_PREC_MIXED ? 1 : 0;
  h->mem = o.mem;
  h->device = o.device;
  h->stream = (cudaStream_t)o.stream;
  h->graph = nullptr;
  h->graph_steps = 0;
  h->gen_cap = 0;
  h->run_cap = 0;
  h->run_gen = 0;
  h->phi_save = nullptr;
  *out = h;
  // ---- host-side argument checks
  if (n < 2) return fail(h, KMC_ERR_ARG, "need at least 2 charges (n = %lld)", (long long)n);
  if (n > 0x7fffffffLL / (o.hops == KMC_HOPS_14 ? KMC_MAXHOP : KMC_NHOP))
    return fail(h, KMC_ERR_ARG, "too many charges (n = %lld)", (long long)n);
  if (levels < 3 || levels > KMC_MAXL) return fail(h, KMC_ERR_ARG, "levels must be in [3, %d] (got %d)", KMC_MAXL, levels);
  if (order < 1 || order > KMC_MAXP) return fail(h, KMC_ERR_ARG, "order must be in [1, %d] (got %d)", KMC_MAXP, order);
  if (!(box > 0.0) || !isfinite(box)) return fail(h, KMC_ERR_ARG, "box must be positive and finite");
  if (!positions || !charges) return fail(h, KMC_ERR_ARG, "positions and charges are required");
  if (o.precision != KMC_PREC_FP64 && o.precision != KMC_PREC_MIXED) return fail(h, KMC_ERR_ARG, "unknown precision");
  if (o.mem != KMC_MEM_HOST && o.mem != KMC_MEM_DEVICE) return fail(h, KMC_ERR_ARG, "unknown memory kind");
  if (!(o.kT > 0.0)) return fail(h, KMC_ERR_ARG, "kT must be positive");
  if (o.m2l != KMC_M2L_TENSOR && o.m2l != KMC_M2L_FP64 && o.m2l != KMC_M2L_TENSOR_SYNC) return fail(h, KMC_ERR_ARG, "unknown M2L arithmetic");
  if (o.hops != KMC_HOPS_6 && o.hops != KMC_HOPS_14) return fail(h, KMC_ERR_ARG, "unknown hop set");
  if (o.bc != KMC_BC_PERIODIC && o.bc != KMC_BC_FREE && o.bc != KMC_BC_DIRICHLET_Z)
    return fail(h, KMC_ERR_ARG, "unknown boundary conditions");
  if (!isfinite(o.field_z)) return fail(h, KMC_ERR_ARG, "field_z must be finite");
  if (o.near_cache != 0 && o.near_cache != 1) return fail(h, KMC_ERR_ARG, "near_cache must be 0 or 1");
  if (o.l2l != KMC_L2L_TENSOR && o.l2l != KMC_L2L_CUDA) return fail(h, KMC_ERR_ARG, "unknown downward-pass arithmetic");
  if (o.near_cache && o.lattice_edge <= 0) return fail(h, KMC_ERR_ARG, "near_cache needs lattice mode");
  // input arrays: read in the caller's memory kind, except with Dirichlet walls,
  // where the library appends the mirrors on the host first
  bool dev_in = h->mem == KMC_MEM_DEVICE;
  std::vector<double> dir_pos, dir_q;
  const int64_t nphys = n;
  if (o.bc == KMC_BC_DIRICHLET_Z) {
    if (o.lattice_edge <= 0 || o.lattice_edge % 2)
      return fail(h, KMC_ERR_ARG, "Dirichlet walls need lattice mode with an even lattice edge");
    if (n > 0x7fffffffLL / (2 * (o.hops == KMC_HOPS_14 ? KMC_MAXHOP : KMC_NHOP)))
      return fail(h, KMC_ERR_ARG, "too many charges (n = %lld)", (long long)n);
    dir_pos.resize(6 * n);
    dir_q.resize(2 * n);
    if (dev_in) {
      CK(cudaMemcpy(dir_pos.data(), positions, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(dir_q.data(), charges, sizeof(double) * n, cudaMemcpyDeviceToHost));
    } else {
      memcpy(dir_pos.data(), positions, sizeof(double) * 3 * n);
      memcpy(dir_q.data(), charges, sizeof(double) * n);
    }
    for (int64_t i = 0; i < n; i++) {
      const double z = dir_pos[3 * i + 2];
      if (!(z >= 0.0 && z < 0.5 * box))
        return fail(h, KMC_ERR_ARG, "Dirichlet walls: charge %lld lies above the mirror plane z = box/2", (long long)i);
      dir_pos[3 * (n + i)] = dir_pos[3 * i];
      dir_pos[3 * (n + i) + 1] = dir_pos[3 * i + 1];
      dir_pos[3 * (n + i) + 2] = box - z;
      dir_q[n + i] = -dir_q[i];
    }
    n *= 2;
    positions = dir_pos.data();
    charges = dir_q.data();
    dev_in = false;
  }
  int r = init_impl(h, n, positions, charges, box, levels, order);
  if (r) return r;
  Geo& g = h->g;
  g.kT = o.kT;
  g.m2l = o.m2l;
  g.nhop = o.hops == KMC_HOPS_14 ? KMC_MAXHOP : KMC_NHOP;
  g.bc = o.bc == KMC_BC_FREE ? 1 : 0;
  g.dirichlet = o.bc == KMC_BC_DIRICHLET_Z ? 1 : 0;
  g.nphys = nphys;
  g.field_z = g.dirichlet ? o.field_z : 0.0;
  g.dipc = g.bc ? 0.0 : 4.0 * M_PI / (3.0 * box * box * box);
  if (o.lattice_edge > 0) {
    int E = o.lattice_edge;
    if (E % g.nL != 0) return fail(h, KMC_ERR_ARG, "lattice edge %d is not a multiple of 2^(levels-1) = %d", E, g.nL);
    if (!(o.lattice_h > 0.0)) return fail(h, KMC_ERR_ARG, "lattice spacing must be positive");
    if (fabs(E * o.lattice_h - box) > 1e-12 * box)
      return fail(h, KMC_ERR_ARG, "box (%g) must equal lattice_edge * lattice_h (%g)", box, E * o.lattice_h);
    g.E = E;
    g.h = o.lattice_h;
    g.W = E / g.nL;
    // the propose kernel keeps a leaf's evaluation points and a source chunk in shared memory
    if (g.W < 1 || g.W > 12) return fail(h, KMC_ERR_ARG, "lattice sites per leaf side must be in [1, 12] (got %d)", g.W);
    if ((int64_t)E * E * E > 0x7fffffffLL) return fail(h, KMC_ERR_ARG, "lattice too large");
    if (n > (int64_t)E * E * E) return fail(h, KMC_ERR_ARG, "more charges than sites");
    g.cap = g.W * g.W * g.W;
    g.near_cache = o.near_cache;
    g.l2l = o.l2l;
  } else {
    g.E = 0;
    g.h = 1.0;
    g.W = 0;
  }
  cudaError_t ce = cudaSetDevice(h->device);
  if (ce != cudaSuccess) return fail(h, KMC_ERR_CUDA, "cudaSetDevice(%d): %s", h->device, cudaGetErrorString(ce));
  // charges to host for the neutrality check
  std::vector<double> qh(n);
  if (dev_in) {
    CK(cudaMemcpy(qh.data(), charges, sizeof(double) * n, cudaMemcpyDeviceToHost));
  } else {
    memcpy(qh.data(), charges, sizeof(double) * n);
  }
  double qs = 0.0, qa = 0.0;
  for (int64_t i = 0; i < n; i++) {
    if (!isfinite(qh[i])) return fail(h, KMC_ERR_ARG, "charge %lld is not finite", (long long)i);
    qs += qh[i];
    qa += fabs(qh[i]);
    g.qmax = fmax(g.qmax, fabs(qh[i]));
  }
  if (!g.bc && fabs(qs) > 1e-12 * qa) return fail(h, KMC_ERR_NOT_NEUTRAL, "sum of charges %.3e is not zero", qs);
  if (g.near_cache) {
    // fixed-point exponent of the cached near-field sums: 2^k bound < 2^61, bound = max|q| x
    // (27 leaves x cap charges) at the smallest separation, one site (lattice units)
    const double bound = fmax(g.qmax, 1e-300) * 27.0 * g.cap;
    g.near_ks = 61 - (ilogb(bound) + 1);
  }
  // off-lattice capacity from the initial occupancy
  std::vector<double> ph;
  if (g.E == 0) {
    ph.resize(3 * n);
    if (h->mem == KMC_MEM_DEVICE) {
      CK(cudaMemcpy(ph.data(), positions, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    } else {
      memcpy(ph.data(), positions, sizeof(double) * 3 * n);
    }
    std::vector<int32_t> cnt(g.ML, 0);
    int mx = 0;
    for (int64_t i = 0; i < n; i++) {
      int c[3];
      for (int k = 0; k < 3; k++) {
        double x = ph[3 * i + k];
        if (!isfinite(x) || x < 0.0 || x >= box) return fail(h, KMC_ERR_ARG, "position of charge %lld outside [0, box)", (long long)i);
        c[k] = (int)floor(x * ((double)g.nL * g.inv_a));
        if (c[k] >= g.nL) c[k] = g.nL - 1;
        if (c[k] < 0) c[k] = 0;
      }
      int64_t lf = c[0] + (int64_t)g.nL * (c[1] + (int64_t)g.nL * c[2]);
      mx = cnt[lf] + 1 > mx ? cnt[lf] + 1 : mx;
      cnt[lf]++;
    }
    int cap = o.leaf_capacity > 0 ? o.leaf_capacity : 2 * mx + 32;
    if (cap < mx) return fail(h, KMC_ERR_CAPACITY, "leaf capacity %d below initial occupancy %d", cap, mx);
    g.cap = cap;
  }
  // ---- allocations
  Dev& d = h->d;
  const int64_t nslot = g.ML * g.cap;
  ALLOC(d.q, sizeof(double) * n);
  ALLOC(d.pos, sizeof(double) * 3 * n);
  ALLOC(d.site, sizeof(int32_t) * n);
  ALLOC(d.slot_of, sizeof(int32_t) * n);
  ALLOC(d.cnt, sizeof(int32_t) * g.ML);
  ALLOC(d.uid, sizeof(int32_t) * nslot);
  ALLOC(d.spos64, sizeof(double4_32a) * nslot);
  ALLOC(d.spos32, sizeof(float4) * nslot);
  if (g.E > 0) {
    ALLOC(d.isq, sizeof(double) * KMC_ISQ_N);
  }
  if (g.near_cache) ALLOC(d.nearfx, sizeof(long long) * (size_t)g.ML * (size_t)g.cap);
  ALLOC(d.Mt, sizeof(double2) * g.ncell_total * g.P);
  ALLOC(d.Psi, sizeof(double2) * g.ncell_total * g.P);
  ALLOC(d.Peff, (h->prec == 0 ? sizeof(double2) : sizeof(float2)) * g.ncell_total * g.P);
  ALLOC(d.Itab, sizeof(double2) * (size_t)(g.L + 1) * 343 * g.P2);
  ALLOC(d.Itab2, sizeof(double2) * (size_t)KMC_TOP_NOFF * g.P2);
  ALLOC(d.S, sizeof(double2) * g.P2);
  ALLOC(d.Rch, sizeof(double2) * (size_t)(g.L + 1) * 8 * g.P);
  ALLOC(d.Rcoarse, sizeof(double2) * (size_t)KMC_COARSE_TABLES * g.P);
  ALLOC(d.selfc, sizeof(double) * KMC_MAXHOP);
  if (g.dirichlet) {
    ALLOC(d.dirA, sizeof(double) * (g.E / 2));
    ALLOC(d.dirB, sizeof(double) * (g.E / 2) * g.nhop);
  }
  ALLOC(d.dip, sizeof(double) * 3);
  ALLOC(d.dip_part, sizeof(double) * 3 * KMC_DIP_BLOCKS);
  ALLOC(d.fdip, sizeof(float) * 4);
  ALLOC(d.U, sizeof(double));
  if (h->prec == 1) {
    ALLOC(d.q32, sizeof(float) * n);
    ALLOC(d.selfc32, sizeof(float) * KMC_MAXHOP);
    ALLOC(d.Psi32, sizeof(float2) * g.ncell_total * g.P);
    ALLOC(d.Rch32, sizeof(float2) * (size_t)(g.L + 1) * 8 * g.P);
    ALLOC(d.Rcoarse32, sizeof(float2) * (size_t)KMC_COARSE_TABLES * g.P);
    if (g.dirichlet) {
      ALLOC(d.dirA32, sizeof(float) * (g.E / 2));
      ALLOC(d.dirB32, sizeof(float) * (g.E / 2) * g.nhop);
    }
    ALLOC(d.phi_old32, sizeof(float) * n);
    ALLOC(d.phi_new32, sizeof(float) * g.nhop * n);
    ALLOC(d.dU32, sizeof(float) * g.nhop * n);
    if (fmm_l2l_tc_first(g)) {
      ALLOC(d.l2lT, sizeof(float) * fmm_l2l_tc_table_floats(g));
      ALLOC(d.l2lA, sizeof(float) * fmm_l2l_tc_split_floats(g));
      CK(cudaMemset(d.l2lA, 0, sizeof(float) * fmm_l2l_tc_split_floats(g)));  // the padding stays zero
    }
  }
  ALLOC(d.phi_old, sizeof(double) * n);
  ALLOC(d.phi_new, sizeof(double) * g.nhop * n);
  ALLOC(d.mask, sizeof(uint8_t) * g.nhop * n);
  ALLOC(d.dU, sizeof(double) * g.nhop * n);
  ALLOC(d.rate, sizeof(double) * g.nhop * n);
  ALLOC(d.bsum, sizeof(double) * ((n + KMC_FIN_PARTICLES - 1) / KMC_FIN_PARTICLES + 1));
  ALLOC(d.event, sizeof(int64_t) * 2);
  ALLOC(d.dtq, sizeof(double) * 2);
  ALLOC(d.move, sizeof(MoveRec));
  ALLOC(d.acc_scratch, sizeof(double2) * (size_t)kmc_coarse_slots() * g.P);
  ALLOC(d.err, sizeof(int) * 4);
  ALLOC(d.uni_small, sizeof(double) * 2);
  ALLOC(d.stepc, sizeof(int) * 2);
  ALLOC(h->drift2, sizeof(double) * 2);
  ALLOC(h->iota, sizeof(int32_t) * n);
  {
    const int nr = 13, nk = 19;
    size_t terms = (size_t)(nr * nr * nr + nk * nk * nk) * g.P2 * sizeof(double2);
    ALLOC(d.scratch, terms);
  }
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(d.err, 0, sizeof(int) * 4, s));
  if (g.E > 0) {  // correctly rounded 1/sqrt(n) of the squared lattice distances (FP64 near field)
    std::vector<double> isq(KMC_ISQ_N, 0.0);
    for (int k = 1; k < KMC_ISQ_N; k++) isq[k] = 1.0 / sqrt((double)k);
    CK(cudaMemcpy(d.isq, isq.data(), sizeof(double) * KMC_ISQ_N, cudaMemcpyHostToDevice));
  }
  CK(cudaMemsetAsync(d.uid, 0xff, sizeof(int32_t) * nslot, s));
  CK(cudaMemsetAsync(d.mask, 0, (size_t)g.nhop * n, s));
  CK(cudaMemsetAsync(d.Psi, 0, sizeof(double2) * g.ncell_total * g.P, s));
  const cudaMemcpyKind ik = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(d.q, charges, sizeof(double) * n, ik, s));
  CK(cudaMemcpyAsync(d.pos, positions, sizeof(double) * 3 * n, ik, s));
  if (h->prec == 1) {
    std::vector<float> q32(n);
    for (int64_t i = 0; i < n; i++) q32[i] = (float)qh[i];
    CK(cudaMemcpyAsync(d.q32, q32.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  {
    std::vector<int32_t> io(n);
    for (int64_t i = 0; i < n; i++) io[i] = (int32_t)i;
    CK(cudaMemcpyAsync(h->iota, io.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  fmm_upload_constants(order);
  kmc_upload_constants(order);
  kmc_prepare(g, h->prec);
  fmm_prepare(g, h->prec);
  CKLAUNCH();
  kmc_validate(g, d, s);
  CKLAUNCH();
  r = check_flags(h, "init");
  if (r) return r;
  if (g.E > 0) {  // two charges on one site?
    std::vector<int32_t> sh(n);
    CK(cudaMemcpy(sh.data(), d.site, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> occ((size_t)g.E * g.E * g.E, 0);
    for (int64_t i = 0; i < n; i++) {
      if (occ[sh[i]]) return fail(h, KMC_ERR_ARG, "two charges on lattice site %d", sh[i]);
      occ[sh[i]] = 1;
    }
  }
  fmm_bin(g, d, s);
  CKLAUNCH();
  r = check_flags(h, "init binning");
  if (r) return r;
  fmm_itab(g, d, s);
  fmm_child_tables(g, d, s);
  fmm_l2l_tc_tables(g, d, s);
  fmm_lattice_sums(g, d, s);
  if (g.dirichlet) fmm_dirichlet_tables(g, d, s);
  CKLAUNCH();
  r = full_fmm(h);
  if (r) return r;
  r = compute_energy(h);
  if (r) return r;
  return check_flags(h, "init");
}

int kmc_fmm_energy(kmc_handle h, double* U) {
  KMC_TRACE("kmc_fmm_energy");
  int r = guard(h);
  if (r) return r;
  if (!U) return fail(h, KMC_ERR_ARG, "U is NULL");
  CK(cudaMemcpyAsync(U, h->d.U, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return KMC_OK;
}

static int propose_lattice_impl(kmc_fmm* h, uint8_t* mask, double* dU, float* dU32) {
  int r = guard(h);
  if (r) return r;
  if (h->g.E <= 0) return fail(h, KMC_ERR_STATE, "kmc_fmm_propose_lattice needs lattice mode");
  if (dU32 && h->prec != 1) return fail(h, KMC_ERR_STATE, "FP32 dU needs the mixed-precision form");
  r = refresh_peff(h);
  if (r) return r;
  kmc_propose_lattice(h->g, h->d, h->prec, h->stream);
  kmc_finalize_rates(h->g, h->d, h->prec, h->stream);
  CKLAUNCH();
  h->rates_valid = true;
  const int64_t m = (int64_t)h->g.nhop * h->g.nphys;  // the caller's charges (not the mirrors)
  if (mask) CK(cudaMemcpyAsync(mask, h->d.mask, m, out_kind(h), h->stream));
  if (dU) {
    if (h->prec == 1) kmc_widen(h->d.dU32, h->d.dU, m, h->stream);
    CK(cudaMemcpyAsync(dU, h->d.dU, sizeof(double) * m, out_kind(h), h->stream));
  }
  if (dU32) CK(cudaMemcpyAsync(dU32, h->d.dU32, sizeof(float) * m, out_kind(h), h->stream));
  return check_flags(h, "propose_lattice");
}

int kmc_fmm_propose_lattice(kmc_handle h, uint8_t* mask, double* dU) {
  KMC_TRACE("kmc_fmm_propose_lattice");
  return propose_lattice_impl(h, mask, dU, nullptr);
}

int kmc_fmm_propose_lattice_f32(kmc_handle h, uint8_t* mask, float* dU) {
  KMC_TRACE("kmc_fmm_propose_lattice_f32");
  return propose_lattice_impl(h, mask, nullptr, dU);
}

int kmc_fmm_propose_lattice_async(kmc_handle h, uint8_t* mask, float* dU) {
  KMC_TRACE("kmc_fmm_propose_lattice_async");
  int r = guard(h, false);  // the downward pass runs beside the previous call's copies
  if (r) return r;
  if (h->g.E <= 0) return fail(h, KMC_ERR_STATE, "kmc_fmm_propose_lattice_async needs lattice mode");
  if (h->prec != 1) return fail(h, KMC_ERR_STATE, "FP32 dU needs the mixed-precision form");
  if (!h->cstream) {
    CK(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_ready, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
  }
  r = refresh_peff(h);
  if (r) return r;
  if (h->copy_pending) CK(cudaStreamWaitEvent(h->stream, h->ev_copied, 0));  // before masks and dU are rewritten
  kmc_propose_lattice(h->g, h->d, h->prec, h->stream);
  kmc_finalize_rates(h->g, h->d, h->prec, h->stream);
  CKLAUNCH();
  h->rates_valid = true;
  const int64_t m = (int64_t)h->g.nhop * h->g.nphys;
  CK(cudaEventRecord(h->ev_ready, h->stream));
  CK(cudaStreamWaitEvent(h->cstream, h->ev_ready, 0));
  if (mask) CK(cudaMemcpyAsync(mask, h->d.mask, m, out_kind(h), h->cstream));
  if (dU) CK(cudaMemcpyAsync(dU, h->d.dU32, sizeof(float) * m, out_kind(h), h->cstream));
  CK(cudaEventRecord(h->ev_copied, h->cstream));
  h->copy_pending = true;
  return KMC_OK;  // the kernels' error flags are read by the next call that synchronises
}

int kmc_fmm_outputs_wait(kmc_handle h) {
  KMC_TRACE("kmc_fmm_outputs_wait");
  int r = guard(h, false);
  if (r) return r;
  if (h->copy_pending) {
    CK(cudaEventSynchronize(h->ev_copied));
    h->copy_pending = false;
  }
  return check_flags(h, "outputs_wait");
}

static int ensure_gen(kmc_fmm* h, int64_t m) {
  if ((size_t)m <= h->gen_cap) return KMC_OK;
  size_t c = (size_t)m < 1024 ? 1024 : (size_t)m;
  ALLOC(h->gen_part, sizeof(int32_t) * c);
  ALLOC(h->gen_tgt, sizeof(double) * 3 * c);
  ALLOC(h->gen_old, sizeof(double) * 3 * c);
  ALLOC(h->gen_pn, sizeof(double) * c);
  ALLOC(h->gen_po, sizeof(double) * c);
  ALLOC(h->gen_dv, sizeof(double) * 3 * c);
  ALLOC(h->gen_du, sizeof(double) * c);
  ALLOC(h->gen_mask, sizeof(uint8_t) * c);
  h->gen_cap = c;
  return KMC_OK;
}

// stage general proposals on the device: inputs copied (host memory) or used
// in place (device memory), then wrapped / gathered by a kernel.
static int stage_general(kmc_fmm* h, int64_t m, const int32_t* particle, const double* target, const uint8_t* mask,
                         bool host_inputs) {
  int r = ensure_gen(h, m);
  if (r) return r;
  cudaStream_t s = h->stream;
  const int32_t* pd = particle;
  const double* td = target;
  const uint8_t* md = mask;
  if (host_inputs) {
    CK(cudaMemcpyAsync(h->gen_part, particle, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->gen_dv, target, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, s));
    pd = h->gen_part;
    td = h->gen_dv;
    if (mask) {
      CK(cudaMemcpyAsync(h->gen_mask, mask, m, cudaMemcpyHostToDevice, s));
      md = h->gen_mask;
    }
  } else {
    CK(cudaMemcpyAsync(h->gen_part, particle, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    pd = h->gen_part;
  }
  // targets are read before dv is written (same thread, same index), so the
  // dv buffer may double as the staging area for host targets
  kmc_stage_general(h->g, h->d, m, pd, td, md, h->gen_tgt, h->gen_old, h->gen_dv, h->gen_mask, s);
  CKLAUNCH();
  return KMC_OK;
}

static int general_du(kmc_fmm* h, int64_t m) {
  int r = refresh_peff(h);
  if (r) return r;
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  // Phi at the target includes every charge (the moving one too: its old
  // position's contribution is removed by the self term C(d)); Phi at the old
  // position omits only the moving charge itself.
  kmc_eval_points(g, h->d, h->prec, m, h->gen_tgt, nullptr, h->gen_pn, s);
  kmc_eval_points(g, h->d, h->prec, m, h->gen_old, h->gen_part, h->gen_po, s);
  fmm_selfcorr_list(g, h->d, m, h->gen_dv, h->gen_du, s);
  kmc_assemble_general(g, h->d, m, h->gen_part, h->gen_tgt, h->gen_mask, h->gen_pn, h->gen_po, h->gen_du, s);
  CKLAUNCH();
  return KMC_OK;
}

int kmc_fmm_propose(kmc_handle h, int64_t m, const int32_t* particle, const double* target, const uint8_t* mask,
                    double* dU) {
  KMC_TRACE("kmc_fmm_propose");
  int r = guard(h);
  if (r) return r;
  if (h->g.dirichlet)
    return fail(h, KMC_ERR_STATE, "general proposals and moves are not available with Dirichlet walls");
  if (m < 0) return fail(h, KMC_ERR_ARG, "negative proposal count");
  if (m == 0) return KMC_OK;
  if (!particle || !target || !dU) return fail(h, KMC_ERR_ARG, "particle, target and dU are required");
  r = stage_general(h, m, particle, target, mask, h->mem == KMC_MEM_HOST);
  if (r) return r;
  r = check_flags(h, "propose");
  if (r) return r;
  r = general_du(h, m);
  if (r) return r;
  CK(cudaMemcpyAsync(dU, h->gen_du, sizeof(double) * m, out_kind(h), h->stream));
  return check_flags(h, "propose");
}

static int accept_general(kmc_fmm* h, int32_t particle, const double* tgt_host, double* dU_out) {
  const Geo& g = h->g;
  if (particle < 0 || particle >= g.n) return fail(h, KMC_ERR_ARG, "particle index out of range");
  int r = stage_general(h, 1, &particle, tgt_host, nullptr, true);
  if (r) return r;
  r = check_flags(h, "accept");
  if (r) return r;
  double th[3];
  CK(cudaMemcpy(th, h->gen_tgt, sizeof(th), cudaMemcpyDeviceToHost));
  MoveRec mv;
  memset(&mv, 0, sizeof(mv));
  mv.valid = 1;
  mv.i = particle;
  mv.site_old = -1;
  mv.site_new = -1;
  double old[3];
  CK(cudaMemcpy(old, h->gen_old, sizeof(old), cudaMemcpyDeviceToHost));
  double qv;
  CK(cudaMemcpy(&qv, h->d.q + particle, sizeof(double), cudaMemcpyDeviceToHost));
  mv.q = qv;
  for (int k = 0; k < 3; k++) {
    mv.r[k] = old[k];
    mv.rn[k] = th[k];
  }
  if (g.E > 0) {
    int ix[3], ox[3];
    for (int k = 0; k < 3; k++) {
      double f = mv.rn[k] / g.h - 0.5;
      double rf = rint(f);
      if (fabs(f - rf) > 1e-9) return fail(h, KMC_ERR_ARG, "accept: target is not a lattice site");
      ix[k] = ((int)rf % g.E + g.E) % g.E;
      mv.rn[k] = (ix[k] + 0.5) * g.h;
      ox[k] = (int)rint(mv.r[k] / g.h - 0.5);
    }
    mv.site_new = ix[0] + g.E * (ix[1] + g.E * ix[2]);
    mv.site_old = ox[0] + g.E * (ox[1] + g.E * ox[2]);
    CK(cudaMemcpy(h->gen_tgt, mv.rn, sizeof(mv.rn), cudaMemcpyHostToDevice));
  }
  r = general_du(h, 1);
  if (r) return r;
  double du;
  CK(cudaMemcpyAsync(&du, h->gen_du, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  r = check_flags(h, "accept");
  if (r) return r;
  if (!isfinite(du)) return fail(h, KMC_ERR_ARG, "accept: singular move");
  mv.dU = du;
  CK(cudaMemcpyAsync(h->d.move, &mv, sizeof(mv), cudaMemcpyHostToDevice, h->stream));
  kmc_accept_apply(g, h->d, h->stream);
  CKLAUNCH();
  h->peff_valid = false;
  h->rates_valid = false;
  r = check_flags(h, "accept");
  if (r) return r;
  if (dU_out) *dU_out = du;
  return KMC_OK;
}

int kmc_fmm_accept(kmc_handle h, int32_t particle, const double target[3], double* dU_accepted) {
  KMC_TRACE("kmc_fmm_accept");
  int r = guard(h);
  if (r) return r;
  if (h->g.dirichlet)
    return fail(h, KMC_ERR_STATE, "general proposals and moves are not available with Dirichlet walls");
  if (!target) return fail(h, KMC_ERR_ARG, "target is NULL");
  double t[3];
  if (h->mem == KMC_MEM_DEVICE) {
    CK(cudaMemcpy(t, target, sizeof(t), cudaMemcpyDeviceToHost));
  } else {
    memcpy(t, target, sizeof(t));
  }
  return accept_general(h, particle, t, dU_accepted);
}

int kmc_fmm_accept_event(kmc_handle h, int64_t event, double* dU_accepted) {
  KMC_TRACE("kmc_fmm_accept_event");
  int r = guard(h, false);
  if (r) return r;
  const Geo& g = h->g;
  if (g.E <= 0) return fail(h, KMC_ERR_STATE, "kmc_fmm_accept_event needs lattice mode");
  if (event < 0 || event >= (int64_t)g.nhop * g.nphys) return fail(h, KMC_ERR_ARG, "event index out of range");
  // the device accept path: the move record built from the event on the device (with grounded
  // walls, twice: the charge and its mirror); without walls it needs the current proposal's
  // rates, else the general path below validates and applies the move
  if (g.dirichlet || h->rates_valid) {
    cudaStream_t s = h->stream;
    if (!h->rates_valid) {
      if (h->copy_pending) CK(cudaStreamWaitEvent(s, h->ev_copied, 0));  // a proposal rewrites masks and dU
      r = refresh_peff(h);
      if (r) return r;
      kmc_propose_lattice(g, h->d, h->prec, s);
      kmc_finalize_rates(g, h->d, h->prec, s);
      CKLAUNCH();
      h->rates_valid = true;
    }
    uint8_t mk = 0;
    float f = 0.f;
    double du = 0.0;
    CK(cudaMemcpyAsync(&mk, h->d.mask + event, 1, cudaMemcpyDeviceToHost, s));
    if (h->prec == 1) CK(cudaMemcpyAsync(&f, h->d.dU32 + event, sizeof(f), cudaMemcpyDeviceToHost, s));
    else CK(cudaMemcpyAsync(&du, h->d.dU + event, sizeof(du), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!mk)
      return fail(h, KMC_ERR_ARG, "event %lld is masked (occupied target%s)", (long long)event,
                  g.dirichlet ? " or a wall" : "");
    if (h->prec == 1) du = f;
    CK(cudaMemcpyAsync(h->d.event, &event, sizeof(event), cudaMemcpyHostToDevice, s));
    kmc_accept_from_event(g, h->d, s);
    kmc_accept_apply(g, h->d, s);
    if (g.dirichlet) {
      kmc_mirror_move(g, h->d, s);
      kmc_accept_apply(g, h->d, s);
    }
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
    h->peff_valid = false;
    h->rates_valid = false;
    if (dU_accepted) *dU_accepted = du;
    return check_flags(h, "accept_event");
  }
  int32_t i = (int32_t)(event / g.nhop);
  int k = (int)(event % g.nhop);
  double p[3];
  CK(cudaMemcpy(p, h->d.pos + 3 * (int64_t)i, sizeof(p), cudaMemcpyDeviceToHost));
  double t[3];
  for (int c = 0; c < 3; c++) t[c] = p[c] + hop_c(k, c) * g.h;
  return accept_general(h, i, t, dU_accepted);
}

int kmc_step(kmc_handle h, const double* rates, double zeta, double xi, int64_t* event, double* dt, double* Q) {
  KMC_TRACE("kmc_step");
  int r = guard(h, false);
  if (r) return r;
  if (!(zeta > 0.0 && zeta <= 1.0 && xi > 0.0 && xi <= 1.0))
    return fail(h, KMC_ERR_ARG, "zeta and xi must lie in (0, 1]");
  cudaStream_t s = h->stream;
  if (rates && h->g.dirichlet) return fail(h, KMC_ERR_STATE, "kmc_step with Dirichlet walls takes the device rates");
  if (rates) {
    CK(cudaMemcpyAsync(h->d.rate, rates, sizeof(double) * h->g.nhop * h->g.n, in_kind(h), s));
    kmc_rate_bsum(h->g, h->d, s);
    CKLAUNCH();
  } else if (!h->rates_valid) {
    return fail(h, KMC_ERR_STATE, "kmc_step without rates needs a kmc_fmm_propose_lattice after the last accept");
  }
  double u[2] = {zeta, xi};
  CK(cudaMemcpyAsync(h->d.uni_small, u, sizeof(u), cudaMemcpyHostToDevice, s));
  kmc_select(h->g, h->d, 0, s);
  CKLAUNCH();
  int64_t ev;
  double dq[2];
  CK(cudaMemcpyAsync(&ev, h->d.event, sizeof(ev), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(dq, h->d.dtq, sizeof(dq), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (rates) h->rates_valid = false;  // device rates now hold the caller's values
  if (event) *event = ev;
  if (dt) *dt = dq[0];
  if (Q) *Q = dq[1];
  return KMC_OK;
}

// one device-driven step: downward pass, propose, rates, select, record, accept
static void enqueue_step(kmc_fmm* h) {
  const Geo& g = h->g;
  const Dev& d = h->d;
  cudaStream_t s = h->stream;
  fmm_downward(g, d, h->prec, s);
  kmc_propose_lattice(g, d, h->prec, s);
  kmc_finalize_rates(g, d, h->prec, s);
  kmc_select(g, d, 1, s);
  kmc_record(g, d, s);
  kmc_accept_from_event(g, d, s);
  kmc_accept_apply(g, d, s);
  if (g.dirichlet) {  // the mirror moves with the charge
    kmc_mirror_move(g, d, s);
    kmc_accept_apply(g, d, s);
  }
}

#define KMC_GRAPH_STEPS 8

int kmc_run(kmc_handle h, int steps, const double* uniforms, int64_t* events, double* dts) {
  KMC_TRACE("kmc_run");
  int r = guard(h);
  if (r) return r;
  if (h->g.E <= 0) return fail(h, KMC_ERR_STATE, "kmc_run needs lattice mode");
  if (steps < 0) return fail(h, KMC_ERR_ARG, "negative step count");
  if (steps == 0) return KMC_OK;
  if (!uniforms) return fail(h, KMC_ERR_ARG, "uniforms are required");
  cudaStream_t s = h->stream;
  if (steps > h->run_cap) {
    int cap = steps < 1024 ? 1024 : steps;
    ALLOC(h->d.uni_run, sizeof(double) * 2 * (size_t)cap);
    ALLOC(h->d.ev_hist, sizeof(int64_t) * (size_t)cap);
    ALLOC(h->d.dt_hist, sizeof(double) * (size_t)cap);
    h->run_cap = cap;
    h->run_gen++;
    if (h->graph) {  // kernel arguments changed
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
  }
  CK(cudaMemcpyAsync(h->d.uni_run, uniforms, sizeof(double) * 2 * steps, in_kind(h), s));
  CK(cudaMemsetAsync(h->d.stepc, 0, sizeof(int), s));
  // graph of KMC_GRAPH_STEPS steps, built once per handle and shape
  if (!h->graph) {
    cudaGraph_t gr;
    cudaStream_t cs = s;
    bool own = false;
    if (cs == nullptr) {  // the legacy stream cannot be captured
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    cudaStream_t saved = h->stream;
    h->stream = cs;
    CK(cudaStreamSynchronize(s));
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < KMC_GRAPH_STEPS; k++) enqueue_step(h);
    cudaError_t ce = cudaStreamEndCapture(cs, &gr);
    h->stream = saved;
    if (ce != cudaSuccess) {
      if (own) cudaStreamDestroy(cs);
      return fail(h, KMC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&h->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (own) cudaStreamDestroy(cs);
    if (ce != cudaSuccess) return fail(h, KMC_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
  }
  int full = steps / KMC_GRAPH_STEPS, rest = steps % KMC_GRAPH_STEPS;
  for (int b = 0; b < full; b++) CK(cudaGraphLaunch(h->graph, s));
  for (int k = 0; k < rest; k++) enqueue_step(h);
  CKLAUNCH();
  h->peff_valid = false;
  h->rates_valid = false;
  if (events) CK(cudaMemcpyAsync(events, h->d.ev_hist, sizeof(int64_t) * steps, out_kind(h), s));
  if (dts) CK(cudaMemcpyAsync(dts, h->d.dt_hist, sizeof(double) * steps, out_kind(h), s));
  return check_flags(h, "run");
}

int kmc_run_profiled(kmc_handle h, int steps, const double* uniforms, int64_t* events, double* dts,
                     double* phase_ms) {
  KMC_TRACE("kmc_run_profiled");
  int r = guard(h);
  if (r) return r;
  if (h->g.E <= 0) return fail(h, KMC_ERR_STATE, "kmc_run_profiled needs lattice mode");
  if (steps < 0) return fail(h, KMC_ERR_ARG, "negative step count");
  if (steps == 0) return KMC_OK;
  if (!uniforms) return fail(h, KMC_ERR_ARG, "uniforms are required");
  cudaStream_t s = h->stream;
  if (steps > h->run_cap) {
    int cap = steps < 1024 ? 1024 : steps;
    ALLOC(h->d.uni_run, sizeof(double) * 2 * (size_t)cap);
    ALLOC(h->d.ev_hist, sizeof(int64_t) * (size_t)cap);
    ALLOC(h->d.dt_hist, sizeof(double) * (size_t)cap);
    h->run_cap = cap;
    h->run_gen++;
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
  }
  CK(cudaMemcpyAsync(h->d.uni_run, uniforms, sizeof(double) * 2 * steps, in_kind(h), s));
  CK(cudaMemsetAsync(h->d.stepc, 0, sizeof(int), s));
  std::vector<cudaEvent_t> ev((size_t)steps * (KMC_NPHASE + 1));
  for (auto& e : ev) CK(cudaEventCreate(&e));
  const Geo& g = h->g;
  const Dev& d = h->d;
  for (int k = 0; k < steps; k++) {
    cudaEvent_t* e = &ev[(size_t)k * (KMC_NPHASE + 1)];
    CK(cudaEventRecord(e[0], s));
    fmm_downward(g, d, h->prec, s);
    CK(cudaEventRecord(e[1], s));
    kmc_propose_lattice(g, d, h->prec, s);
    CK(cudaEventRecord(e[2], s));
    kmc_finalize_rates(g, d, h->prec, s);
    CK(cudaEventRecord(e[3], s));
    kmc_select(g, d, 1, s);
    kmc_record(g, d, s);
    CK(cudaEventRecord(e[4], s));
    kmc_accept_from_event(g, d, s);
    kmc_accept_apply(g, d, s);
    if (g.dirichlet) {
      kmc_mirror_move(g, d, s);
      kmc_accept_apply(g, d, s);
    }
    CK(cudaEventRecord(e[5], s));
  }
  CKLAUNCH();
  h->peff_valid = false;
  h->rates_valid = false;
  if (events) CK(cudaMemcpyAsync(events, h->d.ev_hist, sizeof(int64_t) * steps, out_kind(h), s));
  if (dts) CK(cudaMemcpyAsync(dts, h->d.dt_hist, sizeof(double) * steps, out_kind(h), s));
  CK(cudaStreamSynchronize(s));
  if (phase_ms) {
    for (int p = 0; p < KMC_NPHASE; p++) phase_ms[p] = 0.0;
    for (int k = 0; k < steps; k++)
      for (int p = 0; p < KMC_NPHASE; p++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[(size_t)k * (KMC_NPHASE + 1) + p], ev[(size_t)k * (KMC_NPHASE + 1) + p + 1]));
        phase_ms[p] += ms;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return check_flags(h, "run_profiled");
}

int kmc_fmm_recompute(kmc_handle h, double* drift) {
  KMC_TRACE("kmc_fmm_recompute");
  int r = guard(h);
  if (r) return r;
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  // potentials at the charges and the tracked energy from the incremental state
  r = compute_phi_old(h);
  if (r) return r;
  if (!h->phi_save) ALLOC(h->phi_save, sizeof(double) * g.n);
  CK(cudaMemcpyAsync(h->phi_save, h->d.phi_old, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, s));
  double U_tracked;
  CK(cudaMemcpyAsync(&U_tracked, h->d.U, sizeof(double), cudaMemcpyDeviceToHost, s));
  double2* saved = (double2*)h->d.scratch;  // lattice-sum scratch is free after init
  size_t need = sizeof(double2) * g.ncell_total * g.P;
  const int nr = 13, nk = 19;
  size_t have = (size_t)(nr * nr * nr + nk * nk * nk) * g.P2 * sizeof(double2);
  if (need > have) {
    double2* tmp = nullptr;
    ALLOC(tmp, need);
    saved = tmp;
  }
  CK(cudaMemcpyAsync(saved, h->d.Psi, need, cudaMemcpyDeviceToDevice, s));
  r = full_fmm(h);
  if (r) return r;
  fmm_drift(g, saved, h->d.Psi, g.ncell_total * g.P, h->drift2, s);
  CKLAUNCH();
  double dc[2];
  CK(cudaMemcpyAsync(dc, h->drift2, sizeof(dc), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  r = compute_energy(h);
  if (r) return r;
  fmm_drift1(h->phi_save, h->d.phi_old, g.n, h->drift2, s);
  CKLAUNCH();
  double dp[2], U_fresh;
  CK(cudaMemcpyAsync(dp, h->drift2, sizeof(dp), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&U_fresh, h->d.U, sizeof(double), cudaMemcpyDeviceToHost, s));
  r = check_flags(h, "recompute");
  if (r) return r;
  if (drift) {
    drift[0] = dp[1] > 0.0 ? dp[0] / dp[1] : 0.0;
    drift[1] = dc[1] > 0.0 ? dc[0] / dc[1] : 0.0;
    drift[2] = U_fresh != 0.0 ? fabs(U_tracked - U_fresh) / fabs(U_fresh) : fabs(U_tracked - U_fresh);
  }
  return KMC_OK;
}

int kmc_fmm_leaf_index(kmc_handle h, int32_t* leaf) {
  int r = guard(h);
  if (r) return r;
  if (!leaf) return fail(h, KMC_ERR_ARG, "leaf is NULL");
  const int64_t n = h->g.nphys;
  std::vector<int32_t> so(n);
  CK(cudaMemcpyAsync(so.data(), h->d.slot_of, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t i = 0; i < n; i++) so[i] = so[i] / h->g.cap;
  if (h->mem == KMC_MEM_DEVICE) {
    CK(cudaMemcpy(leaf, so.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  } else {
    memcpy(leaf, so.data(), sizeof(int32_t) * n);
  }
  return KMC_OK;
}

int kmc_fmm_positions(kmc_handle h, double* positions) {
  int r = guard(h);
  if (r) return r;
  if (!positions) return fail(h, KMC_ERR_ARG, "positions is NULL");
  CK(cudaMemcpyAsync(positions, h->d.pos, sizeof(double) * 3 * h->g.nphys, out_kind(h), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return KMC_OK;
}

// ------------------------------------------------------------------ replica batches
// A batch advances many independent lattice systems together.  When the
// members share precision, hop set and near-field mode (and have no Dirichlet
// walls), a step of the whole batch is L_max + 6 launches, each covering every
// member (BatchPlan: member r owns a block range of each launch), replayed
// from a CUDA graph of KMC_GRAPH_STEPS steps; each member keeps its own
// uniforms, step counter and event history in batch-owned arrays.  Otherwise
// the members' own steps are the parallel branches of one graph (fork/join
// over one stream per member).
struct kmc_batch {
  std::vector<kmc_fmm*> h;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaStream_t s0;
  cudaEvent_t fork;
  cudaGraphExec_t graph;
  int graph_cap;
  std::vector<int> gen;  // members' buffer generations the graph was captured with
  bool parallel;         // members captured as parallel branches
  // batched kernels
  bool fused;
  BatchPlan bp;
  BatchRep* reps;        // [R] device
  int* offs;             // block offsets of every launch, device
  double* uni;           // [R][cap][2] uniforms
  int* stepc;            // [R] step counters
  int64_t* ev;           // [R][cap] events
  double* dt;            // [R][cap] time increments
  int cap;
  int chunk_req;         // requested near-field pass capacity (0: the smallest that fits)
  cudaGraphExec_t fgraph;
  std::vector<BatchRep> reps_host;
  cudaEvent_t t0, t1;
  char msg[512];
};

static int bfail(kmc_batch* b, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
  va_end(ap);
  return code;
}

// block offsets of one batched launch from per-member block counts
static void push_offsets(std::vector<int>& all, const std::vector<int>& cnt, int* total) {
  int acc = 0;
  for (int c : cnt) {
    all.push_back(acc);
    acc += c;
  }
  all.push_back(acc);
  *total = acc;
}

// the launch plan of the batched step (offsets uploaded to b->offs)
static int batch_plan(kmc_batch* b) {
  const int R = (int)b->h.size();
  BatchPlan& bp = b->bp;
  bp.R = R;
  bp.prec = b->h[0]->prec;
  bp.nhop = b->h[0]->g.nhop;
  bp.near_cache = b->h[0]->g.near_cache;
  bp.Lmax = 0;
  int cmin = 2;
  for (kmc_fmm* h : b->h) {
    bp.Lmax = h->g.L > bp.Lmax ? h->g.L : bp.Lmax;
    const int c = kmc_propose_chunk_min(h->g);
    cmin = c > cmin ? c : cmin;
  }
  if (b->chunk_req > 0 && (b->chunk_req < cmin || (b->chunk_req & 1)))
    return bfail(b, KMC_ERR_ARG, "near-field pass capacity %d below %d or odd", b->chunk_req, cmin);
  bp.chunk = b->chunk_req;
  // members' pass capacities: the smallest that fits their leaves, or the requested one; members
  // of equal capacity share a propose launch (its shared memory fits the class, not the largest leaf)
  std::vector<int> mch(R);
  std::vector<int> classes;
  for (int r = 0; r < R; r++) {
    const int c = kmc_propose_chunk_min(b->h[r]->g);
    mch[r] = b->chunk_req > c ? b->chunk_req : c;
    bool seen = false;
    for (int x : classes) seen |= x == mch[r];
    if (!seen) classes.push_back(mch[r]);
  }
  std::sort(classes.begin(), classes.end());
  if ((int)classes.size() > KMC_MAXL) return bfail(b, KMC_ERR_ARG, "too many leaf shapes in one batch");
  bp.nprop = (int)classes.size();
  std::vector<int> all, cnt(R);
  std::vector<size_t> pos;  // index of each launch's offsets in all
  size_t ts = bp.prec == 0 ? sizeof(double2) : sizeof(float2);
  bp.smem_down = 0;
  bp.smem_acr = 0;
  // downward: one launch per level, the parent cells of the members that have the level (with many
  // members a level's launch is wide enough; the single-system path fuses the coarse levels instead)
  for (int l = 2; l <= bp.Lmax; l++) {
    for (int r = 0; r < R; r++) cnt[r] = b->h[r]->g.L >= l ? 1 << (3 * (l - 2)) : 0;
    pos.push_back(all.size());
    push_offsets(all, cnt, &bp.nblk_down[l]);
  }
  for (int r = 0; r < R; r++) {
    const Geo& g = b->h[r]->g;
    const size_t sd = 9 * (size_t)(g.p + 1) * (g.p + 1) * ts;
    bp.smem_down = sd > bp.smem_down ? sd : bp.smem_down;
    const size_t sa = kmc_acr_smem_for(g);
    bp.smem_acr = sa > bp.smem_acr ? sa : bp.smem_acr;
  }
  size_t p_prop[KMC_MAXL];
  for (int c = 0; c < bp.nprop; c++) {
    bp.chunk_c[c] = classes[c];
    bp.smem_prop[c] = 0;
    for (int r = 0; r < R; r++) {
      cnt[r] = mch[r] == classes[c] ? (int)b->h[r]->g.ML : 0;
      if (cnt[r]) {
        const size_t sp = kmc_propose_smem_for(b->h[r]->g, bp.prec, classes[c], bp.near_cache);
        bp.smem_prop[c] = sp > bp.smem_prop[c] ? sp : bp.smem_prop[c];
      }
    }
    p_prop[c] = all.size();
    push_offsets(all, cnt, &bp.nblk_prop[c]);
  }
  for (int r = 0; r < R; r++) cnt[r] = (int)((b->h[r]->g.n + KMC_FIN_PARTICLES - 1) / KMC_FIN_PARTICLES);
  const size_t p_fin = all.size();
  push_offsets(all, cnt, &bp.nblk_fin);
  for (int r = 0; r < R; r++) cnt[r] = kmc_acc_blocks_for(b->h[r]->g);
  const size_t p_acc = all.size();
  push_offsets(all, cnt, &bp.nblk_acc);
  for (int r = 0; r < R; r++) cnt[r] = kmc_acr_blocks();
  const size_t p_acr = all.size();
  push_offsets(all, cnt, &bp.nblk_acr);
  for (int r = 0; r < R; r++) cnt[r] = bp.near_cache ? 2 * 27 : 0;
  const size_t p_nu = all.size();
  push_offsets(all, cnt, &bp.nblk_nu);
  if (b->offs) cudaFree(b->offs);
  b->offs = nullptr;
  if (cudaMalloc(&b->offs, sizeof(int) * all.size()) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, KMC_ERR_OOM, "batch offsets: device allocation failed");
  }
  if (cudaMemcpy(b->offs, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, KMC_ERR_CUDA, "batch offsets: copy failed");
  for (int l = 2; l <= bp.Lmax; l++) bp.off_down[l] = b->offs + pos[l - 2];
  for (int c = 0; c < bp.nprop; c++) bp.off_prop[c] = b->offs + p_prop[c];
  bp.off_fin = b->offs + p_fin;
  bp.off_acc = b->offs + p_acc;
  bp.off_acr = b->offs + p_acr;
  bp.off_nu = b->offs + p_nu;
  bp.reps = b->reps;
  kmc_batch_prepare(bp);
  if (cudaGetLastError() != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "batch kernels could not be prepared");
  return KMC_OK;
}

// batch-owned run buffers for at least `need` steps per member
static int batch_reserve(kmc_batch* b, int need) {
  if (need <= b->cap) return KMC_OK;
  const int R = (int)b->h.size();
  const int cap = need < 1024 ? 1024 : need;
  cudaFree(b->uni);
  cudaFree(b->ev);
  cudaFree(b->dt);
  b->uni = nullptr;
  b->ev = nullptr;
  b->dt = nullptr;
  b->cap = 0;
  if (cudaMalloc(&b->uni, sizeof(double) * 2 * (size_t)cap * R) != cudaSuccess ||
      cudaMalloc(&b->ev, sizeof(int64_t) * (size_t)cap * R) != cudaSuccess ||
      cudaMalloc(&b->dt, sizeof(double) * (size_t)cap * R) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, KMC_ERR_OOM, "batch run buffers: device allocation failed");
  }
  b->cap = cap;
  return KMC_OK;
}

int kmc_batch_create(kmc_batch_handle* out, int count, const kmc_handle* handles) {
  KMC_TRACE("kmc_batch_create");
  if (!out) return KMC_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !handles) return KMC_ERR_ARG;
  kmc_batch* b = new kmc_batch();
  b->graph = nullptr;
  b->graph_cap = 0;
  b->parallel = false;
  b->fused = false;
  b->reps = nullptr;
  b->offs = nullptr;
  b->uni = nullptr;
  b->stepc = nullptr;
  b->ev = nullptr;
  b->dt = nullptr;
  b->cap = 0;
  b->chunk_req = 0;
  b->fgraph = nullptr;
  b->t0 = b->t1 = nullptr;
  b->msg[0] = 0;
  *out = b;
  int dev = -1;
  for (int r = 0; r < count; r++) {
    kmc_fmm* h = handles[r];
    if (!h || h->broken) return bfail(b, KMC_ERR_ARG, "member %d is NULL or broken", r);
    if (h->g.E <= 0) return bfail(b, KMC_ERR_STATE, "member %d is not in lattice mode", r);
    if (dev >= 0 && h->device != dev) return bfail(b, KMC_ERR_ARG, "members must share one device");
    dev = h->device;
    for (int q = 0; q < r; q++)
      if (handles[q] == h) return bfail(b, KMC_ERR_ARG, "member %d appears twice", r);
    b->h.push_back(h);
  }
  if (cudaSetDevice(dev) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "cudaSetDevice failed");
  if (cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return bfail(b, KMC_ERR_CUDA, "stream / event creation failed");
  b->streams.resize(count);
  b->join.resize(count);
  for (int r = 0; r < count; r++)
    if (cudaStreamCreateWithFlags(&b->streams[r], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[r], cudaEventDisableTiming) != cudaSuccess)
      return bfail(b, KMC_ERR_CUDA, "stream / event creation failed");
  if (cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess)
    return bfail(b, KMC_ERR_CUDA, "event creation failed");
  // batched kernels when the members share the kernels' template choices
  bool same = true;
  for (int r = 1; r < count; r++) {
    const kmc_fmm* a = b->h[0];
    const kmc_fmm* h = b->h[r];
    if (h->prec != a->prec || h->g.nhop != a->g.nhop || h->g.near_cache != a->g.near_cache) same = false;
  }
  for (int r = 0; r < count; r++)
    if (b->h[r]->g.dirichlet) same = false;
  if (same) {
    if (cudaMalloc(&b->reps, sizeof(BatchRep) * count) != cudaSuccess ||
        cudaMalloc(&b->stepc, sizeof(int) * count) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, KMC_ERR_OOM, "batch descriptors: device allocation failed");
    }
    int rc = batch_plan(b);
    if (rc) return rc;
    b->fused = true;
  }
  return KMC_OK;
}

int kmc_batch_set_chunk(kmc_batch_handle b, int chunk) {
  KMC_TRACE("kmc_batch_set_chunk");
  if (!b) return KMC_ERR_ARG;
  if (!b->fused) return bfail(b, KMC_ERR_STATE, "the batch runs its members' own kernels (mixed modes)");
  if (chunk < 0) return bfail(b, KMC_ERR_ARG, "negative pass capacity");
  if (cudaSetDevice(b->h[0]->device) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "cudaSetDevice failed");
  if (b->s0) cudaStreamSynchronize(b->s0);
  const int old = b->chunk_req;
  b->chunk_req = chunk;
  // the plan's offsets are reallocated: a captured graph refers to the old ones
  if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
  b->fgraph = nullptr;
  int rc = batch_plan(b);
  if (rc) {
    b->chunk_req = old;
    char keep[sizeof(b->msg)];
    memcpy(keep, b->msg, sizeof(keep));
    if (batch_plan(b)) b->fused = false;  // cannot restore the plan: fall back to the members' own kernels
    memcpy(b->msg, keep, sizeof(keep));
    return rc;
  }
  return KMC_OK;
}

int kmc_batch_info(kmc_batch_handle b, int* fused, int* chunk, int* launches_per_step) {
  if (!b) return KMC_ERR_ARG;
  if (fused) *fused = b->fused ? 1 : 0;
  if (chunk) *chunk = b->fused ? b->bp.chunk_c[b->bp.nprop - 1] : 0;
  if (launches_per_step) {
    int n = 0;
    if (b->fused) {
      n = 1 + 5 + b->bp.nprop + (b->bp.near_cache ? 1 : 0);  // level 1, rates .. accept, propose(s)
      for (int l = 2; l <= b->bp.Lmax; l++) n += b->bp.nblk_down[l] > 0;
    } else {
      for (kmc_fmm* h : b->h) n += h->g.L + 7 + (h->g.near_cache ? 1 : 0) + (h->g.dirichlet ? 3 : 0);
    }
    *launches_per_step = n;
  }
  return KMC_OK;
}

int kmc_check_bounded_wait(int device, double limit_seconds) {
  if (cudaSetDevice(device) != cudaSuccess) return KMC_ERR_CUDA;
  const int f = kmc_wait_probe(limit_seconds, 0);
  if (f < 0) return KMC_ERR_CUDA;
  return (f & KMC_DERR_TIMEOUT) ? KMC_ERR_TIMEOUT : KMC_OK;
}

const char* kmc_batch_last_error(kmc_batch_handle b) { return b ? b->msg : g_static_msg; }

void kmc_batch_destroy(kmc_batch_handle b) {
  if (!b) return;
  if (!b->h.empty()) cudaSetDevice(b->h[0]->device);
  if (b->s0) cudaStreamSynchronize(b->s0);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
  cudaFree(b->reps);
  cudaFree(b->offs);
  cudaFree(b->uni);
  cudaFree(b->stepc);
  cudaFree(b->ev);
  cudaFree(b->dt);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  for (size_t r = 0; r < b->streams.size(); r++) {
    if (b->streams[r]) cudaStreamDestroy(b->streams[r]);
    if (b->join[r]) cudaEventDestroy(b->join[r]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

#define BCK(call, what)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_));   \
  } while (0)

// the batched-kernel path: K steps of every member, device time in *ms
static int batch_run_fused(kmc_batch* b, int steps, const double* uniforms, int64_t* events, double* dts,
                           double* ms) {
  const int R = (int)b->h.size();
  int rc = batch_reserve(b, steps);
  if (rc) return rc;
  const size_t cap = (size_t)b->cap;
  b->reps_host.resize(R);
  for (int r = 0; r < R; r++) {
    kmc_fmm* h = b->h[r];
    BatchRep& x = b->reps_host[r];
    x.g = h->g;
    x.d = h->d;
    x.d.uni_run = b->uni + 2 * cap * r;
    x.d.ev_hist = b->ev + cap * r;
    x.d.dt_hist = b->dt + cap * r;
    x.d.stepc = b->stepc + r;
    if (h->stream) BCK(cudaStreamSynchronize(h->stream), "member stream synchronisation");
  }
  // uniforms [step][member][2] -> [member][step][2] with row pitch 2 cap
  std::vector<double> col(2 * (size_t)steps * R);
  for (int r = 0; r < R; r++)
    for (int st = 0; st < steps; st++) {
      col[((size_t)r * steps + st) * 2] = uniforms[((size_t)st * R + r) * 2];
      col[((size_t)r * steps + st) * 2 + 1] = uniforms[((size_t)st * R + r) * 2 + 1];
    }
  cudaStream_t s = b->s0;
  BCK(cudaMemcpy2DAsync(b->uni, sizeof(double) * 2 * cap, col.data(), sizeof(double) * 2 * steps,
                        sizeof(double) * 2 * steps, R, cudaMemcpyHostToDevice, s), "staging uniforms");
  BCK(cudaMemcpyAsync(b->reps, b->reps_host.data(), sizeof(BatchRep) * R, cudaMemcpyHostToDevice, s),
      "staging member descriptors");
  BCK(cudaMemsetAsync(b->stepc, 0, sizeof(int) * R, s), "clearing step counters");
  if (!b->fgraph) {
    cudaGraph_t gr = nullptr;
    BCK(cudaStreamSynchronize(s), "stream synchronisation");
    BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture begin");
    for (int k = 0; k < KMC_GRAPH_STEPS; k++) {
      fmm_downward_batch(b->bp, s);
      kmc_step_batch(b->bp, s);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(s, &gr);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return bfail(b, KMC_ERR_CUDA, "batch graph capture failed: %s / %s", cudaGetErrorString(le),
                   cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&b->fgraph, gr, 0);
    cudaGraphDestroy(gr);
    if (ce != cudaSuccess) {
      b->fgraph = nullptr;
      return bfail(b, KMC_ERR_CUDA, "batch graph instantiate failed: %s", cudaGetErrorString(ce));
    }
  }
  BCK(cudaEventRecord(b->t0, s), "event record");
  const int full = steps / KMC_GRAPH_STEPS, rest = steps % KMC_GRAPH_STEPS;
  for (int k = 0; k < full; k++) BCK(cudaGraphLaunch(b->fgraph, s), "graph launch");
  for (int k = 0; k < rest; k++) {
    fmm_downward_batch(b->bp, s);
    kmc_step_batch(b->bp, s);
  }
  BCK(cudaGetLastError(), "batch kernel launch");
  BCK(cudaEventRecord(b->t1, s), "event record");
  BCK(cudaStreamSynchronize(s), "batch run");
  if (ms) {
    float f = 0.f;
    BCK(cudaEventElapsedTime(&f, b->t0, b->t1), "event timing");
    *ms = f;
  }
  std::vector<int64_t> ev((size_t)steps * R);
  std::vector<double> dt((size_t)steps * R);
  BCK(cudaMemcpy2D(ev.data(), sizeof(int64_t) * steps, b->ev, sizeof(int64_t) * cap, sizeof(int64_t) * steps, R,
                   cudaMemcpyDeviceToHost), "reading events");
  BCK(cudaMemcpy2D(dt.data(), sizeof(double) * steps, b->dt, sizeof(double) * cap, sizeof(double) * steps, R,
                   cudaMemcpyDeviceToHost), "reading time increments");
  for (int r = 0; r < R; r++) {
    kmc_fmm* h = b->h[r];
    h->peff_valid = false;
    h->rates_valid = false;
    int rc2 = check_flags(h, "batch run");
    if (rc2) return bfail(b, rc2, "member %d: %s", r, h->msg);
    for (int st = 0; st < steps; st++) {
      if (events) events[(size_t)st * R + r] = ev[(size_t)r * steps + st];
      if (dts) dts[(size_t)st * R + r] = dt[(size_t)r * steps + st];
    }
  }
  return KMC_OK;
}

static int batch_run_impl(kmc_batch* b, int steps, const double* uniforms, int64_t* events, double* dts,
                          double* ms) {
  if (!b) return KMC_ERR_ARG;
  const int R = (int)b->h.size();
  if (steps < 0 || !uniforms) return bfail(b, KMC_ERR_ARG, "steps >= 0 and uniforms are required");
  if (ms) *ms = 0.0;
  if (steps == 0) return KMC_OK;
  if (cudaSetDevice(b->h[0]->device) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "cudaSetDevice failed");
  for (int r = 0; r < R; r++)
    if (b->h[r]->broken) return bfail(b, KMC_ERR_STATE, "member %d broken: %s", r, b->h[r]->msg);
  if (b->fused) return batch_run_fused(b, steps, uniforms, events, dts, ms);
  // per-member buffers for the uniforms and the event history
  int need = steps;
  bool realloc = false;
  for (int r = 0; r < R; r++) {
    kmc_fmm* h = b->h[r];
    if (need > h->run_cap) {
      int cap = need < 1024 ? 1024 : need;
      if (dalloc(h, &h->d.uni_run, sizeof(double) * 2 * (size_t)cap) || dalloc(h, &h->d.ev_hist, sizeof(int64_t) * (size_t)cap) ||
          dalloc(h, &h->d.dt_hist, sizeof(double) * (size_t)cap))
        return bfail(b, KMC_ERR_OOM, "member %d: %s", r, h->msg);
      h->run_cap = cap;
      h->run_gen++;
      if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
      }
    }
    if (b->gen.size() == (size_t)R && b->gen[r] != h->run_gen) realloc = true;
  }
  if (realloc && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  std::vector<double> col(2 * (size_t)steps);
  for (int r = 0; r < R; r++) {
    kmc_fmm* h = b->h[r];
    for (int s = 0; s < steps; s++) {
      col[2 * s] = uniforms[((size_t)s * R + r) * 2];
      col[2 * s + 1] = uniforms[((size_t)s * R + r) * 2 + 1];
    }
    if (cudaMemcpy(h->d.uni_run, col.data(), sizeof(double) * 2 * steps, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d.stepc, 0, sizeof(int)) != cudaSuccess)
      return bfail(b, KMC_ERR_CUDA, "staging uniforms failed");
    if (h->stream && cudaStreamSynchronize(h->stream) != cudaSuccess)
      return bfail(b, KMC_ERR_CUDA, "member stream synchronisation failed");
  }
  if (!b->graph) {
    // fork/join capture (members' steps as parallel branches); if the driver
    // refuses it, the members are captured one after another on one stream
    for (int attempt = 0; attempt < 2 && !b->graph; attempt++) {
      const bool parallel = attempt == 0;
      cudaGraph_t gr = nullptr;
      cudaGetLastError();
      if (cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bfail(b, KMC_ERR_CUDA, "capture begin failed");
      cudaError_t first = cudaSuccess;
      if (parallel) first = cudaEventRecord(b->fork, b->s0);
      for (int r = 0; r < R && first == cudaSuccess; r++) {
        kmc_fmm* h = b->h[r];
        cudaStream_t st = parallel ? b->streams[r] : b->s0;
        if (parallel) first = cudaStreamWaitEvent(st, b->fork, 0);
        if (first != cudaSuccess) break;
        cudaStream_t saved = h->stream;
        h->stream = st;
        enqueue_step(h);
        h->stream = saved;
        first = cudaGetLastError();
        if (first == cudaSuccess && parallel) first = cudaEventRecord(b->join[r], st);
        if (first == cudaSuccess && parallel) first = cudaStreamWaitEvent(b->s0, b->join[r], 0);
      }
      cudaError_t ce = cudaStreamEndCapture(b->s0, &gr);
      if (first == cudaSuccess && ce == cudaSuccess) {
        ce = cudaGraphInstantiate(&b->graph, gr, 0);
        if (ce != cudaSuccess) b->graph = nullptr;
      }
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      if (!b->graph && attempt == 1)
        return bfail(b, KMC_ERR_CUDA, "graph capture failed: %s / %s", cudaGetErrorString(first),
                     cudaGetErrorString(ce));
      b->parallel = parallel && b->graph != nullptr;
    }
    b->gen.resize(R);
    for (int r = 0; r < R; r++) b->gen[r] = b->h[r]->run_gen;
  }
  if (cudaEventRecord(b->t0, b->s0) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "event record failed");
  for (int s = 0; s < steps; s++)
    if (cudaGraphLaunch(b->graph, b->s0) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "graph launch failed");
  if (cudaEventRecord(b->t1, b->s0) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "event record failed");
  if (cudaStreamSynchronize(b->s0) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "batch run failed");
  if (ms) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, b->t0, b->t1) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "event timing failed");
    *ms = f;
  }
  std::vector<int64_t> ev(steps);
  std::vector<double> dt(steps);
  for (int r = 0; r < R; r++) {
    kmc_fmm* h = b->h[r];
    h->peff_valid = false;
    h->rates_valid = false;
    if (cudaMemcpy(ev.data(), h->d.ev_hist, sizeof(int64_t) * steps, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(dt.data(), h->d.dt_hist, sizeof(double) * steps, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(b, KMC_ERR_CUDA, "reading events failed");
    int rc = check_flags(h, "batch run");
    if (rc) return bfail(b, rc, "member %d: %s", r, h->msg);
    for (int s = 0; s < steps; s++) {
      if (events) events[(size_t)s * R + r] = ev[s];
      if (dts) dts[(size_t)s * R + r] = dt[s];
    }
  }
  return KMC_OK;
}

int kmc_batch_run(kmc_batch_handle b, int steps, const double* uniforms, int64_t* events, double* dts) {
  KMC_TRACE("kmc_batch_run");
  return batch_run_impl(b, steps, uniforms, events, dts, nullptr);
}

int kmc_batch_run_timed(kmc_batch_handle b, int steps, const double* uniforms, int64_t* events, double* dts,
                        double* device_ms) {
  KMC_TRACE("kmc_batch_run_timed");
  return batch_run_impl(b, steps, uniforms, events, dts, device_ms);
}


int kmc_fmm_m2l_timed(kmc_handle h, int reps, double* level_ms, double* total_ms) {
  KMC_TRACE("kmc_fmm_m2l_timed");
  if (!h || reps <= 0 || !level_ms || !total_ms) return KMC_ERR_ARG;
  int rc = guard(h);
  if (rc) return rc;
  const Geo& g = h->g;
  cudaStream_t s = h->stream;
  for (int l = 0; l <= KMC_MAXL; l++) level_ms[l] = 0.0;
  *total_ms = 0.0;
  Dev d2 = h->d;  // the products go to a scratch copy of the local expansions
  void* scratch = nullptr;
  double2* psi = nullptr;
  cudaEvent_t ev[2 * (KMC_MAXL + 1)], t0 = nullptr, t1 = nullptr;
  int made = 0;
  rc = KMC_OK;
  for (; made < 2 * (KMC_MAXL + 1); made++)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  if (made < 2 * (KMC_MAXL + 1) || cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess ||
      cudaMallocAsync(&scratch, fmm_m2l_scratch_bytes(g), s) != cudaSuccess ||
      cudaMallocAsync((void**)&psi, sizeof(double2) * g.ncell_total * g.P, s) != cudaSuccess) {
    rc = fail(h, KMC_ERR_OOM, "M2L timing: events or scratch unavailable");
  } else {
    d2.Psi = psi;
    for (int r = 0; r < reps && rc == KMC_OK; r++) {
      cudaEventRecord(t0, s);
      fmm_m2l(g, d2, scratch, s, ev);
      cudaEventRecord(t1, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        rc = fail(h, KMC_ERR_CUDA, "M2L timing: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float f = 0.f;
      cudaEventElapsedTime(&f, t0, t1);
      *total_ms += f / reps;
      for (int l = 3; l <= g.L; l++) {
        cudaEventElapsedTime(&f, ev[2 * l], ev[2 * l + 1]);
        level_ms[l] += f / reps;
      }
    }
  }
  if (scratch) cudaFreeAsync(scratch, s);
  if (psi) cudaFreeAsync(psi, s);
  cudaStreamSynchronize(s);
  for (int k = 0; k < made; k++) cudaEventDestroy(ev[k]);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (rc) return rc;
  return check_flags(h, "M2L timing");
}

int kmc_batch_propose_timed(kmc_batch_handle b, int reps, double* device_ms) {
  KMC_TRACE("kmc_batch_propose_timed");
  if (!b || reps <= 0 || !device_ms) return KMC_ERR_ARG;
  *device_ms = 0.0;
  if (!b->fused) return bfail(b, KMC_ERR_ARG, "propose timing needs a batch on the batched kernels");
  if (!b->fgraph) return bfail(b, KMC_ERR_ARG, "run the batch once before timing its propose launches");
  if (cudaSetDevice(b->h[0]->device) != cudaSuccess) return bfail(b, KMC_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = b->s0;
  BCK(cudaEventRecord(b->t0, s), "event record");
  for (int k = 0; k < reps; k++) kmc_propose_batch(b->bp, s);
  BCK(cudaGetLastError(), "batch propose launch");
  BCK(cudaEventRecord(b->t1, s), "event record");
  BCK(cudaStreamSynchronize(s), "batch propose");
  float f = 0.f;
  BCK(cudaEventElapsedTime(&f, b->t0, b->t1), "event timing");
  *device_ms = f / reps;
  for (kmc_fmm* h : b->h) {
    h->rates_valid = false;
    const int rc = check_flags(h, "batch propose");
    if (rc) return bfail(b, rc, "%s", h->msg);
  }
  return KMC_OK;
}

}  // extern "C"
