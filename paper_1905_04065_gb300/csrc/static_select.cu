// static_select.cu -- allocation-free rejection-free event selection.
//
// Some callers cannot allocate device memory.  A library that runs inside a
// framework whose caching allocator owns the device memory must not take
// memory behind that allocator's back (it can fail, or fragment the pool the
// framework sized for itself); a host loop with a latency budget must not
// stall on the implicit device synchronisation that cudaMalloc and cudaFree
// can cause; a plugin host may simply forbid its plugins to own device
// memory.  For them this file offers kmc_select_static: the same block-sum
// and selection kernels as kmc_step, with their scratch (block sums, the two
// uniforms, the selected event, dt and Q) in a file-scope __device__ array
// instead of memory owned by a handle.  It needs no handle and allocates
// nothing.  It copies the uniforms from the host and synchronises the
// caller's stream to return the event, dt and Q as host scalars.
//
// The array is a static object of the module: every GPU that loads this
// library holds it (KMC_STATIC_BLOCKS + 8 doubles, about 1 MB) until the
// process exits.  All calls share it, so calls whose GPU work overlaps (two
// streams, two host threads) race on it; order them on one stream or
// serialise them.  Every element a call reads is written earlier in the same
// call, so nothing has to start at zero.
#include <string.h>

#include <atomic>

#include "../../include/kmcfmm.h"
#include "common.cuh"

#define KMC_STATIC_THREADS KMC_FIN_PARTICLES  // particles per block sum, as in kmc_step
#define KMC_STATIC_BLOCKS ((KMC_STATIC_MAX_N + KMC_STATIC_THREADS - 1) / KMC_STATIC_THREADS)

// [0, KMC_STATIC_BLOCKS): block sums; then zeta, xi; event (as int64); dt, Q
static __device__ __align__(256) double g_select_scratch[KMC_STATIC_BLOCKS + 8];

// Device address of g_select_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up by
// cudaGetSymbolAddress on the first call on each device, with that device
// current.  Two host threads making their first call on one device at once
// both look it up and store the same value; the atomic makes that benign.
#define KMC_STATIC_MAX_DEVICES 64
static std::atomic<double*> g_select_addr[KMC_STATIC_MAX_DEVICES];

extern "C" int kmc_select_static(const double* rates, int64_t n, double zeta, double xi, int64_t* event,
                                 double* dt, double* Q, void* stream) {
  if (!rates || !event || !dt || !Q) return KMC_ERR_ARG;
  if (n < 1 || n > KMC_STATIC_MAX_N) return KMC_ERR_ARG;  // beyond the static scratch
  if (!(zeta > 0.0 && zeta <= 1.0 && xi > 0.0 && xi <= 1.0)) return KMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= KMC_STATIC_MAX_DEVICES) return KMC_ERR_CUDA;
  double* base = g_select_addr[dev].load(std::memory_order_relaxed);
  if (!base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KMC_ERR_CUDA;
    }
    base = (double*)p;
    g_select_addr[dev].store(base, std::memory_order_relaxed);
  }
  cudaStream_t s = (cudaStream_t)stream;
  Geo g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  g.nhop = KMC_NHOP;
  Dev d;
  memset(&d, 0, sizeof(d));
  d.rate = (double*)rates;
  d.bsum = base;
  d.uni_small = base + KMC_STATIC_BLOCKS;
  d.event = (int64_t*)(base + KMC_STATIC_BLOCKS + 2);
  d.dtq = base + KMC_STATIC_BLOCKS + 4;
  const double u[2] = {zeta, xi};
  if (cudaMemcpyAsync(d.uni_small, u, sizeof(u), cudaMemcpyHostToDevice, s) != cudaSuccess) return KMC_ERR_CUDA;
  kmc_rate_bsum(g, d, s);
  kmc_select(g, d, 0, s);
  if (cudaGetLastError() != cudaSuccess) return KMC_ERR_CUDA;
  int64_t ev = -1;
  double dq[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(&ev, d.event, sizeof(ev), cudaMemcpyDeviceToHost, s) != cudaSuccess) return KMC_ERR_CUDA;
  if (cudaMemcpyAsync(dq, d.dtq, sizeof(dq), cudaMemcpyDeviceToHost, s) != cudaSuccess) return KMC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KMC_ERR_CUDA;
  *event = ev;
  *dt = dq[0];
  *Q = dq[1];
  return KMC_OK;
}
