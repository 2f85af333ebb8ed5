"""GB300 (sm_103a) FMM for kinetic Monte Carlo -- Python binding of libkmcfmm.

Every function here marshals arguments for the C ABI declared in
include/kmcfmm.h and calls it; all arithmetic runs in the CUDA library.
There is no CPU fallback: importing works without a GPU, but creating a
handle needs the built library and a CUDA device, and fails loudly
otherwise.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); the kind is fixed per handle by the positions passed to
kmc_fmm_init.  Hop k of particle i is event j = nh i + k with nh = 6 (the
faces +x, -x, +y, -y, +z, -z) or 14 (then the body diagonals, x fastest).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB, build as build_library

KMC_OK = 0
KMC_ERR_ARG = 1
KMC_ERR_NOT_NEUTRAL = 2
KMC_ERR_OOM = 3
KMC_ERR_CUDA = 4
KMC_ERR_CAPACITY = 5
KMC_ERR_TIMEOUT = 6
KMC_ERR_STATE = 7
KMC_PREC_FP64 = 0
KMC_PREC_MIXED = 1
KMC_MEM_HOST = 0
KMC_MEM_DEVICE = 1
KMC_M2L_TENSOR = 0
KMC_M2L_FP64 = 1
KMC_M2L_TENSOR_SYNC = 2
KMC_L2L_TENSOR = 0
KMC_L2L_CUDA = 1
KMC_HOPS_6 = 0
KMC_HOPS_14 = 1
KMC_BC_PERIODIC = 0
KMC_BC_FREE = 1
KMC_BC_DIRICHLET_Z = 2

EXPORTS = [
    "kmc_opts_default", "kmc_fmm_init", "kmc_fmm_energy", "kmc_fmm_propose", "kmc_fmm_propose_lattice",
    "kmc_fmm_propose_lattice_f32", "kmc_fmm_propose_lattice_async", "kmc_fmm_outputs_wait",
    "kmc_fmm_accept", "kmc_fmm_accept_event", "kmc_step", "kmc_run", "kmc_run_profiled", "kmc_fmm_recompute",
    "kmc_fmm_leaf_index", "kmc_fmm_positions", "kmc_last_error", "kmc_fmm_destroy", "kmc_select_static",
    "kmc_check_bounded_wait",
    "kmc_check_tensor_mma",
    "kmc_fmm_m2l_timed",
    "kmc_batch_create", "kmc_batch_run", "kmc_batch_run_timed", "kmc_batch_set_chunk", "kmc_batch_info",
    "kmc_batch_propose_timed", "kmc_batch_last_error", "kmc_batch_destroy",
]


class KmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kmcfmm error {code}: {msg}")
        self.code = code


class kmc_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("lattice_edge", ctypes.c_int),
        ("lattice_h", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("mem", ctypes.c_int),
        ("device", ctypes.c_int),
        ("leaf_capacity", ctypes.c_int),
        ("m2l", ctypes.c_int),
        ("hops", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("field_z", ctypes.c_double),
        ("near_cache", ctypes.c_int),
        ("l2l", ctypes.c_int),
    ]


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libkmcfmm.so (building it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build_library())
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "kmc_opts_default": (None, [P]),
            "kmc_fmm_init": (I, [P, I64, P, P, D, I, I, P]),
            "kmc_fmm_energy": (I, [P, P]),
            "kmc_fmm_propose": (I, [P, I64, P, P, P, P]),
            "kmc_fmm_propose_lattice": (I, [P, P, P]),
            "kmc_fmm_propose_lattice_f32": (I, [P, P, P]),
            "kmc_fmm_propose_lattice_async": (I, [P, P, P]),
            "kmc_fmm_outputs_wait": (I, [P]),
            "kmc_fmm_accept": (I, [P, ctypes.c_int32, P, P]),
            "kmc_fmm_accept_event": (I, [P, I64, P]),
            "kmc_step": (I, [P, P, D, D, P, P, P]),
            "kmc_run": (I, [P, I, P, P, P]),
            "kmc_run_profiled": (I, [P, I, P, P, P, P]),
            "kmc_fmm_recompute": (I, [P, P]),
            "kmc_fmm_leaf_index": (I, [P, P]),
            "kmc_fmm_positions": (I, [P, P]),
            "kmc_last_error": (ctypes.c_char_p, [P]),
            "kmc_fmm_destroy": (None, [P]),
            "kmc_select_static": (I, [P, I64, D, D, P, P, P, P]),
            "kmc_check_bounded_wait": (I, [I, D]),
            "kmc_check_tensor_mma": (I, [I, I, ctypes.c_void_p]),
            "kmc_fmm_m2l_timed": (I, [P, I, P, P]),
            "kmc_batch_create": (I, [P, I, P]),
            "kmc_batch_run": (I, [P, I, P, P, P]),
            "kmc_batch_run_timed": (I, [P, I, P, P, P, P]),
            "kmc_batch_set_chunk": (I, [P, I]),
            "kmc_batch_info": (I, [P, P, P, P]),
            "kmc_batch_propose_timed": (I, [P, I, P]),
            "kmc_batch_last_error": (ctypes.c_char_p, [P]),
            "kmc_batch_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Handle:
    """An initialised FMM-KMC system (owns the C handle)."""

    def __init__(self, ptr, n: int, mem: int, lattice: bool, device: int, nhop: int = 6):
        self.ptr = ptr
        self.n = n
        self.mem = mem
        self.lattice = lattice
        self.device = device
        self.nhop = nhop  # lattice hops per charge (events j = nhop * i + k)
        self._pending = None  # output buffers of an asynchronous proposal still being copied

    def __del__(self):
        try:
            kmc_fmm_destroy(self)
        except Exception:
            pass


def _check(h, code: int):
    if code != KMC_OK:
        lib = load_library()
        msg = lib.kmc_last_error(h.ptr if isinstance(h, Handle) else h)
        raise KmcError(code, msg.decode() if msg else "")


def _host(x, dtype):
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _arg(h: Handle, x, dtype, torch_dtype=None):
    """(keep-alive object, pointer) for an input array in the handle's memory kind."""
    if x is None:
        return None, None
    if h.mem == KMC_MEM_DEVICE:
        import torch
        if not (_is_torch(x) and x.is_cuda):
            x = torch.as_tensor(np.asarray(x, dtype=dtype), device=f"cuda:{h.device}")
        x = x.contiguous()
        return x, ctypes.c_void_p(x.data_ptr())
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return _host(x, dtype)


def _out(h: Handle, shape, dtype):
    if h.mem == KMC_MEM_DEVICE:
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8, np.int64: torch.int64,
               np.int32: torch.int32}[np.dtype(dtype).type]
        t = torch.empty(shape, dtype=tdt, device=f"cuda:{h.device}")
        return t, ctypes.c_void_p(t.data_ptr())
    a = np.empty(shape, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ C-ABI calls
def kmc_fmm_init(positions, charges, box: float, levels: int, order: int, precision: str = "fp64",
                 lattice_edge: int = 0, lattice_h: float = 1.0, kT: float = 1.0, stream=None, device: int = 0,
                 leaf_capacity: int = 0, m2l: str = "tensor", hops: int = 6, bc: str = "periodic",
                 field_z: float = 0.0, near_cache: bool = False, l2l: str = "tensor") -> Handle:
    """Create a handle and run the one-off full FMM.  precision: 'fp64' or 'mixed';
    m2l: 'tensor' (bf16 tensor cores with exact slicing, tcgen05 MMA), 'tensor_sync' (the same slicing on
    the mma.sync form, bit for bit the same result) or 'fp64' (FP64 CUDA cores);
    hops: the lattice hop set, 6 (faces) or 14 (faces and body diagonals);
    bc: 'periodic' (neutral systems), 'free' (free space) or 'dirichlet' (grounded walls at z = 0 and
    z = box/2, lattice mode, every charge below box/2, applied field field_z along z);
    near_cache: lattice mode, keep every site's near-field sum on the device and update it per
    accepted move instead of summing the pairs every step;
    l2l: the mixed form's per-step downward pass on its two finest levels, 'tensor' (tcgen05 tf32
    MMAs, FP32 operands split in two, p <= 14) or 'cuda' (FP32 CUDA cores)."""
    lib = load_library()
    opts = kmc_opts()
    lib.kmc_opts_default(ctypes.byref(opts))
    opts.precision = {"fp64": KMC_PREC_FP64, "mixed": KMC_PREC_MIXED}[precision]
    opts.lattice_edge = int(lattice_edge)
    opts.lattice_h = float(lattice_h)
    opts.kT = float(kT)
    opts.device = int(device)
    opts.leaf_capacity = int(leaf_capacity)
    opts.m2l = {"tensor": KMC_M2L_TENSOR, "fp64": KMC_M2L_FP64, "tensor_sync": KMC_M2L_TENSOR_SYNC}[m2l]
    opts.hops = {6: KMC_HOPS_6, 14: KMC_HOPS_14}[int(hops)]
    opts.bc = {"periodic": KMC_BC_PERIODIC, "free": KMC_BC_FREE, "dirichlet": KMC_BC_DIRICHLET_Z}[bc]
    opts.field_z = float(field_z)
    opts.near_cache = 1 if near_cache else 0
    opts.l2l = {"tensor": KMC_L2L_TENSOR, "cuda": KMC_L2L_CUDA}[l2l]
    dev = _is_torch(positions) and positions.is_cuda
    opts.mem = KMC_MEM_DEVICE if dev else KMC_MEM_HOST
    if stream is not None:
        opts.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    elif dev:
        import torch
        opts.stream = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    n = int(positions.shape[0])
    tmp = Handle(None, n, opts.mem, lattice_edge > 0, device)
    pos_keep, pos_p = _arg(tmp, positions, np.float64)
    q_keep, q_p = _arg(tmp, charges, np.float64)
    ptr = ctypes.c_void_p()
    code = lib.kmc_fmm_init(ctypes.byref(ptr), n, pos_p, q_p, float(box), int(levels), int(order),
                            ctypes.byref(opts))
    h = Handle(ptr, n, opts.mem, lattice_edge > 0, device, int(hops))
    if code != KMC_OK:
        msg = lib.kmc_last_error(ptr)
        text = msg.decode() if msg else ""
        lib.kmc_fmm_destroy(ptr)
        h.ptr = None
        raise KmcError(code, text)
    # what a checkpoint needs to rebuild the system (positions come from the handle)
    h.init_args = dict(charges=np.array(charges.detach().cpu().numpy() if _is_torch(charges) else charges,
                                        dtype=np.float64),
                       box=float(box), levels=int(levels), order=int(order), precision=precision,
                       lattice_edge=int(lattice_edge), lattice_h=float(lattice_h), kT=float(kT),
                       leaf_capacity=int(leaf_capacity), m2l=m2l, hops=int(hops), bc=bc, field_z=float(field_z),
                       near_cache=bool(near_cache), l2l=l2l)
    return h


# ------------------------------------------------------------------ checkpoint / resume
def kmc_checkpoint(h: Handle, path: str, step: int = 0, **extra) -> None:
    """Save the state of a KMC system to an .npz file: the charges' current positions (user
    order), their charges, the arguments the handle was created with, the caller's step counter
    (e.g. the index into its uniform stream) and any extra arrays or numbers."""
    args = dict(h.init_args)
    q = args.pop("charges")
    pos = kmc_fmm_positions(h)
    if _is_torch(pos):
        pos = pos.cpu().numpy()
    np.savez(path, positions=pos, charges=q, step=np.int64(step),
             init_args=np.array(repr(args)), **{f"extra_{k}": np.asarray(v) for k, v in extra.items()})


def kmc_resume(path: str, stream=None, device: int = 0):
    """Rebuild a system from a checkpoint: a new handle (host-memory arguments) initialised from
    the saved positions, the full FMM recomputed as at init.  The expansions then differ from the
    incrementally updated ones of the saved run by the truncation error only (as after
    kmc_fmm_recompute).  Returns (handle, step, extra)."""
    import ast
    z = np.load(path, allow_pickle=False)
    args = ast.literal_eval(str(z["init_args"]))
    h = kmc_fmm_init(z["positions"], z["charges"], stream=stream, device=device, **args)
    extra = {k[len("extra_"):]: z[k] for k in z.files if k.startswith("extra_")}
    return h, int(z["step"]), extra


def kmc_fmm_energy(h: Handle) -> float:
    U = ctypes.c_double()
    _check(h, load_library().kmc_fmm_energy(h.ptr, ctypes.byref(U)))
    return U.value


def kmc_fmm_propose(h: Handle, particle, target, mask=None):
    """dU for proposals particle[t] -> target[t] (m x 3)."""
    lib = load_library()
    pk, pp = _arg(h, particle, np.int32)
    tk, tp = _arg(h, target, np.float64)
    mk, mp = _arg(h, mask, np.uint8)
    m = int(pk.shape[0])
    out, op = _out(h, (m,), np.float64)
    _check(h, lib.kmc_fmm_propose(h.ptr, m, pp, tp, mp, op))
    return out


def flatten_proposals(P):
    """The paper's proposal list (Sec. 4.2, "Proposing moves"): a sequence of tuples
    (i, R_i), R_i an n_i x 3 array of new positions for charge i, flattened into the
    (particle[m], target[m x 3]) form of kmc_fmm_propose, plus the split offsets."""
    idx, tgt, counts = [], [], []
    for i, R in P:
        R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
        idx.append(np.full(R.shape[0], int(i), dtype=np.int32))
        tgt.append(R)
        counts.append(R.shape[0])
    if not counts:
        return np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros(1, np.int64)
    off = np.concatenate(([0], np.cumsum(counts))).astype(np.int64)
    return np.concatenate(idx), np.ascontiguousarray(np.concatenate(tgt)), off


def kmc_fmm_propose_tuples(h: Handle, P):
    """dU for the paper's proposal list P = ((i1, R_i1), (i2, R_i2), ...): returns a tuple
    (U_i1, U_i2, ...) of host arrays, U_i[k] the energy change of moving charge i to R_i[k]."""
    particle, target, off = flatten_proposals(P)
    dU = kmc_fmm_propose(h, particle, target)
    if _is_torch(dU):
        dU = dU.cpu().numpy()
    return tuple(dU[off[k]:off[k + 1]] for k in range(len(off) - 1))


def _given(h: Handle, x, shape, dtype):
    """A caller-provided output buffer (numpy array or torch tensor) in the
    handle's memory kind: checked for shape, dtype and contiguity."""
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8}[np.dtype(dtype).type]
        if tuple(x.shape) != shape or x.dtype != tdt or not x.is_contiguous() or \
                (x.device.type == "cuda") != (h.mem == KMC_MEM_DEVICE):
            raise ValueError(f"output buffer must be a contiguous {shape} {tdt} tensor in the handle's memory")
        return x, ctypes.c_void_p(x.data_ptr())
    if h.mem == KMC_MEM_DEVICE:
        raise ValueError("a device-memory handle needs torch CUDA output tensors")
    if x.shape != shape or x.dtype != np.dtype(dtype) or not x.flags.c_contiguous:
        raise ValueError(f"output buffer must be a C-contiguous {shape} {np.dtype(dtype)} array")
    return x, x.ctypes.data_as(ctypes.c_void_p)


def kmc_fmm_propose_lattice(h: Handle, mask=None, dU=None, dtype=np.float64, wait: bool = True):
    """(mask[n,nh], dU[n,nh]) for all hops of the handle's hop set.  mask and dU may be
    caller-owned buffers (e.g. pinned host memory) that are filled in place.  dtype (or the
    given dU buffer's dtype) float32: the mixed form's FP32 dU, copied without widening.
    wait=False (FP32 only): the copies keep running after the call (kmc_step and
    kmc_fmm_accept_event may run beside them); the buffers hold the outputs after
    kmc_fmm_outputs_wait(h)."""
    lib = load_library()
    nh = h.nhop
    if dU is not None:
        dtype = np.float32 if str(dU.dtype).endswith("float32") else np.float64
    dtype = np.dtype(dtype).type
    mask, mp = _out(h, (h.n, nh), np.uint8) if mask is None else _given(h, mask, (h.n, nh), np.uint8)
    dU, dp = _out(h, (h.n, nh), dtype) if dU is None else _given(h, dU, (h.n, nh), dtype)
    if not wait:
        if dtype is not np.float32:
            raise ValueError("wait=False needs the FP32 output (dtype float32)")
        _check(h, lib.kmc_fmm_propose_lattice_async(h.ptr, mp, dp))
        h._pending = (mask, dU)  # the buffers stay alive while their copies run
    elif dtype is np.float32:
        _check(h, lib.kmc_fmm_propose_lattice_f32(h.ptr, mp, dp))
    else:
        _check(h, lib.kmc_fmm_propose_lattice(h.ptr, mp, dp))
    return mask, dU


def kmc_fmm_outputs_wait(h: Handle) -> None:
    """Block until the copies of the last kmc_fmm_propose_lattice(..., wait=False) are done."""
    _check(h, load_library().kmc_fmm_outputs_wait(h.ptr))
    h._pending = None


def kmc_fmm_accept(h: Handle, particle: int, target) -> float:
    lib = load_library()
    t, tp = _host(np.asarray(target, dtype=np.float64).reshape(3), np.float64)
    du = ctypes.c_double()
    if h.mem == KMC_MEM_DEVICE:
        tk, tp = _arg(h, t, np.float64)
    _check(h, lib.kmc_fmm_accept(h.ptr, int(particle), tp, ctypes.byref(du)))
    return du.value


def kmc_fmm_accept_event(h: Handle, event: int) -> float:
    du = ctypes.c_double()
    _check(h, load_library().kmc_fmm_accept_event(h.ptr, int(event), ctypes.byref(du)))
    return du.value


def kmc_step(h: Handle, rates, zeta: float, xi: float):
    """(event, dt, Q) by rejection-free selection; rates None = last lattice proposal."""
    lib = load_library()
    rk, rp = _arg(h, rates, np.float64)
    ev = ctypes.c_int64()
    dt = ctypes.c_double()
    Q = ctypes.c_double()
    _check(h, lib.kmc_step(h.ptr, rp, float(zeta), float(xi), ctypes.byref(ev), ctypes.byref(dt), ctypes.byref(Q)))
    return ev.value, dt.value, Q.value


def kmc_run(h: Handle, uniforms):
    """Run len(uniforms) device-driven KMC steps; returns (events, dts)."""
    lib = load_library()
    uk, up = _arg(h, uniforms, np.float64)
    steps = int(uk.shape[0])
    ev, evp = _out(h, (steps,), np.int64)
    dt, dtp = _out(h, (steps,), np.float64)
    _check(h, lib.kmc_run(h.ptr, steps, up, evp, dtp))
    return ev, dt


KMC_NPHASE = 5
PHASES = ("downward", "propose", "rates", "select", "accept")


def kmc_run_profiled(h: Handle, uniforms):
    """kmc_run without graph replay; returns (events, dts, phase_ms[5])."""
    lib = load_library()
    uk, up = _arg(h, uniforms, np.float64)
    steps = int(uk.shape[0])
    ev, evp = _out(h, (steps,), np.int64)
    dt, dtp = _out(h, (steps,), np.float64)
    ph = np.zeros(KMC_NPHASE, dtype=np.float64)
    _check(h, lib.kmc_run_profiled(h.ptr, steps, up, evp, dtp, ph.ctypes.data_as(ctypes.c_void_p)))
    return ev, dt, ph


def kmc_fmm_recompute(h: Handle):
    """Full recompute; returns (potential drift, coefficient drift, energy drift)."""
    drift = np.zeros(3, dtype=np.float64)
    _check(h, load_library().kmc_fmm_recompute(h.ptr, drift.ctypes.data_as(ctypes.c_void_p)))
    return tuple(float(x) for x in drift)


def kmc_fmm_leaf_index(h: Handle):
    out, op = _out(h, (h.n,), np.int32)
    _check(h, load_library().kmc_fmm_leaf_index(h.ptr, op))
    return out


def kmc_fmm_positions(h: Handle):
    out, op = _out(h, (h.n, 3), np.float64)
    _check(h, load_library().kmc_fmm_positions(h.ptr, op))
    return out


def kmc_last_error(h: Handle) -> str:
    msg = load_library().kmc_last_error(h.ptr if h is not None else None)
    return msg.decode() if msg else ""


def kmc_fmm_destroy(h: Handle) -> None:
    if h is not None and h.ptr is not None:
        load_library().kmc_fmm_destroy(h.ptr)
        h.ptr = None


KMC_STATIC_MAX_N = 16777216


def kmc_select_static(rates, n: int, zeta: float, xi: float, stream=None):
    """Selection without a handle and without device allocation.

    For callers that cannot allocate device memory: code inside a framework
    whose caching allocator owns the device, host loops that must not stall on
    the synchronisation an allocation can cause, plugin hosts that forbid
    their plugins to own device memory.  rates: CUDA tensor of at least 6 n
    doubles owned by the caller (the first 6 n are read).  Returns (event, dt,
    Q).  Calls share one static scratch array, so calls that overlap on the
    GPU must be serialised by the caller."""
    import torch
    lib = load_library()
    if not (_is_torch(rates) and rates.is_cuda and rates.dtype == torch.float64 and rates.is_contiguous()):
        raise KmcError(KMC_ERR_ARG, "rates must be a contiguous float64 CUDA tensor")
    if int(n) >= 1 and rates.numel() < 6 * int(n):
        raise KmcError(KMC_ERR_ARG, f"rates holds {rates.numel()} entries, fewer than 6 n = {6 * int(n)}")
    s = stream if stream is not None else torch.cuda.current_stream(rates.device)
    sp = ctypes.c_void_p(int(getattr(s, "cuda_stream", s)))
    ev = ctypes.c_int64()
    dt = ctypes.c_double()
    Q = ctypes.c_double()
    with torch.cuda.device(rates.device):
        code = lib.kmc_select_static(ctypes.c_void_p(rates.data_ptr()), int(n), float(zeta), float(xi),
                                     ctypes.byref(ev), ctypes.byref(dt), ctypes.byref(Q), sp)
    if code != KMC_OK:
        raise KmcError(code, "kmc_select_static: invalid argument or CUDA error")
    return ev.value, dt.value, Q.value


class Batch:
    """Several lattice-mode handles advanced together from one CUDA graph."""

    def __init__(self, ptr, handles):
        self.ptr = ptr
        self.handles = list(handles)  # keep the members alive

    def __del__(self):
        try:
            kmc_batch_destroy(self)
        except Exception:
            pass


def kmc_batch_create(handles) -> Batch:
    lib = load_library()
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr for h in handles])
    ptr = ctypes.c_void_p()
    code = lib.kmc_batch_create(ctypes.byref(ptr), len(handles), arr)
    b = Batch(ptr, handles)
    if code != KMC_OK:
        msg = lib.kmc_batch_last_error(ptr)
        kmc_batch_destroy(b)
        raise KmcError(code, msg.decode() if msg else "")
    return b


def _batch_check(b: Batch, code: int):
    if code != KMC_OK:
        msg = load_library().kmc_batch_last_error(b.ptr)
        raise KmcError(code, msg.decode() if msg else "")


def kmc_batch_run(b: Batch, uniforms, timed: bool = False):
    """uniforms: [steps, members, 2]; returns (events, dts), each [steps, members]; with
    timed=True also the device time of the steps in ms."""
    lib = load_library()
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    steps, R = int(u.shape[0]), len(b.handles)
    if u.shape != (steps, R, 2):
        raise ValueError(f"uniforms must have shape (steps, {R}, 2)")
    ev = np.empty((steps, R), dtype=np.int64)
    dt = np.empty((steps, R), dtype=np.float64)
    ms = ctypes.c_double()
    _batch_check(b, lib.kmc_batch_run_timed(b.ptr, steps, u.ctypes.data_as(ctypes.c_void_p),
                                            ev.ctypes.data_as(ctypes.c_void_p), dt.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(ms)))
    return (ev, dt, ms.value) if timed else (ev, dt)


def kmc_batch_set_chunk(b: Batch, chunk: int) -> None:
    """P2P tile of the batched propose: near-field sources staged per pass (0 = smallest that fits)."""
    _batch_check(b, load_library().kmc_batch_set_chunk(b.ptr, int(chunk)))


def kmc_batch_info(b: Batch) -> dict:
    """{'fused': batched kernels?, 'chunk': P2P pass capacity, 'launches_per_step': kernels per step}."""
    f, c, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _batch_check(b, load_library().kmc_batch_info(b.ptr, ctypes.byref(f), ctypes.byref(c), ctypes.byref(n)))
    return {"fused": bool(f.value), "chunk": c.value, "launches_per_step": n.value}


def kmc_batch_propose_timed(b: Batch, reps: int = 10) -> float:
    """Mean device ms of one set of the batch step's propose launches (measurement hook)."""
    ms = ctypes.c_double()
    _batch_check(b, load_library().kmc_batch_propose_timed(b.ptr, int(reps), ctypes.byref(ms)))
    return ms.value


def kmc_batch_last_error(b: Batch) -> str:
    msg = load_library().kmc_batch_last_error(b.ptr if b is not None else None)
    return msg.decode() if msg else ""


def kmc_batch_destroy(b: Batch) -> None:
    if b is not None and b.ptr is not None:
        load_library().kmc_batch_destroy(b.ptr)
        b.ptr = None


def kmc_check_bounded_wait(device: int = 0, limit_seconds: float = 0.05) -> int:
    """Status of the bounded-wait diagnostic: KMC_ERR_TIMEOUT (6) when the
    device-side wait gave up and returned as designed."""
    return int(load_library().kmc_check_bounded_wait(int(device), float(limit_seconds)))


def kmc_fmm_m2l_timed(h: Handle, reps: int = 3):
    """(per-level ms of the M2L product kernel {level: ms}, ms of the whole M2L) over reps runs into
    scratch; the handle's state is unchanged."""
    lv = np.zeros(11, np.float64)
    tot = ctypes.c_double(0.0)
    _check(h, load_library().kmc_fmm_m2l_timed(h.ptr, int(reps), lv.ctypes.data, ctypes.byref(tot)))
    return {l: float(lv[l]) for l in range(3, 11) if lv[l] > 0.0}, float(tot.value)


def kmc_check_tensor_mma(device: int = 0, out=None, kind: int = 0) -> int:
    """One tcgen05 MMA of small integer operands, staged as the tensor-core M2L stages them, against
    the exact product: 0 agreement, 1 mismatch, negative: unavailable or timed out.  out: None or a
    float32 array of 128 x 192 that receives the product read back from tensor memory."""
    ptr = None
    if out is not None:
        assert out.dtype == np.float32 and out.size == 128 * 192 and out.flags["C_CONTIGUOUS"]
        ptr = out.ctypes.data
    return int(load_library().kmc_check_tensor_mma(int(device), int(kind), ptr))

