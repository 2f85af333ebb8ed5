"""Benchmark: dU evaluations/s and KMC steps/s of FMM-for-KMC on one GB300.

Workload (default): 256^3-site periodic simple-cubic lattice, 1,048,576 +-1
charges on uniform-random distinct sites, 6 nearest-neighbour hop proposals
per charge, FMM with 6 levels and order p = 12, kT = 0.05, mixed precision
(FP32 near-field pairs, L2P and dU assembly; FP64 M2L, lattice sums, accept
updates of the expansions and cumulative rate sums).  A step is one full KMC step: downward pass, propose (all hops),
rates, selection, accept.

Timed regions (CUDA events on the library's stream, after W warm-up steps):
  value   K steps of kmc_run_profiled, one step per call, L2 flushed (a
          256 MiB write) before every step; the step time is the device time
          of the step's kernels, from the library's events recorded on the
          launching stream before the first and after the last kernel (the
          per-phase events inside the same call give the propose kernel's
          duration); dU evals/s = unmasked proposals / step time.  The time
          including the host-side call overhead is reported beside it.
  e2e     the host API path per step (kmc_fmm_propose_lattice into host
          buffers, kmc_step, kmc_fmm_accept_event), host<->device copies inside.
  fp64    the same step loop with the FP64 form (context line).
  cpu     the FP64 oracle on a bounded sample (host cores).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload small|medium|large]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "dU evals/sec and KMC steps/sec at N=1M, FP32-mixed vs FP64"
DTYPE_MIXED = "f32-mixed (f32 near field, L2P and dU assembly; f64 M2L, lattice sums, accept updates, rate sums)"
UNIT = "dU evals/s"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(units: float, ms: float, device=None):
    """Whole-job figures of independent replicas, one per rank: the units all
    ranks processed (sum) and the slowest rank's time (max).  No collective
    touches the data path; this is the only cross-rank exchange."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


def launches_per_step(L: int, bc: str = "periodic") -> int:
    """Kernels of one device-driven step: the downward pass (levels 2..4 in one launch, each deeper
    level one), propose, rates, select, move record, event decode, the fused accept and its coarse
    reduction; grounded walls add the mirror move and its accept (3)."""
    return 1 + max(L - 4, 0) + 7 + (3 if bc == "dirichlet" else 0)


# --------------------------------------------------------------- algorithmic work
def step_bytes(E: int, L: int, N: int, p: int) -> int:
    """Lower bound of the device bytes one lattice step touches: FP64 rates and
    FP32 dU for the 6N hops, the leaf-major FP32 coordinates (capacity W^3 per
    leaf) and the FP32 leaf expansions."""
    nL = 2 ** (L - 1)
    ML, W = nL ** 3, E // nL
    P = (p + 1) * (p + 2) // 2
    return 6 * N * (8 + 4) + ML * W ** 3 * 16 + ML * P * 8


def pair_count(E: int, L: int, sites: np.ndarray, nhop: int = 6, bc: str = "periodic") -> dict:
    """Evaluation sites and near-field pairs of one propose launch, counted
    from the configuration.  The potential is needed once per distinct site:
    every occupied site (old positions) and every empty site that some charge
    can hop to; per leaf, pairs = needed sites x charges in the 27
    neighbouring leaves (the pair at distance 0 included in the count).
    hops = the unmasked proposals (dU evaluations) of the caller's charges.
    Free space: no wrapping, hops out of the box masked.  Dirichlet walls: the
    kernel works on the mirrored cell (the charges and their mirrors); hops
    through a wall are masked."""
    nL = 2 ** (L - 1)
    W = E // nL
    phys = np.asarray(sites, dtype=np.int64)
    if bc == "dirichlet":
        x, y, z = phys % E, (phys // E) % E, phys // (E * E)
        sites = np.concatenate([phys, x + E * (y + E * (E - 1 - z))])
    xyz = workloads.site_xyz(E, sites)
    occ = np.zeros(E ** 3, dtype=bool)
    occ[sites] = True
    needed = occ.copy()
    hops = 0
    nph = len(phys)
    for (dx, dy, dz) in workloads.hop_vectors(nhop).tolist():
        raw = xyz + np.array([dx, dy, dz])
        t = raw % E
        ts = t[:, 0] + E * (t[:, 1] + E * t[:, 2])
        ok = ~occ[ts]
        if bc == "free":
            ok &= np.all((raw >= 0) & (raw < E), axis=1)
        if bc == "dirichlet":
            wall = (raw[:, 2] < 0) | (raw[:, 2] >= E // 2)
            hops += int((ok[:nph] & ~wall[:nph]).sum())
        else:
            hops += int(ok.sum())
        needed[ts[ok]] = True
    ns = np.nonzero(needed)[0]
    nxyz = workloads.site_xyz(E, ns) // W
    pts = np.bincount(nxyz[:, 0] + nL * (nxyz[:, 1] + nL * nxyz[:, 2]), minlength=nL ** 3).astype(np.int64)
    leafc = xyz // W
    cnt = np.bincount(leafc[:, 0] + nL * (leafc[:, 1] + nL * leafc[:, 2]), minlength=nL ** 3).reshape(nL, nL, nL)
    src = np.zeros_like(cnt)
    if bc == "free":  # no neighbour leaves beyond the box
        pad = np.pad(cnt, 1)
        for oz in (0, 1, 2):
            for oy in (0, 1, 2):
                for ox in (0, 1, 2):
                    src += pad[oz:oz + nL, oy:oy + nL, ox:ox + nL]
    else:
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    src += np.roll(cnt, shift=(oz, oy, ox), axis=(0, 1, 2))
    pairs = int(np.sum(pts * src.reshape(-1)))
    return dict(points=int(pts.sum()), pairs=pairs, hops=hops, leaves=nL ** 3)


# DRAM bytes (read + write) of one summing propose launch per leaf, from the ncu capture of the
# 128^3 tile case (4096 leaves of 8^3 sites, 32 charges each, 6 hops, mixed precision:
# 6.16 MB read, 1 kB written).  Valid for workloads with the same
# leaf shape (tile, large); scaled by the number of leaves.
PROPOSE_DRAM_BYTES_PER_LEAF = (6.16448e6 + 1.024e3) / 4096
TRAFFIC_WORKLOADS = ("tile", "large")


def l2p_flops(p: int) -> int:
    """FP32 operations of one L2P (recurrence 6 + accumulate 2 per (n, m), m >= 0)."""
    return 8 * (p + 1) * (p + 2) // 2


def l2l_cmacs(p: int) -> int:
    """Complex multiply-adds of one L2L translation (parent to child, degree p, outputs 0 <= m <= n):
    out(k, l) = sum_{n >= k} sum_m L(n, m) R(n - k, m - l) over the m the child table holds."""
    tot = 0
    for k in range(p + 1):
        for lo in range(k + 1):
            for n in range(k, p + 1):
                j = n - k
                tot += min(lo + j, n) - max(lo - j, -n) + 1
    return tot


def phase_rooflines(work: dict, phases: dict, E: int, L: int, N: int, p: int, nhop: int, peaks: dict,
                    nsm: int, mixed: bool = True) -> dict:
    """Roofline of every per-step phase (ms per step from the library's events), from the
    algorithmic work of the phase: the operations or bytes the method needs, not what the
    kernels issue.  Peaks: HBM from MEASURED_PEAKS.json; FP32 and FP64 FMA from unit counts
    (128 and 2 FMA per clock per SM) at the maximum SM clock."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    hbm = float(peaks["hbm_gbs"]) * 1e9
    fp32 = 2 * 128 * nsm * sm_max
    fp64 = 2 * 2 * nsm * sm_max
    P = (p + 1) * (p + 2) // 2
    cells = sum(8 ** (l - 1) for l in range(2, L + 1))
    parents = sum(8 ** (l - 2) for l in range(2, L + 1))
    ts = 4 if mixed else 8  # bytes of a real coefficient in the downward pass's precision
    out = {}
    # downward: L2L of every cell of levels 2..L from its parent plus its own list expansion
    fl = 8 * l2l_cmacs(p) * cells
    by = cells * P * 2 * ts * 2 + parents * P * 2 * ts  # own + write, parent once
    t = phases["downward"] * 1e-3
    out["downward"] = {"kernels": "k_downward_coarse (levels 2-4 in one launch), k_downward_par (deeper levels); "
                                  "the mixed form's leaf level with >= 4096 parents on tcgen05 tf32 (k_l2l_tc)",
                       "bound": "alu", "unit": "TFLOP/s", "achieved": fl / t / 1e12,
                       "peak": (fp32 if mixed else fp64) / 1e12, "frac": fl / t / (fp32 if mixed else fp64),
                       "work": f"{fl:.3e} {'FP32' if mixed else 'FP64'} flops ({l2l_cmacs(p)} complex MACs per cell, "
                               f"{cells} cells); {by / 1e6:.1f} MB",
                       "hbm_frac": by / t / hbm,
                       "note": "L levels launched in sequence; the work counts the complex MACs of the L2L "
                               "(the tensor-core leaf level does the dense 2P x 2P products, three tf32 products "
                               "each); the per-parent kernel is bound by shared-memory loads, the coarse levels "
                               "and the tensor-core leaf level by latency"}
    # rates: per charge q, site, phi_old, nhop (phi_new, mask) read; nhop (dU, rate) written
    b_rates = N * (4 + 4 + ts + nhop * (ts + 1) + nhop * (ts + 8))
    t = phases["rates"] * 1e-3
    out["rates"] = {"kernels": "k_finalize", "bound": "hbm", "unit": "GB/s", "achieved": b_rates / t / 1e9,
                    "peak": hbm / 1e9, "frac": b_rates / t / hbm,
                    "work": f"{b_rates / 1e6:.1f} MB ({b_rates / N:.0f} B per charge)"}
    # select: the block sums and one block's rates
    nb = (N + 127) // 128
    b_sel = nb * 8 + 128 * nhop * 8
    t = phases["select"] * 1e-3
    out["select"] = {"kernels": "k_select, k_record", "bound": "latency", "unit": "GB/s",
                     "achieved": b_sel / t / 1e9, "peak": hbm / 1e9, "frac": b_sel / t / hbm,
                     "work": f"{b_sel / 1e3:.0f} kB: {nb} block sums and one block of rates",
                     "note": "one CTA walks the cumulative sums: a chain of dependent reductions"}
    # accept: FP64 P2L of the move (two positions) into every cell whose interaction list holds an
    # image of them -- levels 2 (all images of the 5^3 block), 3 (27 images), >= 4 (<= 432
    # candidate cells) -- the multipole changes of all levels, H += R dK, and the slot move
    nl = 2 * (8 * 250 + 64 * 54) + 2 * 189 * max(L - 3, 0)  # P2L evaluations (upper estimate)
    fl_acc = nl * P * 8 * 2 + L * P * 8 * 2 + P * P * 8
    b_acc = (8 + 64 + 432 * max(L - 3, 0)) * P * (16 * 2 + 8)
    t = phases["accept"] * 1e-3
    out["accept"] = {"kernels": "k_move_from_event, k_acc_fused, k_acc_coarse_reduce", "bound": "latency",
                     "unit": "TFLOP/s", "achieved": fl_acc / t / 1e12, "peak": fp64 / 1e12, "frac": fl_acc / t / fp64,
                     "work": f"{fl_acc / 1e6:.1f} M FP64 flops (P2L of both positions into the cells whose lists "
                             f"hold them), {b_acc / 1e6:.1f} MB",
                     "hbm_frac": b_acc / t / hbm,
                     "note": "three dependent launches of small grids; no unit is saturated"}
    return out


# --------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, device: int):
        self.proc = None
        self.path = None
        self.device = device

    def start(self, path):
        self.path = path
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"],
                                         stdout=open(path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the sampler takes a moment to start: wait (at most 3 s) for its first line, so that the
        # samples that follow fall inside the timed region
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def m2l_roofline(levels: dict, total_ms: float, L: int, p: int, peaks: dict, precision: str) -> dict:
    """The leaf level's M2L product kernel against the dense bf16 tensor peak: algorithmic bf16 flops
    = 2 (2P)^2 per slice product, translation and cell (189 far translations per cell of the
    periodic box, 10 slice products with four slices, 21 with six), over its CUDA-event time."""
    P = (p + 1) * (p + 2) // 2
    nslp = 10 if precision == "mixed" else 21
    ncell = 8 ** (L - 1)
    flops = 2.0 * (2 * P) ** 2 * 189 * ncell * nslp
    ms = levels.get(L)
    out = {"kernel": "k_m2l_tc (leaf level)", "bound": "tensor", "unit": "TFLOP/s", "peak": peaks["bf16_tflops"],
           "peak_source": "bf16_tflops of MEASURED_PEAKS.json (cuBLAS bf16 burst)",
           "work": f"{flops:.3e} bf16 flops: {nslp} slice products x 189 translations x {ncell} cells x 2 (2P)^2",
           "level_ms": {str(k): v for k, v in sorted(levels.items())}, "m2l_total_ms": total_ms}
    if ms:
        out["achieved"] = flops / (ms * 1e-3) / 1e12
        out["frac"] = out["achieved"] / peaks["bf16_tflops"]
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- CPU oracle sample
def cpu_sample(E, sites, q, seconds_target=10.0, max_props=20000, nhop=6, bc="periodic"):
    """dU evals/s of the FP64 oracle's direct lattice sum (O(N) per proposal,
    tabulated Ewald pair potential; free space: the direct Coulomb sum) on a
    seeded sample of unmasked hops."""
    import oracle
    if bc == "dirichlet":  # the oracle's grounded walls: the periodic mirrored cell (charges and mirrors)
        ext = np.concatenate([sites, oracle.mirror_sites(E, np.asarray(sites, dtype=np.int64))])
        r = cpu_sample(E, ext, np.concatenate([q, -np.asarray(q)]), seconds_target, max_props, nhop, "periodic")
        r["sample"] += " of the mirrored cell (the charges and their mirrors)"
        return r
    G = oracle.psi_table(E) if bc == "periodic" else None
    pos = workloads.site_positions(E, sites)

    def evaluate(p, t):
        if G is not None:
            oracle.lattice_delta_u_direct(E, G, sites, q, p, t)
        else:
            oracle.free_delta_u(pos, q, p, workloads.site_positions(E, t))
    rng = np.random.default_rng(4242)
    occ = np.zeros(E ** 3, dtype=bool)
    occ[sites] = True
    xyz = workloads.site_xyz(E, sites)
    dirs = workloads.hop_vectors(nhop)

    def draw(m):
        parts, tg = [], []
        while len(parts) < m:
            i = int(rng.integers(0, len(q)))
            k = int(rng.integers(0, nhop))
            t = (xyz[i] + dirs[k]) % E
            s = int(t[0] + E * (t[1] + E * t[2]))
            if not occ[s]:
                parts.append(i)
                tg.append(s)
        return np.array(parts), np.array(tg)

    # calibrate on a small batch, then size the sample to ~seconds_target
    p, t = draw(64)
    t0 = time.perf_counter()
    evaluate(p, t)
    dt = time.perf_counter() - t0
    m = int(min(max_props, max(64, seconds_target / max(dt / 64, 1e-9))))
    p, t = draw(m)
    t0 = time.perf_counter()
    evaluate(p, t)
    dt = time.perf_counter() - t0
    what = ("direct O(N) sum over the tabulated Ewald pair potential" if G is not None
            else "direct O(N) free-space Coulomb sum (numpy, one process)")
    return dict(value=m / dt, unit=UNIT, cores=oracle.num_threads() if G is not None else 1, kind="oracle",
                sample=f"{m} unmasked hops, {what}, FP64")


def cpu_otable(E, sites, q, kT, seed, seconds_target=10.0, max_steps=64):
    """Full KMC steps of the oracle's lattice-table form (O-table): the tabulated Ewald pair
    potential and a site potential kept for all E^3 sites, so that every hop's dU is O(1)
    (propose), Algorithm 1's sequential FP64 selection, and an O(E^3) site-potential update per
    accepted hop.  Periodic, 6 hops.  Returns (measurement dict, number of timed steps); the table
    and the initial FFT site potential are set up before the timed loop."""
    import oracle
    t0 = time.perf_counter()
    st = oracle.LatticeState(E, sites, q)
    setup_s = time.perf_counter() - t0
    u = workloads.uniforms(max_steps, seed + 99)
    steps = hops = 0
    t0 = time.perf_counter()
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < seconds_target):
        dU, mask = st.propose()
        j, Q, dt = oracle.select(oracle.rates(dU, mask, kT), u[steps, 0], u[steps, 1])
        if j >= 0:
            st.accept(j // 6, j % 6)
        hops += int(mask.sum())
        steps += 1
    el = time.perf_counter() - t0
    return dict(value=hops / el, unit=UNIT, kmc_steps_per_s=steps / el, cores=oracle.num_threads(), kind="oracle",
                sample=f"{steps} full KMC steps of the O-table form (every hop's dU from the maintained site "
                       f"potential, sequential FP64 selection, O(E^3) site update per accept), FP64; "
                       f"table + FFT setup {setup_s:.1f} s not timed"), steps


# --------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle timed on the host cores for the same workload and metric.  Periodic 6-hop lattice
    workloads: exactly K full KMC steps of the O-table form after W untimed ones (dU evals/s = the
    unmasked hops of each step over its time).  Other workloads: K bounded samples of the direct
    O(N)-per-hop sum."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    w, sites, q = workloads.workload(args.workload)
    E = w["E"]
    import oracle
    oracle.build()
    if w.get("hops", 6) == 6:
        st = oracle.LatticeState(E, sites, q)
        u = workloads.uniforms(args.warmup + args.steps, w["seed"] + 99)
        times, hops = [], 0
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            dU, mask = st.propose()
            j, Q, dt = oracle.select(oracle.rates(dU, mask, w["kT"]), u[s, 0], u[s, 1])
            if j >= 0:
                st.accept(j // 6, j % 6)
            el = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(el)
                hops += int(mask.sum())
        tot = sum(times)
        v = hops / tot
        sample = (f"{args.steps} full KMC steps of the O-table form (lattice-table Ewald potential, O(1) dU "
                  f"per hop, sequential FP64 selection, O(E^3) site update per accept)")
        extra = {"kmc_steps_per_s": args.steps / tot}
    else:
        G = oracle.psi_table(E)
        per_step = max(16, int(args.ref_props))
        rng = np.random.default_rng(7)
        occ = np.zeros(E ** 3, dtype=bool)
        occ[sites] = True
        xyz = workloads.site_xyz(E, sites)
        dirs = oracle.hop_vectors(w.get("hops", 6))

        def batch():
            parts, tg = [], []
            while len(parts) < per_step:
                i = int(rng.integers(0, len(q)))
                k = int(rng.integers(0, len(dirs)))
                t = (xyz[i] + dirs[k]) % E
                s = int(t[0] + E * (t[1] + E * t[2]))
                if not occ[s]:
                    parts.append(i)
                    tg.append(s)
            return np.array(parts), np.array(tg)

        for _ in range(args.warmup):
            p, t = batch()
            oracle.lattice_delta_u_direct(E, G, sites, q, p, t)
        times = []
        for _ in range(args.steps):
            p, t = batch()
            t0 = time.perf_counter()
            oracle.lattice_delta_u_direct(E, G, sites, q, p, t)
            times.append(time.perf_counter() - t0)
        tot = sum(times)
        v = per_step * args.steps / tot
        sample = f"{per_step} unmasked hops per step, direct O(N) FP64 sum"
        extra = {}
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(w, args.workload), parallelism="replicas x1", bc="periodic"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample, **extra},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        **extra,
    }
    print(json.dumps(line))
    return 0


# The paper's own time per KMC step for the Sec. 5.3 benchmark on one node (Tab. 4, strong scaling
# at P = 1: 10^6 charges on a 300^3 lattice, one charge per 27 sites, 14 hop targets, p = 12,
# L = 6, FP64 generated C, MPI + OpenMP).  Context for the "sec53" workload line, which runs the
# same shape on 288^3 sites (884,736 charges); not the same configuration, so vs_baseline stays null.
PAPER_SEC53 = {"s_per_kmc_step": {"CSD3 Skylake 2x16 cores": 7.43, "Isambard ThunderX2 2x32 cores": 11.93,
                                  "Balena Ivy Bridge 2x8 cores": 21.33, "Balena Skylake 2x12 cores": 10.26},
               "source": "Tab. 4, P = 1 (Sec. 5.3)",
               "configuration": "10^6 charges, 300^3 sites, 14 hops, p = 12, L = 6, FP64"}


def _config(w, name):
    hops = "6 NN hops" if w.get("hops", 6) == 6 else "14 hops (6 faces, 8 body diagonals)"
    return {"workload": f"{name}: {w['E']}^3-site periodic lattice, {w['N']} charges (+-1, neutral), "
                        f"{hops}, L={w['L']}, p={w['p']}, kT={w['kT']}",
            "E": w["E"], "N": w["N"], "levels": w["L"], "order": w["p"], "kT": w["kT"],
            "l2": "flushed (256 MiB write) before every timed step"}


# --------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_1905_04065_gb300 as k

    rank, world, local = _dist()
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w, sites, q = workloads.workload(args.workload)
    E, L, p, kT = w["E"], w["L"], w["p"], w["kT"]
    nhop = w.get("hops", 6)
    # replicas: every rank runs an independent replica with its own seed
    if world > 1 and rank > 0:
        sites, q = workloads.uniform_lattice(E, w["N"], w["seed"] + 7919 * rank)
    if args.bc == "dirichlet":  # the caller's charges below z = E/2; the library adds the mirrors
        sites, q = workloads.lower_half_lattice(E, w["N"], w["seed"] + 7919 * rank)
    pos = workloads.site_positions(E, sites)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    fz = 0.1 if args.bc == "dirichlet" else 0.0
    h = k.kmc_fmm_init(pos, q, float(E), L, p, precision="mixed", lattice_edge=E, kT=kT, stream=stream, device=dev,
                       hops=nhop, bc=args.bc, field_z=fz)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    work = pair_count(E, L, sites, nhop, args.bc)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    u = workloads.uniforms(args.warmup + args.steps + args.e2e_steps + 16, w["seed"])

    # warm-up
    k.kmc_run_profiled(h, u[: args.warmup])
    torch.cuda.synchronize()
    # timed region
    clk = Clocks(dev)
    os.makedirs(args.clocks_dir, exist_ok=True)
    clk.start(os.path.join(args.clocks_dir, f"clocks_rank{rank}.csv"))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, outer_ms, phases = [], [], np.zeros(k.KMC_NPHASE)
    for s in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev, dts, ph = k.kmc_run_profiled(h, u[args.warmup + s: args.warmup + s + 1])
        e1.record(stream)
        e1.synchronize()
        # device time of the step: the library's events on this stream, from
        # before the first kernel to after the last (contiguous phases); the
        # outer pair also holds the host-side call overhead
        step_ms.append(float(ph.sum()))
        outer_ms.append(e0.elapsed_time(e1))
        phases += ph
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    hops = work["hops"]  # unmasked proposals per step (changes negligibly per step)
    units, tot_ms = aggregate(hops * args.steps, float(sum(step_ms)), device=f"cuda:{dev}")
    ms_step = tot_ms / args.steps
    value = units / (tot_ms * 1e-3)
    steps_per_s = world * args.steps / (tot_ms * 1e-3)
    prop_ms = phases[1] / args.steps

    # e2e: host API path with host buffers
    es = args.e2e_steps
    base = args.warmup + args.steps
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # pinned host buffers, allocated once: the caller owns the outputs
    # the mixed form's own FP32 dU (4 bytes per hop); two buffer pairs: the copies of step s run
    # beside its selection and accept, and a pair is reused once the next proposal has returned
    bufs = [(torch.empty((len(q), nhop), dtype=torch.uint8, pin_memory=True),
             torch.empty((len(q), nhop), dtype=torch.float32, pin_memory=True)) for _ in range(2)]
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(es):
        mask_h, dU_h = bufs[s & 1]
        k.kmc_fmm_propose_lattice(h, mask_h, dU_h, wait=False)
        ev, dt, Q = k.kmc_step(h, None, u[base + s, 0], u[base + s, 1])
        if ev >= 0:
            k.kmc_fmm_accept_event(h, ev)
    k.kmc_fmm_outputs_wait(h)  # the last step's outputs are on the host
    e1.record(stream)
    e1.synchronize()
    e2e_units, e2e_tot = aggregate(hops * es, e0.elapsed_time(e1), device=f"cuda:{dev}")
    e2e_ms = e2e_tot / es
    n = len(q)
    e2e = {"value": e2e_units / (e2e_tot * 1e-3), "unit": UNIT,
           # host -> device: kmc_step's two uniforms, the accepted event; device -> host: mask and dU
           # of every hop, the error flags (16 B) after the proposal and after the accept, kmc_step's
           # event and (dt, Q), the accepted event's mask byte and FP32 dU
           "h2d_bytes_per_step": 16 + 8,
           "d2h_bytes_per_step": nhop * n * (1 + 4) + 16 + 8 + 16 + 1 + 4 + 16,
           "path": "kmc_fmm_propose_lattice_async (mask and FP32 dU into pinned host buffers, the copies "
                   "beside kmc_step and kmc_fmm_accept_event) + kmc_step + kmc_fmm_accept_event, "
                   "kmc_fmm_outputs_wait after the last step"}

    # one recompute (full FMM from the current charges, the drift control of kmc_fmm_recompute)
    torch.cuda.synchronize()
    t_r = time.perf_counter()
    k.kmc_fmm_recompute(h)
    torch.cuda.synchronize()
    recompute_s = time.perf_counter() - t_r

    # the one-off M2L's product kernels, timed by the library's events (into scratch: state unchanged)
    m2l_levels, m2l_total_ms = k.kmc_fmm_m2l_timed(h, 3)

    # FP64 form (context)
    fp64 = None
    if args.fp64_steps > 0:
        del h
        torch.cuda.synchronize()
        h64 = k.kmc_fmm_init(pos, q, float(E), L, p, precision="fp64", lattice_edge=E, kT=kT, stream=stream, hops=nhop,
                             bc=args.bc, field_z=fz,
                             device=dev)
        k.kmc_run_profiled(h64, u[:1])
        ms64 = []
        ph64 = np.zeros(k.KMC_NPHASE)
        for s in range(args.fp64_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, ph = k.kmc_run_profiled(h64, u[1 + s: 2 + s])
            e1.record(stream)
            e1.synchronize()
            ms64.append(float(ph.sum()))
            ph64 += ph
        m64 = float(np.mean(ms64))
        fp64 = {"dU_evals_per_s": hops / (m64 * 1e-3), "kmc_steps_per_s": 1e3 / m64, "ms_per_step": m64,
                "propose_ms": ph64[1] / args.fp64_steps, "steps": args.fp64_steps}
        del h64

    # near-field cache form (kmc_opts.near_cache: every site's near-field sum kept on the device and
    # updated per accepted move; proposals read it instead of summing the pairs).  Reported beside
    # the headline, which sums the 27-leaf pairs in every step; timed the same way.
    ncache = None
    if args.near_cache_steps > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hc = k.kmc_fmm_init(pos, q, float(E), L, p, precision="mixed", lattice_edge=E, kT=kT, stream=stream,
                            device=dev, hops=nhop, bc=args.bc, field_z=fz, near_cache=True)
        torch.cuda.synchronize()
        init_c = time.perf_counter() - t0
        k.kmc_run_profiled(hc, u[: args.warmup])
        msc, phc = [], np.zeros(k.KMC_NPHASE)
        for s in range(args.near_cache_steps):
            flush.zero_()
            _, _, ph = k.kmc_run_profiled(hc, u[args.warmup + s: args.warmup + s + 1])
            msc.append(float(ph.sum()))
            phc += ph
        mc = float(np.mean(msc))
        ncache = {"dU_evals_per_s": hops / (mc * 1e-3), "kmc_steps_per_s": 1e3 / mc, "ms_per_step": mc,
                  "phase_ms_per_step": {nm: phc[i] / args.near_cache_steps for i, nm in enumerate(k.PHASES)},
                  "init_s": init_c, "steps": args.near_cache_steps, "dtype": "f32-mixed",
                  "what": "same workload and step; near-field sums kept per site (int64 fixed point, "
                          f"{8 * w['E'] ** 3 / 2 ** 20:.0f} MiB) and updated per accepted move"}
        del hc

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the propose kernel: MUFU rsqrt per pair is the binding unit
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mufu_peak = 16 * nsm * sm_max * 1e6  # rsqrt/s
    pairs = work["pairs"]
    achieved = pairs / (prop_ms * 1e-3)
    # FP32 pipes: one FMA per pair (the squared distances come from the tensor cores) and the L2P
    fp32_ops = 2 * pairs + l2p_flops(p) * work["points"]
    fma_peak = 128 * nsm * sm_max * 1e6
    t_mufu = pairs / mufu_peak
    t_fma = fp32_ops / fma_peak
    roof = {"bound": "alu", "kernel": "k_propose_lattice<float>",
            "achieved": achieved / 1e9, "peak": mufu_peak / 1e9, "unit": "G pair-interactions/s (MUFU rsqrt)",
            "work": "pairs = distinct evaluation sites x charges in the 27 neighbouring leaves",
            "frac": achieved / mufu_peak,
            "traffic": (PROPOSE_DRAM_BYTES_PER_LEAF * work["leaves"]
                        if args.workload in TRAFFIC_WORKLOADS and args.bc == "periodic" else None),
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 128^3 tile case "
                               "(same leaf shape), scaled by leaves" if args.workload in TRAFFIC_WORKLOADS
                               and args.bc == "periodic" else None),
            "peak_source": f"16 MUFU/clk/SM x {nsm} SMs x {sm_max:.0f} MHz ({src} max clock)",
            "pairs_per_launch": pairs, "points_per_launch": work["points"],
            "fp32_ops_per_launch": fp32_ops, "tensor_f16_flops_per_launch": 16 * pairs,
            "t_min_ms": 1e3 * max(t_mufu, t_fma), "t_meas_ms": prop_ms,
            "frac_of_alu_bound": 1e3 * max(t_mufu, t_fma) / prop_ms}

    rooflines = phase_rooflines(work, {nm: phases[i] / args.steps for i, nm in enumerate(k.PHASES)}, E, L, len(q),
                                p, nhop, peaks, nsm, mixed=True)
    rooflines["propose"] = {kk: roof[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac")}
    rooflines["m2l"] = m2l_roofline(m2l_levels, m2l_total_ms, L, p, peaks, precision="mixed")
    if fp64 is not None:
        # FP64 form: one FP64 FMA per pair (the lattice-table near field), at 2 FMA/clk/SM
        fp64_peak = 2 * 2 * nsm * sm_max * 1e6
        a64 = 2 * work["pairs"] / (fp64["propose_ms"] * 1e-3)
        rooflines["propose_fp64_form"] = {"kernel": "k_propose_lattice<double>", "bound": "alu", "unit": "TFLOP/s",
                                          "achieved": a64 / 1e12, "peak": fp64_peak / 1e12, "frac": a64 / fp64_peak,
                                          "work": "one FP64 FMA (2 flops) per pair"}
    cpu = None
    if not args.no_cpu and world == 1 or (world > 1 and rank == 0 and not args.no_cpu):
        direct = cpu_sample(E, sites, q, seconds_target=args.cpu_seconds, nhop=nhop, bc=args.bc)
        if nhop == 6 and args.bc == "periodic":
            # the O-table form is the strongest CPU algorithm for a lattice: it is the headline baseline
            ot, _ = cpu_otable(E, sites, q, kT, w["seed"], seconds_target=args.cpu_seconds)
            cpu = dict(ot, forms={"o_table": dict(ot), "o_direct": direct})
        else:
            cpu = dict(direct, forms={"o_direct": direct})

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_MIXED,
        "data": "synthetic", "config": dict(_config(w, args.workload), parallelism=f"replicas x{world}",
                                            bc=args.bc),
        "kmc_steps_per_s": steps_per_s,
        "propose_only_dU_evals_per_s": hops / (prop_ms * 1e-3),
        "phase_ms_per_step": {nm: phases[i] / args.steps for i, nm in enumerate(k.PHASES)},
        "ms_per_step_incl_call_overhead": float(np.mean(outer_ms)),
        "init_s": init_s, "recompute_s": recompute_s,
        "fp64_form": fp64,
        "near_cache_form": ncache,
        "roofline": roof,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step(L, args.bc) * args.steps,
        "paper_context": PAPER_SEC53 if args.workload == "sec53" else None,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """Batched replicas: independent lattice systems of uneven sizes (edges from
    {32, 48, 64, 96, 128}, occupancy U[0.02, 0.15]) advanced together by the
    batched kernels (every launch covers all replicas); L per replica and the
    batch's P2P tile from the autotuner.  The value is device-timed (CUDA events
    around the K graph-replayed steps); e2e is the host wall clock of the same
    call (uniform staging and event read-back included)."""
    import torch
    import paper_1905_04065_gb300 as k
    from paper_1905_04065_gb300 import autotune

    rank, world, local = _dist()
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    B = workloads.BATCH
    nrep = args.replicas or B["replicas"]
    reps = workloads.batch_replicas(nrep, first=rank * nrep)  # each rank its own replicas
    p, kT = B["p"], B["kT"]
    t0 = time.perf_counter()
    levels, hops, pairs = [], 0, 0
    for r in reps:
        pos = workloads.site_positions(r["E"], r["sites"])
        L = autotune.tune_levels(r["E"], pos, r["q"], p, "mixed", kT) if not args.no_tune else \
            autotune.valid_levels(r["E"])[0]
        levels.append(L)
        pc = pair_count(r["E"], L, r["sites"])
        hops += pc["hops"]
        pairs += pc["pairs"]

    def make(precision):
        return [k.kmc_fmm_init(workloads.site_positions(r["E"], r["sites"]), r["q"], float(r["E"]), L, p,
                               precision=precision, lattice_edge=r["E"], kT=kT, device=dev)
                for r, L in zip(reps, levels)]
    handles = make("mixed")
    torch.cuda.synchronize()
    ws = sum(step_bytes(r["E"], L, r["N"], p) for r, L in zip(reps, levels))
    setup_s = time.perf_counter() - t0
    bat = k.kmc_batch_create(handles)
    R = len(handles)
    tune = autotune.tune_batch_chunk(bat) if not args.no_tune else (k.kmc_batch_info(bat)["chunk"], {})
    info = k.kmc_batch_info(bat)
    rng = np.random.default_rng(B["seed"] + 17)
    u = 1.0 - rng.random((args.warmup + args.steps, R, 2))
    k.kmc_batch_run(bat, u[: args.warmup])
    # the replicas' working set (rates, expansions, charges) exceeds the 129 MB
    # L2, so the K timed steps run as one call: the graph is replayed K / 8 times
    clk = Clocks(dev)
    os.makedirs(args.clocks_dir, exist_ok=True)
    clk.start(os.path.join(args.clocks_dir, f"clocks_batch_rank{rank}.csv"))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    _, _, dev_ms = k.kmc_batch_run(bat, u[args.warmup: args.warmup + args.steps], timed=True)
    wall_ms = 1e3 * (time.perf_counter() - t1)
    clocks = clk.stop()
    prop_ms = k.kmc_batch_propose_timed(bat, 10) if info["fused"] else None
    units, tot = aggregate(hops * args.steps, dev_ms, device=f"cuda:{dev}")
    e2e_units, e2e_tot = aggregate(hops * args.steps, wall_ms, device=f"cuda:{dev}")
    del bat
    # FP64 form of the same batch (context: the mixed form's speed-up)
    fp64 = None
    if args.fp64_steps > 0:
        del handles
        torch.cuda.synchronize()
        h64 = make("fp64")
        b64 = k.kmc_batch_create(h64)
        u64 = 1.0 - rng.random((1 + args.fp64_steps, R, 2))
        k.kmc_batch_run(b64, u64[:1])
        _, _, ms64 = k.kmc_batch_run(b64, u64[1:], timed=True)
        fp64 = {"dU_evals_per_s": hops * args.fp64_steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.fp64_steps,
                "steps": args.fp64_steps}
        del b64, h64
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu:
        # the oracle's O-table form: one full KMC step of every replica (one batch step), host cores
        import oracle
        ch, ct, ns = 0, 0.0, 0
        for r in reps:
            st = oracle.LatticeState(r["E"], r["sites"], r["q"])
            t0 = time.perf_counter()
            dU, mask = st.propose()
            j, Q, dt = oracle.select(oracle.rates(dU, mask, kT), 0.5, 0.5)
            if j >= 0:
                st.accept(j // 6, j % 6)
            ct += time.perf_counter() - t0
            ch += int(mask.sum())
            ns += 1
        cpu = {"value": ch / ct, "unit": UNIT, "kmc_steps_per_s": 1.0 / ct, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"one full KMC step of each of the {ns} replicas (one batch step) in the "
                                           "O-table form (lattice-table Ewald potential, O(1) dU per hop, sequential "
                                           "FP64 selection, O(E^3) site update per accept); kmc_steps_per_s = batch "
                                           "steps per second"}
    value = units / (tot * 1e-3)
    roof = None
    if prop_ms:
        peaks, src = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mufu_peak = 16 * nsm * sm_max * 1e6
        roof = {"bound": "alu", "kernel": "k_propose_batch<float> (every member's leaves, one launch per pass "
                                          "capacity class)",
                "achieved": pairs / (prop_ms * 1e-3) / 1e9, "peak": mufu_peak / 1e9,
                "unit": "G pair-interactions/s (MUFU rsqrt)", "frac": pairs / (prop_ms * 1e-3) / mufu_peak,
                "traffic": None, "pairs_per_launch": pairs, "t_meas_ms": prop_ms,
                "work": "pairs = distinct evaluation sites x charges in the 27 neighbouring leaves, summed over "
                        "the replicas (initial configuration)",
                "timing": "the batch step's propose launches alone, 10 times, CUDA events on the batch stream",
                "peak_source": f"16 MUFU/clk/SM x {nsm} SMs x {sm_max:.0f} MHz ({src} max clock)"}
    line = {
        "metric": "dU evals/sec and KMC steps/sec, 64 batched replicas", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_MIXED, "data": "synthetic",
        "config": {"workload": f"batch: {R} replicas, edges {sorted(set(r['E'] for r in reps))}, occupancy "
                               f"U[0.02,0.15], {sum(r['N'] for r in reps)} charges in total, p={p}, kT={kT}",
                   "levels": levels, "working_set_bytes": ws, "p2p_chunk": info["chunk"],
                   "chunk_ms_per_step": {str(c): t for c, t in tune[1].items()},
                   "timing": "CUDA events on the batch's stream around the K graph-replayed steps; working set "
                             "larger than L2, no flush"},
        "kmc_steps_per_s": world * args.steps / (tot * 1e-3),
        "replica_steps_per_s": world * R * args.steps / (tot * 1e-3), "setup_s": setup_s,
        "fp64_form": fp64,
        "mixed_over_fp64": (value / fp64["dU_evals_per_s"]) if fp64 else None,
        "e2e": {"value": e2e_units / (e2e_tot * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 16 * R, "d2h_bytes_per_step": 16 * R,
                "path": "kmc_batch_run from host uniforms to host events and time increments"},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "gpu_launches": info["launches_per_step"] * args.steps,
        "batched_kernels": info["fused"],
        "roofline": roof,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--bc", default="periodic", choices=["periodic", "free", "dirichlet"],
                    help="boundary conditions of the lattice workloads (the configs are periodic)")
    ap.add_argument("--workload", default="large", choices=["small", "medium", "large", "blobs", "tile", "sec53", "batch"])
    ap.add_argument("--replicas", type=int, default=None)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="directory for the nvidia-smi clock samples of the timed region")
    ap.add_argument("--near-cache-steps", type=int, default=20,
                    help="steps of the near-field cache form reported beside the headline (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-props", type=int, default=2048)
    args = ap.parse_args()
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps >= 1 and --warmup >= 0 required")
    if args.impl == "reference":
        if args.workload == "batch":
            args.workload = "medium"
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
