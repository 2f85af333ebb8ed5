"""Autotuner for lattice systems and replica batches.

Leaf tile: the number of FMM levels L sets the leaf width W = E / 2^(L-1) and
so the balance between the near-field pair sums (∝ charges per leaf) and the
expansion work (∝ leaves).  For a lattice system the tuner times a few device
steps for every valid L and keeps the fastest, caching the choice per GPU,
lattice edge, occupancy bucket, order and precision in a JSON file beside
this module.

P2P tile of a batch: the batched propose stages the charges of a leaf's 27
neighbour leaves in shared memory in passes of `chunk` sources; a larger pass
needs fewer passes in dense neighbourhoods but more shared memory per CTA
(fewer resident CTAs).  tune_batch_chunk times the batch's step for a few
pass capacities and keeps the fastest.

Valid L: at least 4 leaves per side (L >= 3) and 2 <= W <= 12 sites per leaf
side (the propose kernel keeps a leaf's sites in shared memory).
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "tuned_levels.json")
_lock = threading.Lock()


def valid_levels(E: int):
    out = []
    for L in range(3, 11):
        nL = 2 ** (L - 1)
        if E % nL == 0 and 2 <= E // nL <= 12:
            out.append(L)
    return out


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _key(E: int, n: int, p: int, precision: str) -> str:
    occ = n / float(E ** 3)
    bucket = round(float(np.log2(max(occ, 1e-6))) * 2) / 2  # half-octave occupancy buckets
    return f"{_gpu_name()}|E{E}|occ2^{bucket:+.1f}|p{p}|{precision}"


def _load() -> dict:
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            return json.load(f)
    return {}


def _store(table: dict) -> None:
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_levels(E: int, positions, charges, p: int, precision: str = "mixed", kT: float = 0.05,
                steps: int = 3, use_cache: bool = True, record: bool = True) -> int:
    """Fastest number of levels for this lattice system (device-timed steps)."""
    import paper_1905_04065_gb300 as k

    cands = valid_levels(E)
    if not cands:
        raise ValueError(f"no valid level count for lattice edge {E}")
    if len(cands) == 1:
        return cands[0]
    key = _key(E, len(charges), p, precision)
    with _lock:
        table = _load() if use_cache else {}
    if key in table:
        return int(table[key]["L"])
    rng = np.random.default_rng(99)
    u = 1.0 - rng.random((2 + steps, 2))
    times = {}
    for L in cands:
        h = k.kmc_fmm_init(positions, charges, float(E), L, p, precision=precision, lattice_edge=E, kT=kT)
        k.kmc_run_profiled(h, u[:2])
        _, _, ph = k.kmc_run_profiled(h, u[2:])
        times[L] = float(np.sum(ph)) / steps
        k.kmc_fmm_destroy(h)
    best = min(times, key=times.get)
    if record:
        with _lock:
            table = _load()
            table[key] = {"L": best, "ms_per_step": {str(L): t for L, t in times.items()}}
            _store(table)
    return best


def tune_batch_chunk(b, steps: int = 8, factors=(1.0, 1.5, 2.0), seed: int = 5):
    """Pick the batched propose's pass capacity (the P2P tile) by device-timing `steps` batch
    steps per candidate: 0 (each member its smallest capacity, members grouped by capacity into
    one propose launch per group) and multiples of the largest member's smallest capacity (one
    launch for all).  The timed steps are real KMC steps of the batch (its members advance).
    Returns (chosen request, {request: ms per step})."""
    import paper_1905_04065_gb300 as k

    info = k.kmc_batch_info(b)
    if not info["fused"]:
        return 0, {}
    k.kmc_batch_set_chunk(b, 0)
    base = k.kmc_batch_info(b)["chunk"]
    cands = [0] + sorted({int(2 * round(base * f / 2)) for f in factors})
    rng = np.random.default_rng(seed)
    R = len(b.handles)
    times = {}
    for c in cands:
        k.kmc_batch_set_chunk(b, c)
        k.kmc_batch_run(b, 1.0 - rng.random((2, R, 2)))  # graph capture, warm-up
        _, _, ms = k.kmc_batch_run(b, 1.0 - rng.random((steps, R, 2)), timed=True)
        times[c] = ms / steps
    best = min(times, key=times.get)
    k.kmc_batch_set_chunk(b, best)
    return best, times
