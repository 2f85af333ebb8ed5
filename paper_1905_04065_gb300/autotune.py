"""Leaf-level autotuner for lattice systems.

The number of FMM levels L sets the leaf width W = E / 2^(L-1) and so the
balance between the near-field pair sums (∝ charges per leaf) and the
expansion work (∝ leaves).  For a lattice system the tuner times a few device
steps for every valid L and keeps the fastest, caching the choice per GPU,
lattice edge, occupancy bucket, order and precision in a JSON file beside
this module.

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
