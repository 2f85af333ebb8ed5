"""Run a lattice KMC simulation and log it as JSON lines.

    python -m paper_1905_04065_gb300.run --workload medium --steps 1000 --recompute-every 100 \
        --log run.jsonl [--precision mixed] [--near-cache] [--checkpoint ckpt.npz] [--resume ckpt.npz]

The steps run on the device in chunks (one CUDA-graph replay per chunk, `kmc_run`); after each
chunk a full FMM recompute reports the drift of the incrementally updated state (the check the
method needs for its accumulated accept updates), and one JSON line records: steps done, wall time,
KMC steps/s and dU evaluations/s of the chunk, simulated time, tracked energy and the three drift
figures (potential at the charges, expansion coefficients, energy).  The uniform stream is seeded,
so a run resumed from a checkpoint continues the same stream.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import (kmc_checkpoint, kmc_fmm_energy, kmc_fmm_init, kmc_fmm_propose_lattice, kmc_fmm_recompute,
               kmc_resume, kmc_run)


def _workload(name: str):
    import workloads
    w, sites, q = workloads.workload(name)
    return w, workloads.site_positions(w["E"], sites), q


def _uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """(zeta, xi) pairs start..start+count of a seeded stream in (0, 1], counter based, so that
    any window can be drawn on its own (a resumed run continues the same stream)."""
    out = np.empty((count, 2))
    for s in range(count):
        rng = np.random.default_rng([seed, start + s])
        out[s] = 1.0 - rng.random(2)
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="medium")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--recompute-every", type=int, default=100)
    ap.add_argument("--near-cache", action="store_true")
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--log", default="-", help="JSON-lines file ('-': standard output)")
    ap.add_argument("--checkpoint", default=None, help="write a checkpoint here after every chunk")
    ap.add_argument("--resume", default=None, help="continue from this checkpoint")
    args = ap.parse_args(argv)
    if args.steps < 0 or args.recompute_every < 1:
        ap.error("steps must be >= 0 and recompute-every >= 1")

    t0 = time.perf_counter()
    if args.resume:
        h, step, extra = kmc_resume(args.resume)
        sim_time = float(extra.get("sim_time", 0.0))
    else:
        w, pos, q = _workload(args.workload)
        h = kmc_fmm_init(pos, q, float(w["E"]), w["L"], w["p"], precision=args.precision, lattice_edge=w["E"],
                         kT=w["kT"], hops=w.get("hops", 6), near_cache=args.near_cache)
        step, sim_time = 0, 0.0
    init_s = time.perf_counter() - t0
    log = sys.stdout if args.log == "-" else open(args.log, "a")
    log.write(json.dumps({"event": "start", "step": step, "init_s": init_s, "energy": kmc_fmm_energy(h),
                          "workload": args.workload, "precision": args.precision,
                          "near_cache": args.near_cache, "resumed": bool(args.resume)}) + "\n")
    end = step + args.steps
    while step < end:
        n = min(args.recompute_every, end - step)
        mask, _ = kmc_fmm_propose_lattice(h)  # proposals per step (changes little within a chunk)
        hops = int(np.asarray(mask.cpu() if hasattr(mask, "cpu") else mask).sum())
        u = _uniforms(args.seed, step, n)
        t1 = time.perf_counter()
        events, dts = kmc_run(h, u)
        wall = time.perf_counter() - t1
        step += n
        sim_time += float(np.sum(dts[np.isfinite(dts)]))
        drift = kmc_fmm_recompute(h)
        rec = {"event": "chunk", "step": step, "wall_s": wall, "kmc_steps_per_s": n / wall,
               "dU_evals_per_s": hops * n / wall, "sim_time": sim_time, "energy": kmc_fmm_energy(h),
               "drift_potential": float(drift[0]), "drift_coefficients": float(drift[1]),
               "drift_energy": float(drift[2]), "no_event_steps": int(np.sum(events < 0))}
        log.write(json.dumps(rec) + "\n")
        log.flush()
        if args.checkpoint:
            kmc_checkpoint(h, args.checkpoint, step=step, sim_time=sim_time)
    if log is not sys.stdout:
        log.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
