"""The checked build (-DKMC_CHECKS: the device-side bounds checks of the propose, rates, accept
and near-field-cache kernels compiled in; the substitute for compute-sanitizer, which is not
available): every mode runs through it without a failed check, and its results equal the
normal build's.  Runs in a subprocess so that the checked library is the only one loaded."""
import ast
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1905_04065_gb300 as k
from paper_1905_04065_gb300 import build
k.load_library(build.build(checked=True))
import workloads

def system(E, n, seed, lower=False):
    rng = np.random.default_rng(seed)
    pool = np.nonzero(np.arange(E ** 3) // (E * E) < E // 2)[0] if lower else np.arange(E ** 3)
    sites = rng.choice(pool, n, replace=False)
    q = np.where(rng.permutation(n) % 2 == 0, 1.0, -1.0)
    return sites, q

out = []
cases = [("fp64", 6, "periodic", False), ("mixed", 6, "periodic", False), ("mixed", 14, "periodic", False),
         ("fp64", 14, "free", False), ("mixed", 6, "dirichlet", False), ("mixed", 6, "periodic", True),
         ("fp64", 14, "periodic", True), ("mixed", 14, "dirichlet", True)]
for prec, nh, bc, nc in cases:
    E, L = 16, 3
    sites, q = system(E, 400, 11 + nh, lower=(bc == "dirichlet"))
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, 8, precision=prec, lattice_edge=E,
                       kT=0.1, hops=nh, bc=bc, field_z=0.2 if bc == "dirichlet" else 0.0, near_cache=nc)
    mask, dU = k.kmc_fmm_propose_lattice(h)
    ev, dt, Q = k.kmc_step(h, None, 0.37, 0.61)
    k.kmc_fmm_accept_event(h, ev)
    evs, dts = k.kmc_run(h, workloads.uniforms(25, 99))
    mask2, dU2 = k.kmc_fmm_propose_lattice(h)
    if bc != "dirichlet":  # general proposals of three charges to empty sites
        occ = set((np.floor(k.kmc_fmm_positions(h)) @ np.array([1, E, E * E])).astype(int).tolist())
        empty = [s for s in range(E ** 3) if s not in occ][:3]
        k.kmc_fmm_propose(h, np.array([0, 1, 2], np.int32), workloads.site_positions(E, empty))
    drift = k.kmc_fmm_recompute(h)
    out.append((prec, nh, bc, nc, float(np.nansum(dU)), float(np.nansum(dU2)), evs.tolist()))
print("RESULTS", repr(out))
print("checked ok")
'''


def _run(lib_checked: bool):
    script = SCRIPT.replace("ROOT", repr(ROOT))
    if not lib_checked:
        script = script.replace("k.load_library(build.build(checked=True))", "k.load_library()")
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULTS")][0]
    return ast.literal_eval(line[len("RESULTS "):])


def test_checked_build_runs_every_mode_clean():
    checked, normal = _run(True), _run(False)
    assert len(checked) == len(normal) == 8
    for a, b in zip(checked, normal):
        assert a[:4] == b[:4] and a[6] == b[6], (a[:4], a[6], b[6])  # same case, same events
        for x, y in ((a[4], b[4]), (a[5], b[5])):
            assert abs(x - y) <= 1e-9 * max(abs(y), 1.0), (a[:4], x, y)

