"""The allocation-free selection entry point (kmc_select_static) gives the
same event, dt and Q as kmc_step on the same rates and uniforms.

It exists for callers that cannot allocate device memory (code running during
a global-mode graph capture, inside a framework-owned memory pool, or in loops
that must not stall on an allocation); its scratch is a static device array.
This file is collected last so that a failure here does not hide the others."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_static_select_matches_kmc_step_two_calls():
    import torch

    import paper_1905_04065_gb300 as k

    w, sites, q = workloads.workload("small")
    E = w["E"]
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), w["L"], 8, lattice_edge=E, kT=w["kT"])
    n = len(q)
    rng = np.random.default_rng(123)
    for call in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
        r = rng.random(6 * n)
        r[rng.random(6 * n) < 0.5] = 0.0
        zeta, xi = 1.0 - rng.random(), 1.0 - rng.random()
        ev1, dt1, Q1 = k.kmc_step(h, r, zeta, xi)
        rt = torch.tensor(r, dtype=torch.float64, device="cuda")
        ev2, dt2, Q2 = k.kmc_select_static(rt, n, zeta, xi)
        assert ev2 == ev1, (call, ev1, ev2)
        assert abs(Q2 - Q1) <= 1e-12 * Q1
        assert abs(dt2 - dt1) <= 1e-12 * dt1
    k.kmc_fmm_destroy(h)


def test_static_select_rejects_sizes_beyond_its_scratch():
    import torch

    import paper_1905_04065_gb300 as k

    rt = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(k.KmcError):
        k.kmc_select_static(rt, k.KMC_STATIC_MAX_N + 1, 0.5, 0.5)
    with pytest.raises(k.KmcError):
        k.kmc_select_static(rt, 0, 0.5, 0.5)
