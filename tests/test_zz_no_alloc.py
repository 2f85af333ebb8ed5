"""The allocation-free selection entry point (kmc_select_static) gives the
same event, dt and Q as kmc_step on the same rates and uniforms.

It exists for callers that cannot allocate device memory (a library inside a
framework whose caching allocator owns the device, host loops that must not
stall on the synchronisation an allocation can cause, plugin hosts that forbid
their plugins to own device memory); its scratch is a static device array.
This file is collected last so that a failure here does not hide the others."""
import numpy as np
import pytest

import oracle
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
    # a rates buffer shorter than 6 n entries is refused before the library reads past it
    with pytest.raises(k.KmcError) as e:
        k.kmc_select_static(rt, 2, 0.5, 0.5)
    assert e.value.code == k.KMC_ERR_ARG


def test_static_select_large_n_matches_oracle():
    """n = 2^21 particles (12.6 M sparse rates, 16384 block sums of the static
    array, 16 per selection thread): event, dt and Q against the oracle's
    sequential FP64 selection, on two calls in a row."""
    import torch

    import paper_1905_04065_gb300 as k

    n = 1 << 21
    rng = np.random.default_rng(321)
    for call in range(2):
        r = rng.random(6 * n)
        r[rng.random(6 * n) < 0.7] = 0.0
        zeta, xi = 1.0 - rng.random(), 1.0 - rng.random()
        j, Q_o, dt_o = oracle.select(r, zeta, xi)
        R = oracle.cumsum(r)
        # the uniform must not fall within rounding of a cumulative boundary (not for this seed)
        assert np.min(np.abs(R - Q_o * zeta)) > 1e-11 * Q_o
        rt = torch.tensor(r, dtype=torch.float64, device="cuda")
        ev, dt, Q = k.kmc_select_static(rt, n, zeta, xi)
        assert ev == j, (call, ev, j)
        assert abs(Q - Q_o) <= 1e-12 * Q_o
        assert abs(dt - dt_o) <= 1e-12 * dt_o
