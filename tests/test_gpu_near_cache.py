"""The near-field cache (kmc_opts.near_cache): every site's near-field sum (the
direct part of the potential over the 27 leaves around the site's leaf, Sec. 3)
kept on the device and updated per accepted move, against the oracle and
against the handle that sums the pairs every step.

Tolerances.  Against the oracle: the p-dependent bounds of the summed path
(the cache changes only the rounding of the near field).  Cached against summed
on the same configuration: FP64 to 1e-9 of max|dU| (both near fields are exact
to ~1e-14; the fixed-point cache rounds at 2^-k, 2^k x bound < 2^61); FP32 to
2e-5 (the summed near field carries FP32 rounding of a few 1e-7 of the largest
partial sums, the cache carries the FP32 sums of its fill plus exact updates).
Masks and positions are compared exactly.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = {8: 2e-3, 12: 1e-4}


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _init(E, sites, q, L, p, precision, kT, hops=6, near_cache=True, **kw):
    k = _k()
    return k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision=precision,
                          lattice_edge=E, kT=kT, hops=hops, near_cache=near_cache, **kw)


def _near_tie(dU, mask, kT, zeta, tol_abs):
    r = oracle.rates(dU, mask, kT)
    R = oracle.cumsum(r)
    Q = R[-1]
    return np.min(np.abs(R - Q * zeta)) <= float(np.sum(r) * tol_abs / kT) + 1e-12 * Q


def _oracle_hops(st, nh):
    """dU (NaN where masked), mask and target sites of every hop, j = nh i + k."""
    tg = oracle.hop_targets(st.E, st.sites, nh).reshape(-1)
    mask = (st.occ[tg] == 0).astype(np.uint8)
    ok = mask.astype(bool)
    dU = np.full(len(tg), np.nan)
    dU[ok] = st.delta_u_list(np.repeat(np.arange(st.n), nh)[ok], tg[ok])
    return dU, mask, tg


@pytest.mark.parametrize("precision,nh", [("fp64", 6), ("mixed", 6), ("mixed", 14)])
def test_cached_trajectory_against_oracle(precision, nh):
    """Masks exactly and every dU within the p = 12 bound against the oracle at
    every step of a 25-step trajectory (the oracle's event accepted on both
    sides), events compared except near ties, energy and positions at the end."""
    k = _k()
    w, sites, q = workloads.workload("small")
    E, kT, p = w["E"], w["kT"], 12
    st = oracle.LatticeState(E, sites, q)
    h = _init(E, sites, q, w["L"], p, precision, kT, hops=nh)
    u = workloads.uniforms(25, w["seed"] + 77)
    agree = 0
    for s in range(25):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o, tg = _oracle_hops(st, nh)
        assert np.array_equal(mask.reshape(-1), mask_o)
        ok = mask_o.astype(bool)
        tol = TOL[p] * np.max(np.abs(dU_o[ok]))
        assert np.max(np.abs(dU.reshape(-1)[ok] - dU_o[ok])) < tol, s
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        j, Q_o, dt_o = oracle.select(oracle.rates(dU_o, mask_o, kT), u[s, 0], u[s, 1])
        if ev == j:
            agree += 1
        else:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], tol), (s, ev, j)
        du_acc = k.kmc_fmm_accept_event(h, j)
        assert abs(du_acc - dU_o[j]) < tol
        st.accept_site(j // nh, tg[j])
    assert agree >= 23
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-4 * abs(st.energy())


def _same_history(precision, steps, seed):
    """A cached handle after `steps` graph-replayed steps (64^3 lattice, 32768
    charges, 8^3-site leaves) and a summing handle given the same accepted
    events, so that both hold the same incrementally updated far field."""
    k = _k()
    w, sites, q = workloads.workload("medium")
    E, kT, L = w["E"], w["kT"], w["L"]
    hc = _init(E, sites, q, L, 12, precision, kT, near_cache=True)
    hs = _init(E, sites, q, L, 12, precision, kT, near_cache=False)
    ev, _ = k.kmc_run(hc, workloads.uniforms(steps, seed))
    for j in ev:
        if j >= 0:
            k.kmc_fmm_accept_event(hs, int(j))
    pos = k.kmc_fmm_positions(hc)
    assert np.array_equal(pos, k.kmc_fmm_positions(hs))
    moved = int(np.sum(np.any(pos != workloads.site_positions(E, sites), axis=1)))
    return hc, hs, moved


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_cached_equals_summed_after_device_loop(precision, tol):
    """300 steps: the proposals from the cached near fields against those of the
    handle that sums the pairs, on the same configuration and far field."""
    k = _k()
    hc, hs, moved = _same_history(precision, 300, 9090)
    assert moved > 100
    mask_c, dU_c = k.kmc_fmm_propose_lattice(hc)
    mask_s, dU_s = k.kmc_fmm_propose_lattice(hs)
    assert np.array_equal(mask_c, mask_s)
    ok = mask_s.astype(bool)
    err = float(np.max(np.abs(dU_c[ok] - dU_s[ok])) / np.max(np.abs(dU_s[ok])))
    assert err < tol, err
    print(f"cached vs summed after 300 steps ({precision}): {err:.2e} of max|dU|, {moved} charges moved")


def test_recompute_refills_cache():
    """kmc_fmm_recompute fills the cache afresh: after the same 200 accepted
    moves the cached and the summing handle report the same potential drift
    (tracked against recomputed, which the far field's incremental updates
    dominate), so the cache has carried no error of its own."""
    k = _k()
    hc, hs, _ = _same_history("fp64", 200, 5151)
    dc = k.kmc_fmm_recompute(hc)
    ds = k.kmc_fmm_recompute(hs)
    assert dc[0] < 1e-4 and abs(dc[0] - ds[0]) < 1e-11, (dc, ds)
    mask_c, dU_c = k.kmc_fmm_propose_lattice(hc)
    mask_s, dU_s = k.kmc_fmm_propose_lattice(hs)
    ok = mask_s.astype(bool)
    assert np.max(np.abs(dU_c[ok] - dU_s[ok])) < 1e-11 * np.max(np.abs(dU_s[ok]))


@pytest.mark.parametrize("bc", ["free", "dirichlet"])
def test_cached_equals_summed_other_boundaries(bc):
    """Free space and grounded walls: 60 graph-replayed steps on a cached and a
    summing handle from the same start (FP64, same uniforms) reach the same
    configuration, where their proposals agree."""
    k = _k()
    E, L, p, kT = 16, 3, 12, 0.1
    rng = np.random.default_rng(31)
    if bc == "dirichlet":
        lower = np.nonzero(np.arange(E ** 3) // (E * E) < E // 2)[0]
        sites = rng.choice(lower, 400, replace=False)
        kw = dict(bc="dirichlet", field_z=0.2)
    else:
        sites = rng.choice(E ** 3, 400, replace=False)
        kw = dict(bc="free")
    q = np.where(rng.permutation(400) % 2 == 0, 1.0, -1.0)
    u = workloads.uniforms(60, 6060)
    hc = _init(E, sites, q, L, p, "fp64", kT, near_cache=True, **kw)
    hs = _init(E, sites, q, L, p, "fp64", kT, near_cache=False, **kw)
    ev_c, _ = k.kmc_run(hc, u)
    ev_s, _ = k.kmc_run(hs, u)
    assert np.array_equal(ev_c, ev_s)
    assert np.array_equal(k.kmc_fmm_positions(hc), k.kmc_fmm_positions(hs))
    mc, dc = k.kmc_fmm_propose_lattice(hc)
    ms, ds = k.kmc_fmm_propose_lattice(hs)
    assert np.array_equal(mc, ms)
    ok = ms.astype(bool)
    assert np.max(np.abs(dc[ok] - ds[ok])) < 1e-9 * np.max(np.abs(ds[ok]))
    assert abs(k.kmc_fmm_energy(hc) - k.kmc_fmm_energy(hs)) < 1e-9 * abs(k.kmc_fmm_energy(hs))


def test_near_cache_needs_lattice_mode():
    k = _k()
    pos = np.array([[0.5, 0.5, 0.5], [2.5, 1.5, 0.5]])
    with pytest.raises(k.KmcError) as ei:
        k.kmc_fmm_init(pos, np.array([1.0, -1.0]), 4.0, 3, 4, near_cache=True)
    assert ei.value.code == k.KMC_ERR_ARG
