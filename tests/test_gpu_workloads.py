"""Parity of the CUDA path with the FP64 oracle on the medium and large
lattice workloads, in the configuration the benchmark times.

medium (64^3 sites, 32768 charges, L=4, p=12): every dU of every step of a
1000-step teacher-forced trajectory (the oracle's event is accepted on both
sides), with a full recompute every 100 steps to measure the accept-update
drift, in the FP64 and the mixed form.

large (256^3 sites, 1,048,576 charges, L=6, p=12, mixed precision -- the
benchmark's launch configuration): every dU and mask of one propose against
the oracle's lattice table, plus a sample of the oracle's own O(N) direct sum.

Tolerances at p = 12 are the measured truncation error, stated against
max |dU| (the targets 1e-6 FP64 / 1e-4 mixed are asserted at the orders that
meet them in test_gpu_contract.py).  The bulk of the distribution is tight
(99th percentile below 1e-5, mean ~5e-7); the largest errors belong to hops
across the boundary of a level-2 or level-3 cell, where the truncation errors
of those levels' M2L translations between distance-two cells do not cancel
between the old and the new site: 8e-5 on the medium workload (so the mixed
form meets its 1e-4 target there), 1.55e-4 on the large one.  Masks and
selected events are compared exactly (events except near ties)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL12 = 2.5e-4    # max over all hops, p = 12, large workload (measured 1.55e-4)
TOL12_MEDIUM = 1e-4  # max over all hops, p = 12, medium workload (measured 8.3e-5 over 1000 steps)
TOL12_P99 = 1e-5  # 99th percentile, p = 12


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _near_tie(dU_o, mask_o, kT, zeta, tol_abs):
    r = oracle.rates(dU_o, mask_o, kT)
    R = oracle.cumsum(r)
    Q = R[-1]
    slack = float(np.sum(r) * tol_abs / kT) + 1e-12 * Q
    return np.min(np.abs(R - Q * zeta)) <= slack


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_medium_teacher_forced_with_recompute(precision):
    k = _k()
    w, sites, q = workloads.workload("medium")
    E, L, p, kT = w["E"], w["L"], w["p"], w["kT"]
    steps = 1000
    st = oracle.LatticeState(E, sites, q)
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision=precision,
                       lattice_edge=E, kT=kT)
    u = workloads.uniforms(steps, w["seed"])
    worst, ties, drifts = 0.0, 0, []
    for s in range(steps):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st.propose()
        assert np.array_equal(mask, mask_o), s
        scale = np.nanmax(np.abs(dU_o))
        e = np.abs(dU - dU_o)[mask_o.astype(bool)] / scale
        err = e.max()
        worst = max(worst, err)
        assert err < TOL12_MEDIUM, (s, err)
        assert np.quantile(e, 0.99) < TOL12_P99, s
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        j, Q_o, dt_o = oracle.select(oracle.rates(dU_o, mask_o, kT), u[s, 0], u[s, 1])
        if ev != j:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], TOL12_MEDIUM * scale), (s, ev, j)
            ties += 1
        k.kmc_fmm_accept_event(h, j)
        st.accept(j // 6, j % 6)
        if (s + 1) % 100 == 0:
            d_phi, d_coef, d_U = k.kmc_fmm_recompute(h)
            drifts.append((d_phi, d_U))
            assert d_phi < 1e-5 and d_U < 1e-6, (s, d_phi, d_U)
    assert ties <= steps // 100 + 1
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    # after the last recompute U is the fresh FMM energy: its p = 12 truncation
    # error is ~1e-6 relative
    U = k.kmc_fmm_energy(h)
    assert abs(U - st.energy()) < 1e-5 * abs(st.energy())
    print(f"{precision}: worst rel dU error {worst:.2e}, near ties {ties}, drift {drifts[-1]}")


def test_large_propose_full_parity():
    """Every hop of the 1M-charge workload in the benchmark's configuration."""
    k = _k()
    w, sites, q = workloads.workload("large")
    E, L, p, kT = w["E"], w["L"], w["p"], w["kT"]
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision="mixed",
                       lattice_edge=E, kT=kT)
    mask, dU = k.kmc_fmm_propose_lattice(h)
    st = oracle.LatticeState(E, sites, q)  # table + FFT site potential
    dU_o, mask_o = st.propose()
    assert np.array_equal(mask, mask_o)
    ok = mask_o.astype(bool)
    scale = np.max(np.abs(dU_o[ok]))
    err = np.abs(dU[ok] - dU_o[ok]) / scale
    print(f"large: max {err.max():.2e} mean {err.mean():.2e} p99 {np.quantile(err, 0.99):.2e}")
    assert err.max() < TOL12
    assert np.quantile(err, 0.99) < TOL12_P99
    assert err.mean() < 2e-6
    # the table-based oracle itself against the direct O(N) sum on a sample
    rng = np.random.default_rng(11)
    ii, kk = np.nonzero(ok)
    pick = rng.choice(len(ii), size=256, replace=False)
    tg = np.array([st.target(int(ii[t]), int(kk[t])) for t in pick])
    d = oracle.lattice_delta_u_direct(E, st.G, st.sites, st.q, ii[pick], tg)
    assert np.max(np.abs(d - dU_o[ii[pick], kk[pick]])) < 1e-10
    U = k.kmc_fmm_energy(h)
    assert abs(U - st.energy()) < 1e-5 * abs(st.energy())


def test_large_run_selects_like_stepwise():
    """The graph-replayed loop on the large workload makes the same choices as
    host-driven steps from the same state (bit-identical kernels)."""
    k = _k()
    w, sites, q = workloads.workload("large")
    E, L, p, kT = w["E"], w["L"], w["p"], w["kT"]
    pos = workloads.site_positions(E, sites)
    u = workloads.uniforms(12, w["seed"] + 3)
    h1 = k.kmc_fmm_init(pos, q, float(E), L, p, precision="mixed", lattice_edge=E, kT=kT)
    ev_run, dt_run = k.kmc_run(h1, u)
    del h1
    h2 = k.kmc_fmm_init(pos, q, float(E), L, p, precision="mixed", lattice_edge=E, kT=kT)
    for s in range(len(u)):
        k.kmc_fmm_propose_lattice(h2)
        ev, dt, Q = k.kmc_step(h2, None, u[s, 0], u[s, 1])
        assert ev == ev_run[s], s
        k.kmc_fmm_accept_event(h2, ev)


def test_blobs_masks_exact_and_sampled_parity():
    """The clustered 512^3 workload (8.4M charges, 70% in Gaussian blobs, full
    leaves of 512 charges): every mask bit-exact against the occupancy, every
    open hop of the most crowded leaf that has open hops and a uniform sample
    of hops against the oracle's direct O(N) lattice sum, at p = 10."""
    k = _k()
    w, sites, q = workloads.workload("blobs")
    E, L, p, kT = w["E"], w["L"], w["p"], w["kT"]
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision="mixed",
                       lattice_edge=E, kT=kT)
    mask, dU = k.kmc_fmm_propose_lattice(h)
    occ = np.zeros(E ** 3, dtype=bool)
    occ[sites] = True
    xyz = workloads.site_xyz(E, sites)
    steps = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    tgt = (xyz[:, None, :] + steps[None, :, :]) % E
    tsite = tgt[..., 0] + E * (tgt[..., 1] + E * tgt[..., 2])
    assert np.array_equal(mask.astype(bool), ~occ[tsite])
    assert np.all(np.isnan(dU[mask == 0]))
    # the densest leaf's charges and a uniform sample
    W = E // 2 ** (L - 1)
    leaf = (xyz[:, 0] // W) + (E // W) * ((xyz[:, 1] // W) + (E // W) * (xyz[:, 2] // W))
    # the most crowded leaf among those whose charges still have open hops
    counts = np.bincount(leaf)
    open_hops = np.bincount(leaf, weights=mask.sum(axis=1))
    dense = np.nonzero(leaf == np.argmax(np.where(open_hops > 0, counts, -1)))[0]
    rng = np.random.default_rng(23)
    ii, kk = np.nonzero(mask)
    pick = rng.choice(len(ii), size=3000, replace=False)
    di, dk = np.nonzero(mask[dense])
    parts = np.concatenate([dense[di], ii[pick]])
    hops = np.concatenate([dk, kk[pick]])
    G = oracle.psi_table(E)
    ref = oracle.lattice_delta_u_direct(E, G, sites, q, parts, tsite[parts, hops])
    got = dU[parts, hops]
    err = np.abs(got - ref) / np.max(np.abs(ref))
    print(f"blobs: {len(parts)} hops ({len(di)} from the densest leaf), max {err.max():.2e} "
          f"mean {err.mean():.2e} p99 {np.quantile(err, 0.99):.2e}")
    assert err.max() < 2e-3
    assert np.quantile(err, 0.99) < 1e-4
