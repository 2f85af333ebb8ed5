"""CUDA path (through the C ABI) against the FP64 oracle, on seeded lattice-gas
inputs.

Tolerances.  The method's only approximation is the truncation of the
expansions at degree p (Sec. 2.2, Tab. 2-3 of the paper), so dU matches the
exact tinfoil energy change to a p-dependent bound.  The bounds below are
stated against max |dU| over the compared proposals and were derived from the
geometric convergence of the truncation error with p on these inputs (about a
factor 10 per 3 degrees, as in Tab. 2); FP32 evaluation adds ~1e-6.
Masks, leaf indices and selected events are compared exactly (events except
where Q*zeta lies within the dU tolerance of a cumulative-rate boundary).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = {8: 2e-3, 10: 3e-4, 12: 1e-4, 16: 2e-6}


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _init(E, sites, q, L, p, precision="fp64", kT=0.1, positions=None, hops=6):
    k = _k()
    pos = workloads.site_positions(E, sites) if positions is None else positions
    return k.kmc_fmm_init(pos, q, float(E), L, p, precision=precision, lattice_edge=E, kT=kT, hops=hops)


def _rel_err(a, b, mask):
    ok = mask.astype(bool)
    return float(np.max(np.abs(a[ok] - b[ok])) / np.max(np.abs(b[ok])))


@pytest.fixture(scope="module")
def small():
    w, sites, q = workloads.workload("small")
    st = oracle.LatticeState(w["E"], sites, q)
    return w, sites, q, st


@pytest.mark.parametrize("p", [8, 12, 16])
def test_small_propose_fp64(small, p):
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], p)
    mask, dU = k.kmc_fmm_propose_lattice(h)
    dU_o, mask_o = st.propose()
    assert np.array_equal(mask, mask_o)
    assert np.all(np.isnan(dU[mask == 0]))
    err = _rel_err(dU, dU_o, mask_o)
    assert err < TOL[p], err


def test_small_propose_mixed(small):
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 12, precision="mixed")
    mask, dU = k.kmc_fmm_propose_lattice(h)
    dU_o, mask_o = st.propose()
    assert np.array_equal(mask, mask_o)
    err = _rel_err(dU, dU_o, mask_o)
    assert err < 1e-4, err


def test_energy_matches_oracle(small):
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 12)
    U = k.kmc_fmm_energy(h)
    U_o = st.energy()
    assert abs(U - U_o) < 1e-5 * abs(U_o), (U, U_o)


def test_madelung_energy_fmm():
    """Full FMM energy of an ideal rock-salt block reproduces the Madelung constant."""
    k = _k()
    E = 8
    s = np.arange(E ** 3)
    q = (-1.0) ** workloads.site_xyz(E, s).sum(1)
    h = _init(E, s, q, 3, 12)
    U = k.kmc_fmm_energy(h)
    assert abs(U / E ** 3 + 1.747564594633182 / 2) < 1e-6


def test_fully_occupied_lattice_has_no_event():
    """Degenerate case: every site occupied, so every hop is masked: masks all
    zero, dU all NaN, total rate Q = 0, no event (-1) and an infinite waiting
    time; the host-driven and graph-replayed loops agree."""
    k = _k()
    E = 8
    s = np.arange(E ** 3)
    q = (-1.0) ** workloads.site_xyz(E, s).sum(1)
    for precision in ("fp64", "mixed"):
        h = _init(E, s, q, 3, 8, precision=precision)
        mask, dU = k.kmc_fmm_propose_lattice(h)
        assert not mask.any() and np.all(np.isnan(dU))
        ev, dt, Q = k.kmc_step(h, None, 0.5, 0.5)
        assert ev == -1 and Q == 0.0 and math.isinf(dt)
        evs, dts = k.kmc_run(h, np.full((3, 2), 0.5))
        assert np.all(np.asarray(evs) == -1)


def test_two_charge_system():
    """Smallest neutral system: one +1 and one -1 on a 16^3 lattice; every dU
    against the oracle, a trajectory of accepted hops, and the tracked energy
    against the oracle's after the moves.  All dU are tiny here (~1e-2), so
    the bound is absolute: the p = 12 truncation error of one pair
    interaction across two leaves is ~2e-4 of 1/r ~ 0.08."""
    k = _k()
    E = 16
    sites = np.array([0, 9 + E * (3 + E * 7)])
    q = np.array([1.0, -1.0])
    st = oracle.LatticeState(E, sites, q)
    h = _init(E, sites, q, 3, 12)
    u = workloads.uniforms(20, 77)
    for t in range(20):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st.propose()
        assert np.array_equal(mask, mask_o)
        ok = mask_o.astype(bool)
        assert np.max(np.abs(dU[ok] - dU_o[ok])) < 1e-4
        j, _, _ = oracle.select(oracle.rates(dU_o, mask_o, 0.1), u[t, 0], u[t, 1])
        k.kmc_fmm_accept_event(h, j)
        st.accept(j // 6, j % 6)
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-4


def test_leaf_index_exact(small):
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 8)
    leaf = k.kmc_fmm_leaf_index(h)
    xyz = workloads.site_xyz(w["E"], sites)
    W = w["E"] // 2 ** (w["L"] - 1)
    n = 2 ** (w["L"] - 1)
    c = xyz // W
    ref = c[:, 0] + n * (c[:, 1] + n * c[:, 2])
    assert np.array_equal(leaf, ref.astype(np.int32))


def test_general_propose_matches_oracle(small):
    """Arbitrary targets (one to a few sites away, across the periodic boundary)."""
    k = _k()
    w, sites, q, st = small
    E = w["E"]
    h = _init(E, sites, q, w["L"], 12)
    rng = np.random.default_rng(5)
    occ = set(sites.tolist())
    parts, tsites = [], []
    while len(parts) < 200:
        i = int(rng.integers(0, len(q)))
        d = rng.integers(-3, 4, size=3)
        if not d.any():
            continue
        t = (workloads.site_xyz(E, [sites[i]])[0] + d) % E
        s = int(t[0] + E * (t[1] + E * t[2]))
        if s in occ:
            continue
        parts.append(i)
        tsites.append(s)
    tgt = workloads.site_positions(E, tsites)
    # unwrapped targets too: the library wraps them
    tgt[::3] += E
    dU = k.kmc_fmm_propose(h, np.array(parts, np.int32), tgt)
    ref = st.delta_u_list(parts, tsites)
    err = float(np.max(np.abs(dU - ref)) / np.max(np.abs(ref)))
    assert err < 1e-4, err


def test_proposal_tuples_match_oracle(small):
    """The paper's proposal list ((i, R_i), ...) with 1-4 targets per charge (Sec. 4.2): one
    array of energy changes per tuple, each entry against the oracle."""
    k = _k()
    w, sites, q, st = small
    E = w["E"]
    h = _init(E, sites, q, w["L"], 12)
    rng = np.random.default_rng(17)
    occ = set(sites.tolist())
    P, ref_parts, ref_sites = [], [], []
    for i in rng.choice(len(q), size=60, replace=False):
        ts = set()
        for _ in range(int(rng.integers(1, 5))):
            d = rng.integers(-2, 3, size=3)
            t = (workloads.site_xyz(E, [sites[i]])[0] + d) % E
            s = int(t[0] + E * (t[1] + E * t[2]))
            if d.any() and s not in occ:
                ts.add(s)
        ts = sorted(ts)
        if not ts:
            continue
        P.append((int(i), workloads.site_positions(E, ts)))
        ref_parts += [int(i)] * len(ts)
        ref_sites += ts
    U = k.kmc_fmm_propose_tuples(h, P)
    assert isinstance(U, tuple) and len(U) == len(P)
    assert [len(u) for u in U] == [len(R) for _, R in P]
    ref = st.delta_u_list(ref_parts, ref_sites)
    got = np.concatenate(U)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < 1e-4, err


def test_singular_general_proposal_rejected(small):
    k = _k()
    w, sites, q, st = small
    E = w["E"]
    h = _init(E, sites, q, w["L"], 8)
    tgt = workloads.site_positions(E, [sites[1], sites[2]])  # 0 -> occupied site; 1 -> itself
    with pytest.raises(k.KmcError) as ei:
        k.kmc_fmm_propose(h, np.array([0, 2], np.int32), tgt)
    assert ei.value.code == k.KMC_ERR_ARG


def test_selection_matches_oracle_given_rates(small):
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 8)
    rng = np.random.default_rng(9)
    n = len(q)
    for trial in range(30):
        r = rng.random(6 * n)
        r[rng.random(6 * n) < 0.4] = 0.0
        zeta, xi = 1.0 - rng.random(), 1.0 - rng.random()
        ev, dt, Q = k.kmc_step(h, r, zeta, xi)
        j, Qo, dto = oracle.select(r, zeta, xi)
        R = oracle.cumsum(r)
        near = np.min(np.abs(R - Qo * zeta)) <= 1e-12 * Qo
        assert abs(Q - Qo) <= 1e-12 * Qo
        assert abs(dt - dto) <= 1e-12 * dto
        if not near:
            assert ev == j, (trial, ev, j)


def _near_tie(dU_o, mask_o, kT, zeta, tol_abs):
    """True if Q*zeta is within the rate uncertainty implied by the dU tolerance."""
    r = oracle.rates(dU_o, mask_o, kT)
    R = oracle.cumsum(r)
    Q = R[-1]
    # each rate may move by |dr| <= r * tol/kT; a boundary moves by at most the sum
    slack = float(np.sum(r) * tol_abs / kT) + 1e-12 * Q
    return np.min(np.abs(R - Q * zeta)) <= slack


def test_teacher_forced_trajectory_small(small):
    """Propose, select and accept for 40 steps with the oracle's event forced
    into both paths (Sec. 3 propose/accept); dU, masks and events compared each
    step, then a recompute measures the accept-update drift."""
    k = _k()
    w, sites, q, _ = small
    E, kT = w["E"], w["kT"]
    p = 12
    st = oracle.LatticeState(E, sites, q)
    h = _init(E, sites, q, w["L"], p, kT=kT)
    u = workloads.uniforms(40, w["seed"])
    agree = 0
    for s in range(40):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st.propose()
        assert np.array_equal(mask, mask_o)
        tol = TOL[p] * np.nanmax(np.abs(dU_o))
        assert np.nanmax(np.abs(dU - dU_o)) < tol
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        r_o = oracle.rates(dU_o, mask_o, kT)
        j, Q_o, dt_o = oracle.select(r_o, u[s, 0], u[s, 1])
        if ev == j:
            agree += 1
        else:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], tol), (s, ev, j)
        du_acc = k.kmc_fmm_accept_event(h, j)
        assert abs(du_acc - dU_o.reshape(-1)[j]) < tol
        st.accept(j // 6, j % 6)
    assert agree >= 38
    pos = k.kmc_fmm_positions(h)
    assert np.array_equal(pos, workloads.site_positions(E, st.sites))
    U = k.kmc_fmm_energy(h)
    assert abs(U - st.energy()) < 1e-4 * abs(st.energy())
    d_phi, d_coef, d_U = k.kmc_fmm_recompute(h)
    # incremental P2L updates vs fresh M2L differ by truncation only
    assert d_phi < 1e-5, d_phi
    assert d_U < 1e-5, d_U
    U2 = k.kmc_fmm_energy(h)
    assert abs(U2 - st.energy()) < 1e-4 * abs(st.energy())


def _oracle_hops(st, nh):
    """Masks and dU of every hop of the hop set (event order j = nh i + k) from
    the oracle's site potential; the targets come from the workload's hop list."""
    tg = oracle.hop_targets(st.E, st.sites, nh).reshape(-1)
    mask = (st.occ[tg] == 0).astype(np.uint8)
    ok = mask.astype(bool)
    dU = np.full(len(tg), np.nan)
    dU[ok] = st.delta_u_list(np.repeat(np.arange(st.n), nh)[ok], tg[ok])
    return dU, mask, tg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_teacher_forced_trajectory_14_hops(small, precision):
    """The hop set of the paper's Sec. 5.3 benchmark (6 faces and 8 body
    diagonals): masks exactly and dU within the p = 12 tolerance against the
    oracle at every step of a trajectory on which the oracle's event is
    accepted on both sides (diagonal hops included), events compared except
    near ties, and the energy after the trajectory."""
    k = _k()
    w, sites, q, _ = small
    E, kT, p, nh = w["E"], w["kT"], 12, 14
    st = oracle.LatticeState(E, sites, q)
    h = _init(E, sites, q, w["L"], p, precision=precision, kT=kT, hops=nh)
    u = workloads.uniforms(30, w["seed"] + 14)
    agree, diag = 0, 0
    for s in range(30):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        assert mask.shape == (len(q), nh)
        dU_o, mask_o, tg = _oracle_hops(st, nh)
        assert np.array_equal(mask.reshape(-1), mask_o)
        assert np.all(np.isnan(dU.reshape(-1)[mask_o == 0]))
        ok = mask_o.astype(bool)
        tol = TOL[p] * np.max(np.abs(dU_o[ok]))
        assert np.max(np.abs(dU.reshape(-1)[ok] - dU_o[ok])) < tol
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        r_o = oracle.rates(dU_o, mask_o, kT)
        j, Q_o, dt_o = oracle.select(r_o, u[s, 0], u[s, 1])
        if ev == j:
            agree += 1
        else:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], tol), (s, ev, j)
        du_acc = k.kmc_fmm_accept_event(h, j)
        assert abs(du_acc - dU_o[j]) < tol
        diag += int(j % nh >= 6)
        st.accept_site(j // nh, tg[j])
    assert agree >= 28
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-4 * abs(st.energy())
    print(f"14 hops ({precision}): {agree}/30 events agree, {diag} diagonal hops accepted")


def test_run_matches_stepwise(small):
    """The graph-replayed device loop makes the same choices as the host-driven
    propose/step/accept sequence (same precision, same inputs)."""
    k = _k()
    w, sites, q, _ = small
    E, kT = w["E"], w["kT"]
    steps = 21
    u = workloads.uniforms(steps, w["seed"] + 1)
    h1 = _init(E, sites, q, w["L"], 8, kT=kT)
    ev_run, dt_run = k.kmc_run(h1, u)
    h2 = _init(E, sites, q, w["L"], 8, kT=kT)
    for s in range(steps):
        k.kmc_fmm_propose_lattice(h2)
        ev, dt, Q = k.kmc_step(h2, None, u[s, 0], u[s, 1])
        assert ev == ev_run[s], s
        assert abs(dt - dt_run[s]) <= 1e-12 * dt
        k.kmc_fmm_accept_event(h2, ev)
    assert np.array_equal(k.kmc_fmm_positions(h1), k.kmc_fmm_positions(h2))


def test_run_against_oracle_trajectory(small):
    """Untethered device loop vs the oracle's own trajectory: identical events
    for as long as no near tie occurs."""
    k = _k()
    w, sites, q, _ = small
    E, kT = w["E"], w["kT"]
    steps = 30
    u = workloads.uniforms(steps, w["seed"] + 2)
    h = _init(E, sites, q, w["L"], 12, kT=kT)
    ev_run, dt_run = k.kmc_run(h, u)
    st = oracle.LatticeState(E, sites, q)
    for s in range(steps):
        dU_o, mask_o = st.propose()
        r = oracle.rates(dU_o, mask_o, kT)
        j, Q, dt = oracle.select(r, u[s, 0], u[s, 1])
        if ev_run[s] != j:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], TOL[12] * np.nanmax(np.abs(dU_o))), s
            return
        assert abs(dt_run[s] - dt) < 1e-3 * dt
        st.accept(j // 6, j % 6)


@pytest.mark.parametrize("bad", ["levels", "order", "neutral", "outside", "offsite", "edge", "duplicate"])
def test_init_errors(bad):
    k = _k()
    E, L, p = 16, 3, 8
    sites, q = workloads.random_small(E, 40, 3)
    pos = workloads.site_positions(E, sites)
    kw = dict(lattice_edge=E)
    if bad == "levels":
        L = 2
    elif bad == "order":
        p = 0
    elif bad == "neutral":
        q = q.copy()
        q[0] = 3.0
    elif bad == "outside":
        pos = pos.copy()
        pos[3, 1] = E + 0.5
    elif bad == "offsite":
        pos = pos.copy()
        pos[3, 1] += 0.25
    elif bad == "edge":
        kw = dict(lattice_edge=E)
        L = 6  # 16 is not a multiple of 32
    elif bad == "duplicate":
        pos = pos.copy()
        pos[4] = pos[5]
    with pytest.raises(k.KmcError) as ei:
        k.kmc_fmm_init(pos, q, float(E), L, p, **kw)
    expect = k.KMC_ERR_NOT_NEUTRAL if bad == "neutral" else k.KMC_ERR_ARG
    assert ei.value.code == expect


def test_device_memory_interface(small):
    """Same results with torch CUDA tensors in and out (device pointers)."""
    import torch
    k = _k()
    w, sites, q, st = small
    E = w["E"]
    pos = torch.tensor(workloads.site_positions(E, sites), device="cuda")
    qt = torch.tensor(q, device="cuda")
    h = k.kmc_fmm_init(pos, qt, float(E), w["L"], 8, lattice_edge=E, kT=w["kT"])
    mask, dU = k.kmc_fmm_propose_lattice(h)
    assert mask.is_cuda and dU.is_cuda
    h2 = _init(E, sites, q, w["L"], 8, kT=w["kT"])
    mask2, dU2 = k.kmc_fmm_propose_lattice(h2)
    assert np.array_equal(mask.cpu().numpy(), mask2)
    np.testing.assert_array_equal(dU.cpu().numpy(), dU2)


def test_mixed_form_fp32_output(small):
    """The mixed form's FP32 dU: the same values as its widened FP64 output (NaN where masked), the
    same mask, into a caller-owned pinned float32 buffer too; refused for an FP64-form handle."""
    import torch
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 12, precision="mixed")
    m64, d64 = k.kmc_fmm_propose_lattice(h)
    m32, d32 = k.kmc_fmm_propose_lattice(h, dtype=np.float32)
    assert d32.dtype == np.float32 and np.array_equal(m32, m64)
    np.testing.assert_array_equal(d32.astype(np.float64), d64)
    buf = torch.empty((len(q), 6), dtype=torch.float32, pin_memory=True)
    _, d32b = k.kmc_fmm_propose_lattice(h, None, buf)
    assert d32b is buf
    np.testing.assert_array_equal(buf.numpy(), d32)
    h64 = _init(w["E"], sites, q, w["L"], 8)
    with pytest.raises(k.KmcError):
        k.kmc_fmm_propose_lattice(h64, dtype=np.float32)


def test_asynchronous_outputs_follow_the_synchronous_path(small):
    """kmc_fmm_propose_lattice(..., wait=False): the copies overlap kmc_step and the accept; after
    kmc_fmm_outputs_wait (or the next proposal) the buffers hold what the synchronous FP32 call gives
    on a second handle driven by the same uniforms, step by step; FP64 output refused."""
    import torch
    k = _k()
    w, sites, q, st = small
    ha = _init(w["E"], sites, q, w["L"], 12, precision="mixed", kT=w["kT"])
    hs = _init(w["E"], sites, q, w["L"], 12, precision="mixed", kT=w["kT"])
    u = workloads.uniforms(6, 17)
    bufs = [(torch.empty((len(q), 6), dtype=torch.uint8, pin_memory=True),
             torch.empty((len(q), 6), dtype=torch.float32, pin_memory=True)) for _ in range(2)]
    ref = []
    for s in range(6):
        k.kmc_fmm_propose_lattice(ha, *bufs[s & 1], wait=False)
        ev_a, dt_a, _ = k.kmc_step(ha, None, u[s, 0], u[s, 1])
        k.kmc_fmm_accept_event(ha, ev_a)
        m_s, d_s = k.kmc_fmm_propose_lattice(hs, dtype=np.float32)
        ev_s, dt_s, _ = k.kmc_step(hs, None, u[s, 0], u[s, 1])
        k.kmc_fmm_accept_event(hs, ev_s)
        assert ev_a == ev_s and dt_a == dt_s
        ref.append((m_s, d_s))
        if s >= 1:  # the previous step's buffers are complete once this step's proposal returned
            mp, dp = bufs[(s - 1) & 1]
            assert np.array_equal(mp.numpy(), ref[s - 1][0])
            np.testing.assert_array_equal(dp.numpy(), ref[s - 1][1])
    k.kmc_fmm_outputs_wait(ha)
    assert np.array_equal(bufs[1][0].numpy(), ref[5][0])
    np.testing.assert_array_equal(bufs[1][1].numpy(), ref[5][1])
    with pytest.raises(ValueError):
        k.kmc_fmm_propose_lattice(ha, wait=False)


def test_caller_owned_pinned_outputs(small):
    """Outputs written in place into caller-owned pinned host buffers equal the
    library-allocated ones; mismatched buffers are refused."""
    import torch
    k = _k()
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 8, kT=w["kT"])
    mask_h = torch.empty((len(q), 6), dtype=torch.uint8, pin_memory=True)
    dU_h = torch.empty((len(q), 6), dtype=torch.float64, pin_memory=True)
    m1, d1 = k.kmc_fmm_propose_lattice(h, mask_h, dU_h)
    assert m1 is mask_h and d1 is dU_h
    m2, d2 = k.kmc_fmm_propose_lattice(h)
    assert np.array_equal(mask_h.numpy(), m2)
    np.testing.assert_array_equal(dU_h.numpy(), d2)
    with pytest.raises(ValueError):
        k.kmc_fmm_propose_lattice(h, mask_h, torch.empty((len(q), 5), dtype=torch.float64))


def test_offlattice_propose_and_accept():
    """Off-lattice positions (the paper's general interface): dU against the
    direct Ewald oracle, then an accepted move and U(after) - U(before)."""
    k = _k()
    rng = np.random.default_rng(17)
    a = 12.0
    n = 120
    pos = rng.random((n, 3)) * a
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    h = k.kmc_fmm_init(pos, q, a, 3, 14)
    parts = rng.integers(0, n, size=40).astype(np.int32)
    tgt = (pos[parts] + rng.normal(0, 0.7, size=(40, 3))) % a
    dU = k.kmc_fmm_propose(h, parts, tgt)
    ref = oracle.delta_u(pos, q, a, parts, tgt)
    err = float(np.max(np.abs(dU - ref)) / np.max(np.abs(ref)))
    assert err < 1e-4, err
    U0 = k.kmc_fmm_energy(h)
    assert abs(U0 - oracle.energy(pos, q, a)) < 1e-4 * abs(U0)
    du = k.kmc_fmm_accept(h, int(parts[0]), tgt[0])
    assert abs(du - ref[0]) < 1e-4 * np.max(np.abs(ref))
    U1 = k.kmc_fmm_energy(h)
    assert abs((U1 - U0) - du) < 1e-12 * abs(U0) + 1e-12


def test_bounded_device_wait_gives_up_and_context_survives(small):
    """The bounded mbarrier wait of the propose kernel, run against a phase
    that never completes, returns KMC_ERR_TIMEOUT after its limit; the CUDA
    context stays usable (a propose afterwards matches the oracle)."""
    import time
    k = _k()
    t0 = time.perf_counter()
    assert k.kmc_check_bounded_wait(0, 0.05) == k.KMC_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.05
    w, sites, q, st = small
    h = _init(w["E"], sites, q, w["L"], 8, precision="mixed")
    mask, dU = k.kmc_fmm_propose_lattice(h)
    dU_o, mask_o = st.propose()
    assert np.array_equal(mask, mask_o)
    assert _rel_err(dU, dU_o, mask_o) < TOL[8]


@pytest.mark.parametrize("near_cache", [False, True])
def test_checkpoint_resume_continues_the_trajectory(small, tmp_path, near_cache):
    """40 device-driven steps in one go against 20 steps, a checkpoint, a new handle from it and
    the next 20 uniforms: the same events and positions (the resumed far field differs from the
    incrementally updated one by truncation only, far below the gaps the uniforms fall into),
    energies within 1e-5."""
    k = _k()
    w, sites, q, _ = small
    E, kT = w["E"], w["kT"]
    u = workloads.uniforms(40, w["seed"] + 40)

    def make():
        return k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), w["L"], 12, precision="fp64",
                              lattice_edge=E, kT=kT, near_cache=near_cache)
    h1 = make()
    ev_all, _ = k.kmc_run(h1, u)
    h2 = make()
    ev_a, _ = k.kmc_run(h2, u[:20])
    path = str(tmp_path / "ckpt.npz")
    k.kmc_checkpoint(h2, path, step=20)
    del h2
    h3, step, _ = k.kmc_resume(path)
    assert step == 20
    ev_b, _ = k.kmc_run(h3, u[step:])
    assert np.array_equal(np.concatenate([ev_a, ev_b]), ev_all)
    assert np.array_equal(k.kmc_fmm_positions(h3), k.kmc_fmm_positions(h1))
    assert abs(k.kmc_fmm_energy(h3) - k.kmc_fmm_energy(h1)) < 1e-5 * abs(k.kmc_fmm_energy(h1))

