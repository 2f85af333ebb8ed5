"""Replica batches (the ensemble parallelism of Sec. 5.4, on one GPU).

* The batched kernels (every launch covering all members) give the same
  events and positions as running each member alone, in both precisions and
  with the near-field cache, and the same time increments up to rounding (the
  single-system downward pass sums the coarse levels' translations in one
  launch, the batch level by level: the same expansions in another order);
  members of mixed modes fall back to their own kernels as parallel graph
  branches, with identical results.
* Config-4 replicas (64 systems, edges 32..128, occupancy U[0.02, 0.15],
  p = 10, mixed form) through the batched path against the oracle: every
  event equals the oracle's selection from the exact dU with the same
  uniforms except near ties, and after the run every member's masks and dU
  match the oracle's.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _replicas():
    out = []
    for r, (E, occ, L) in enumerate([(16, 0.10, 3), (32, 0.05, 3), (24, 0.12, 3), (32, 0.02, 4)]):
        N = int(round(occ * E ** 3 / 2)) * 2
        sites, q = workloads.uniform_lattice(E, N, 2000 + r)
        out.append((E, N, L, sites, q))
    return out


def _same_as_single_runs(make, steps, seed, twice=False, rtol=1e-6):
    import paper_1905_04065_gb300 as k
    reps = _replicas()
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random((steps, len(reps), 2))
    hs = make()
    b = k.kmc_batch_create(hs)
    info = k.kmc_batch_info(b)
    ev_b, dt_b = k.kmc_batch_run(b, u)
    if twice:
        ev_b2, dt_b2 = k.kmc_batch_run(b, u)  # graph reused, state continues
    pos_b = [k.kmc_fmm_positions(h) for h in hs]
    del b
    for r, h in enumerate(make()):
        ev, dt = k.kmc_run(h, u[:, r, :])
        assert np.array_equal(ev, ev_b[:, r]), r
        np.testing.assert_allclose(dt, dt_b[:, r], rtol=rtol)
        if twice:
            ev2, dt2 = k.kmc_run(h, u[:, r, :])
            assert np.array_equal(ev2, ev_b2[:, r]), r
        assert np.array_equal(k.kmc_fmm_positions(h), pos_b[r])
    return info


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_equals_single_runs(precision):
    import paper_1905_04065_gb300 as k

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision=precision,
                               lattice_edge=E, kT=0.1) for (E, N, L, s, q) in _replicas()]
    info = _same_as_single_runs(make, 17, 77, twice=True)
    assert info["fused"]  # one set of launches for all members
    # level-1 copy, downward levels 2..4, propose, rates, select, record and move, fused accept, reduction
    assert info["launches_per_step"] == 4 + 6


def test_batch_14_hops_with_near_cache_equals_single_runs():
    """Batched kernels with the 14-hop set and the near-field cache (the cached propose and the
    per-move cache update of every member in the batched launches)."""
    import paper_1905_04065_gb300 as k

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision="mixed",
                               lattice_edge=E, kT=0.1, hops=14, near_cache=True) for (E, N, L, s, q) in _replicas()]
    info = _same_as_single_runs(make, 13, 79)
    assert info["fused"]


def test_batch_chunk_setting_keeps_results():
    """The P2P tile (sources staged per pass) changes how the pair sums are staged, not what they
    are: the same events for two pass capacities; a capacity below a member's leaf is refused."""
    import paper_1905_04065_gb300 as k
    reps = _replicas()
    rng = np.random.default_rng(80)
    u = 1.0 - rng.random((9, len(reps), 2))
    out = []
    for chunk in (0, 4000):
        hs = [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision="mixed",
                             lattice_edge=E, kT=0.1) for (E, N, L, s, q) in reps]
        b = k.kmc_batch_create(hs)
        k.kmc_batch_set_chunk(b, chunk)
        assert k.kmc_batch_info(b)["chunk"] == (chunk or k.kmc_batch_info(b)["chunk"])
        out.append(k.kmc_batch_run(b, u)[0])
        with pytest.raises(k.KmcError):
            k.kmc_batch_set_chunk(b, 2)
    assert np.array_equal(out[0], out[1])


def test_batch_rejects_off_lattice_member():
    import paper_1905_04065_gb300 as k
    rng = np.random.default_rng(3)
    pos = rng.random((20, 3)) * 8.0
    q = np.repeat([1.0, -1.0], 10)
    h = k.kmc_fmm_init(pos, q, 8.0, 3, 6)
    with pytest.raises(k.KmcError):
        k.kmc_batch_create([h])


def test_batch_with_mixed_modes_uses_member_kernels():
    """Replicas with the near-field cache (every other one) in the same batch as replicas that sum
    the pairs: the members' own kernels as graph branches, with the same events, times and
    positions as each handle run alone with its own setting."""
    import paper_1905_04065_gb300 as k

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision="mixed",
                               lattice_edge=E, kT=0.1, near_cache=(r % 2 == 0))
                for r, (E, N, L, s, q) in enumerate(_replicas())]
    info = _same_as_single_runs(make, 23, 78, rtol=1e-12)  # the members' own kernels: bit-identical
    assert not info["fused"]


TOL10 = 1e-3  # max |dU - dU_oracle| / max |dU| at p = 10 (mixed form)


def test_config4_replicas_through_the_batch_against_the_oracle():
    """Three replicas of the 64-replica workload (the smallest, a mid-sized one and an E = 128
    one), p = 10, mixed form, leaf level from the valid levels' largest leaf: 2 x 24 batch steps
    (graph-replayed), every event against the oracle's selection on its exact dU with the same
    uniforms (near ties excepted; the oracle then follows the batch's event), then every member's
    masks and dU against the oracle."""
    import paper_1905_04065_gb300 as k
    from paper_1905_04065_gb300 import autotune
    B = workloads.BATCH
    allr = workloads.batch_replicas()
    e128 = [r for r in allr if r["E"] == 128]
    mid = [r for r in allr if r["E"] in (48, 64, 96)]
    pick = [min(allr, key=lambda r: r["N"]), max(mid, key=lambda r: r["N"]), max(e128, key=lambda r: r["N"])]
    assert pick[2]["E"] == 128
    hs, st = [], []
    for r in pick:
        L = autotune.valid_levels(r["E"])[0]
        hs.append(k.kmc_fmm_init(workloads.site_positions(r["E"], r["sites"]), r["q"], float(r["E"]), L, B["p"],
                                 precision="mixed", lattice_edge=r["E"], kT=B["kT"]))
        st.append(oracle.LatticeState(r["E"], r["sites"], r["q"]))
    b = k.kmc_batch_create(hs)
    assert k.kmc_batch_info(b)["fused"]
    rng = np.random.default_rng(B["seed"] + 3)
    ties = 0
    for call in range(2):
        u = 1.0 - rng.random((24, len(pick), 2))
        ev, dt = k.kmc_batch_run(b, u)
        for s in range(24):
            for r in range(len(pick)):
                dU_o, mask_o = st[r].propose()
                ok = mask_o.astype(bool)
                scale = np.max(np.abs(dU_o[ok]))
                rate = oracle.rates(dU_o, mask_o, B["kT"])
                j, Q_o, dt_o = oracle.select(rate, u[s, r, 0], u[s, r, 1])
                e = int(ev[s, r])
                assert mask_o.reshape(-1)[e] == 1, (call, s, r)
                if e != j:
                    R = oracle.cumsum(rate)
                    slack = float(Q_o * TOL10 * scale / B["kT"]) + 1e-12 * Q_o
                    assert np.min(np.abs(R - Q_o * u[s, r, 0])) <= slack, (call, s, r, e, j)
                    ties += 1
                assert abs(dt[s, r] - dt_o) <= dt_o * (np.expm1(TOL10 * scale / B["kT"]) + 1e-6)
                st[r].accept(e // 6, e % 6)  # the oracle follows the batch's event
    assert ties <= 2
    for r, h in enumerate(hs):
        assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(pick[r]["E"], st[r].sites))
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st[r].propose()
        assert np.array_equal(mask, mask_o)
        ok = mask_o.astype(bool)
        err = np.max(np.abs(dU[ok] - dU_o[ok])) / np.max(np.abs(dU_o[ok]))
        print(f"replica E={pick[r]['E']} N={pick[r]['N']}: max dU error {err:.2e} of max|dU|")
        assert err < TOL10


def test_batch_propose_timing_leaves_the_state():
    """The propose-only timing hook: a positive device time, refused before the first run, and the
    run after it gives the same events as the same batch that was not timed."""
    import paper_1905_04065_gb300 as k
    reps = _replicas()
    rng = np.random.default_rng(81)
    u = 1.0 - rng.random((12, len(reps), 2))

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision="mixed",
                               lattice_edge=E, kT=0.1) for (E, N, L, s, q) in reps]
    evs = []
    for timed in (False, True):
        b = k.kmc_batch_create(make())
        if timed:
            with pytest.raises(k.KmcError):
                k.kmc_batch_propose_timed(b, 2)
        e1, _ = k.kmc_batch_run(b, u[:6])
        if timed:
            assert k.kmc_batch_propose_timed(b, 3) > 0.0
        e2, _ = k.kmc_batch_run(b, u[6:])
        evs.append(np.concatenate([e1, e2]))
    assert np.array_equal(evs[0], evs[1])
