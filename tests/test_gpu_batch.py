"""Replica batches: several independent lattice systems of different sizes
advanced from one graph give the same events as running each alone (the
ensemble parallelism of Sec. 5.4, on one GPU)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _replicas():
    out = []
    for r, (E, occ, L) in enumerate([(16, 0.10, 3), (32, 0.05, 3), (24, 0.12, 3), (32, 0.02, 4)]):
        N = int(round(occ * E ** 3 / 2)) * 2
        sites, q = workloads.uniform_lattice(E, N, 2000 + r)
        out.append((E, N, L, sites, q))
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_equals_single_runs(precision):
    import paper_1905_04065_gb300 as k
    reps = _replicas()
    steps = 17
    rng = np.random.default_rng(77)
    u = 1.0 - rng.random((steps, len(reps), 2))

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision=precision,
                               lattice_edge=E, kT=0.1) for (E, N, L, s, q) in reps]

    hs = make()
    b = k.kmc_batch_create(hs)
    ev_b, dt_b = k.kmc_batch_run(b, u)
    ev_b2, dt_b2 = k.kmc_batch_run(b, u)  # graph reused, state continues
    pos_b = [k.kmc_fmm_positions(h) for h in hs]
    del b
    hs2 = make()
    for r, h in enumerate(hs2):
        ev, dt = k.kmc_run(h, u[:, r, :])
        assert np.array_equal(ev, ev_b[:, r]), r
        np.testing.assert_allclose(dt, dt_b[:, r], rtol=1e-12)
        ev2, dt2 = k.kmc_run(h, u[:, r, :])
        assert np.array_equal(ev2, ev_b2[:, r]), r
        assert np.array_equal(k.kmc_fmm_positions(h), pos_b[r])


def test_batch_rejects_off_lattice_member():
    import paper_1905_04065_gb300 as k
    rng = np.random.default_rng(3)
    pos = rng.random((20, 3)) * 8.0
    q = np.repeat([1.0, -1.0], 10)
    h = k.kmc_fmm_init(pos, q, 8.0, 3, 6)
    with pytest.raises(k.KmcError):
        k.kmc_batch_create([h])


def test_batch_with_near_cache_members():
    """Replicas with the near-field cache (every other one) in the same graph as replicas that sum
    the pairs: the same events, times and positions as each handle run alone with its own setting
    (the cache's per-move update is part of every replica's captured step)."""
    import paper_1905_04065_gb300 as k
    reps = _replicas()
    steps = 23
    rng = np.random.default_rng(78)
    u = 1.0 - rng.random((steps, len(reps), 2))

    def make():
        return [k.kmc_fmm_init(workloads.site_positions(E, s), q, float(E), L, 8, precision="mixed",
                               lattice_edge=E, kT=0.1, near_cache=(r % 2 == 0))
                for r, (E, N, L, s, q) in enumerate(reps)]

    hs = make()
    b = k.kmc_batch_create(hs)
    ev_b, dt_b = k.kmc_batch_run(b, u)
    pos_b = [k.kmc_fmm_positions(h) for h in hs]
    del b
    for r, h in enumerate(make()):
        ev, dt = k.kmc_run(h, u[:, r, :])
        assert np.array_equal(ev, ev_b[:, r]), r
        np.testing.assert_allclose(dt, dt_b[:, r], rtol=1e-12)
        assert np.array_equal(k.kmc_fmm_positions(h), pos_b[r])
