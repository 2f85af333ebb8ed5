"""Grounded walls at z = 0 and z = a/2 with an applied field (the Dirichlet case
of Sec. 2.2, by mirror charges and the periodic method on the mirrored cell):
the CUDA path through the C ABI against the oracle (Ewald sums on the mirrored
cell, ``oracle.DirichletLattice``, itself pinned by the vanishing wall potential
and brute-force energies).

Tolerances: the periodic ones at p = 12 (1e-4 of max |dU|; the mirror terms
add tabulated C(d) values of the same accuracy).  Masks are exact: a hop is
masked when its target is occupied or lies beyond a wall.  Events are compared
except near ties.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL12 = 1e-4


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _system(E, n, seed):
    rng = np.random.default_rng(seed)
    lower = np.nonzero(np.arange(E ** 3) // (E * E) < E // 2)[0]
    sites = rng.choice(lower, n, replace=False)
    q = np.where(rng.permutation(n) % 2 == 0, 1.0, -1.0)
    return sites, q


def _near_tie(dU, mask, kT, zeta, tol_abs):
    r = oracle.rates(dU, mask, kT)
    R = oracle.cumsum(r)
    Q = R[-1]
    return np.min(np.abs(R - Q * zeta)) <= float(np.sum(r) * tol_abs / kT) + 1e-12 * Q


@pytest.mark.parametrize("precision,nh", [("fp64", 6), ("mixed", 14)])
def test_dirichlet_trajectory(precision, nh):
    """Energy at start and end, masks, every dU, events and accepted dU along a
    15-step host-driven trajectory (the oracle's event accepted on both sides),
    then 10 device-driven steps (graph replay) against the oracle's choices."""
    k = _k()
    E, L, p, kT, fz = 16, 3, 12, 0.1, 0.2
    sites, q = _system(E, 500, 41 + nh)
    st = oracle.DirichletLattice(E, sites, q, oracle.hop_vectors(nh), field_z=fz)
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision=precision,
                       lattice_edge=E, kT=kT, hops=nh, bc="dirichlet", field_z=fz)
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-5 * abs(st.energy())
    u = workloads.uniforms(25, 4242 + nh)
    agree, worst, wall = 0, 0.0, 0
    for s in range(15):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st.propose()
        assert np.array_equal(mask, mask_o)
        ok = mask_o.astype(bool)
        zn = (st.sites // (E * E))[:, None] + oracle.hop_vectors(nh)[None, :, 2]
        through = (zn < 0) | (zn >= E // 2)  # hops through a wall (a face hop lands on its own mirror)
        assert not np.any(mask[through])
        wall += int(np.sum(through))
        tol = TOL12 * np.max(np.abs(dU_o[ok]))
        err = np.max(np.abs(dU[ok] - dU_o[ok]))
        assert err < tol, (s, err)
        worst = max(worst, err / np.max(np.abs(dU_o[ok])))
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        j, Q_o, dt_o = oracle.select(oracle.rates(dU_o, mask_o, kT), u[s, 0], u[s, 1])
        if ev == j:
            agree += 1
        else:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], tol), (s, ev, j)
        du_acc = k.kmc_fmm_accept_event(h, j)
        assert abs(du_acc - dU_o.reshape(-1)[j]) < tol
        st.accept(j // nh, oracle.hop_targets(E, st.sites[j // nh:j // nh + 1], nh)[0, j % nh])
    assert agree >= 13 and wall > 0
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-5 * abs(st.energy())
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    # device-driven steps: the mirrors move inside the graph
    events, dts = k.kmc_run(h, u[15:25])
    run_agree = 0
    for s in range(10):
        dU_o, mask_o = st.propose()
        j, _, _ = oracle.select(oracle.rates(dU_o, mask_o, kT), u[15 + s, 0], u[15 + s, 1])
        if events[s] != j:
            ok = mask_o.astype(bool)
            assert _near_tie(dU_o, mask_o, kT, u[15 + s, 0], TOL12 * np.max(np.abs(dU_o[ok]))), (s, events[s], j)
            j = int(events[s])
        else:
            run_agree += 1
        st.accept(j // nh, oracle.hop_targets(E, st.sites[j // nh:j // nh + 1], nh)[0, j % nh])
    assert run_agree >= 8
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    assert abs(k.kmc_fmm_energy(h) - st.energy()) < 1e-5 * abs(st.energy())
    print(f"dirichlet ({precision}, {nh} hops): worst rel dU error {worst:.2e}, {agree}/15 and "
          f"{run_agree}/10 events agree, {wall} wall-masked hops")


def test_dirichlet_rejects_charges_above_the_plane_and_general_moves():
    k = _k()
    E = 8
    sites = np.array([0, 1, E * E * (E // 2)])  # the third charge sits on the mirror plane
    with pytest.raises(k.KmcError):
        k.kmc_fmm_init(workloads.site_positions(E, sites), np.array([1.0, -1.0, 1.0]), float(E), 3, 4,
                       lattice_edge=E, bc="dirichlet")
    h = k.kmc_fmm_init(workloads.site_positions(E, sites[:2]), np.array([1.0, -1.0]), float(E), 3, 4,
                       lattice_edge=E, bc="dirichlet")
    with pytest.raises(k.KmcError):
        k.kmc_fmm_propose(h, np.array([0], dtype=np.int32), np.array([[0.5, 0.5, 1.5]]))
