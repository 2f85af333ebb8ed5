"""Free-space boundary conditions (Sec. 2.2 and Sec. 3, Eq. (proposed_energy)
as written): the CUDA path through the C ABI against the oracle's direct FP64
free-space sums.

The only approximation is the expansion truncation at degree p; the tolerances
are the periodic ones at p = 12 (stated against max |dU| over the compared
hops), which the free-space form meets with room since it has no image
sums.  Masks are exact: a hop is masked when its target is occupied or lies
outside the box (a free-space lattice has no sites beyond its faces).
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


def _oracle_lattice(E, sites, q, nh):
    """Masks and dU of every lattice hop in free space (event order j = nh i + k)."""
    xyz = workloads.site_xyz(E, sites)
    raw = xyz[:, None, :] + oracle.hop_vectors(nh)[None, :, :]
    inside = np.all((raw >= 0) & (raw < E), axis=2).reshape(-1)
    tg = oracle.hop_targets(E, sites, nh).reshape(-1)
    occ = np.zeros(E ** 3, dtype=bool)
    occ[sites] = True
    mask = (inside & ~occ[tg]).astype(np.uint8)
    ok = mask.astype(bool)
    pos = workloads.site_positions(E, sites)
    part = np.repeat(np.arange(len(q)), nh)
    dU = np.full(len(tg), np.nan)
    dU[ok] = oracle.free_delta_u(pos, q, part[ok], workloads.site_positions(E, tg[ok]))
    return dU, mask, tg


@pytest.mark.parametrize("precision,nh", [("fp64", 6), ("mixed", 6), ("mixed", 14)])
def test_free_space_lattice_trajectory(precision, nh):
    """Masks, every dU, the selected event and the accepted dU against the
    oracle at each step of a 20-step trajectory (the oracle's event accepted
    on both sides), then the energy; with the 14-hop set, diagonal hops that
    leave the box through an edge or a corner are masked too."""
    k = _k()
    w, sites, q = workloads.workload("small")
    E, kT = w["E"], w["kT"]
    sites = sites.copy()
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), w["L"], 12, precision=precision,
                       lattice_edge=E, kT=kT, bc="free", hops=nh)
    U0 = oracle.free_energy(workloads.site_positions(E, sites), q)
    assert abs(k.kmc_fmm_energy(h) - U0) < 1e-5 * abs(U0)
    u = workloads.uniforms(20, w["seed"] + 21)
    agree, worst = 0, 0.0
    for s in range(20):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o, tg = _oracle_lattice(E, sites, q, nh)
        assert np.array_equal(mask.reshape(-1), mask_o)
        ok = mask_o.astype(bool)
        tol = TOL12 * np.max(np.abs(dU_o[ok]))
        err = np.max(np.abs(dU.reshape(-1)[ok] - dU_o[ok]))
        assert err < tol, (s, err / np.max(np.abs(dU_o[ok])))
        worst = max(worst, err / np.max(np.abs(dU_o[ok])))
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        j, Q_o, dt_o = oracle.select(oracle.rates(dU_o, mask_o, kT), u[s, 0], u[s, 1])
        agree += int(ev == j)
        du_acc = k.kmc_fmm_accept_event(h, j)
        assert abs(du_acc - dU_o[j]) < tol
        sites[j // nh] = tg[j]
    assert agree >= 18
    U1 = oracle.free_energy(workloads.site_positions(E, sites), q)
    assert abs(k.kmc_fmm_energy(h) - U1) < 1e-5 * abs(U1)
    print(f"free space ({precision}, {nh} hops): worst rel dU error {worst:.2e}, {agree}/20 events agree, "
          f"energy rel error {abs(k.kmc_fmm_energy(h) - U1) / abs(U1):.1e}")


def test_free_space_general_proposals_and_net_charge():
    """Off-lattice charges with a net charge (allowed in free space), general
    proposals inside the box against the oracle; a target outside the box is
    rejected."""
    k = _k()
    rng = np.random.default_rng(77)
    n, a = 600, 12.0
    pos = rng.random((n, 3)) * a
    q = rng.choice([-1.0, 1.0, 1.0], size=n)  # net positive
    h = k.kmc_fmm_init(pos, q, a, 3, 12, precision="fp64", bc="free")
    U = oracle.free_energy(pos, q)
    assert abs(k.kmc_fmm_energy(h) - U) < 1e-5 * abs(U)
    m = 400
    part = rng.integers(0, n, size=m).astype(np.int32)
    tgt = np.clip(pos[part] + rng.normal(scale=0.7, size=(m, 3)), 0.0, a - 1e-9)
    dU = k.kmc_fmm_propose(h, part, tgt)
    dU_o = oracle.free_delta_u(pos, q, part, tgt)
    err = np.max(np.abs(dU - dU_o)) / np.max(np.abs(dU_o))
    assert err < TOL12
    print(f"free space, off-lattice, net charge {q.sum():+.0f}: worst rel dU error {err:.2e}")
    with pytest.raises(k.KmcError):
        k.kmc_fmm_propose(h, part[:1], np.array([[a + 0.5, 1.0, 1.0]]))


def test_periodic_still_requires_neutrality():
    k = _k()
    pos = np.array([[0.5, 0.5, 0.5], [1.5, 1.5, 1.5]])
    with pytest.raises(k.KmcError):
        k.kmc_fmm_init(pos, np.array([1.0, 1.0]), 4.0, 3, 4)
    h = k.kmc_fmm_init(pos, np.array([1.0, 1.0]), 4.0, 3, 4, bc="free")
    assert abs(k.kmc_fmm_energy(h) - 1.0 / np.sqrt(3.0)) < 1e-10
