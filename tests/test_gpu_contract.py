"""The dU accuracy targets on every hop, at the orders that meet them.

Targets: the FP64 form within 1e-6 max|dU| of the exact tinfoil energy
change, the mixed form (FP32 near field, L2P and dU assembly) within
1e-4 max|dU|.  The method's one approximation is the truncation of the
expansions at degree p (Sec. 2.2, Eq. (multipole_local_expansion); Sec. 5.1,
Tabs. 2-3): the error falls geometrically with p and is largest for hops that
cross the boundary of a coarse cell (level 2 or 3), where the truncation
errors of the M2L translations between distance-two cells of those levels do
not cancel between the old and the new position.  At p = 12 that worst case
is 1.5e-4 max|dU| on the 256^3 workload (8e-5 on the 64^3 one); the FP64
target needs p = 20 on the 64^3 workload and p = 22 on the 256^3 one, the
mixed target p = 12 on the 64^3 and p = 14 on the 256^3 workload.

Every test compares each unmasked hop with the oracle (masks exactly), and the
trajectories accept the oracle's event on both sides (teacher forcing), so
that each step starts from the same configuration; events must agree except
where Q zeta lies within the dU tolerance of a cumulative-rate boundary."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FP64_TARGET = 1e-6
MIXED_TARGET = 1e-4


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _near_tie(dU_o, mask_o, kT, zeta, tol_abs):
    r = oracle.rates(dU_o, mask_o, kT)
    R = oracle.cumsum(r)
    Q = R[-1]
    slack = float(np.sum(r) * tol_abs / kT) + 1e-12 * Q
    return np.min(np.abs(R - Q * zeta)) <= slack


def _trajectory(name, precision, p, steps, target, recompute_every=0):
    k = _k()
    w, sites, q = workloads.workload(name)
    E, L, kT = w["E"], w["L"], w["kT"]
    st = oracle.LatticeState(E, sites, q)
    h = k.kmc_fmm_init(workloads.site_positions(E, sites), q, float(E), L, p, precision=precision,
                       lattice_edge=E, kT=kT)
    u = workloads.uniforms(steps, w["seed"] + 77)
    worst, ties = 0.0, 0
    for s in range(steps):
        mask, dU = k.kmc_fmm_propose_lattice(h)
        dU_o, mask_o = st.propose()
        assert np.array_equal(mask, mask_o), s
        ok = mask_o.astype(bool)
        scale = np.max(np.abs(dU_o[ok]))
        err = float(np.max(np.abs(dU[ok] - dU_o[ok]))) / scale
        worst = max(worst, err)
        assert err <= target, (s, err)
        ev, dt, Q = k.kmc_step(h, None, u[s, 0], u[s, 1])
        j, Q_o, dt_o = oracle.select(oracle.rates(dU_o, mask_o, kT), u[s, 0], u[s, 1])
        # every rate moves by at most a factor exp(|d dU| / kT) (FP32 rate mantissas: 1e-6 more)
        assert abs(Q - Q_o) <= Q_o * (np.expm1(target * scale / kT) + 1e-6)
        if ev != j:
            assert _near_tie(dU_o, mask_o, kT, u[s, 0], target * scale), (s, ev, j)
            ties += 1
        du = k.kmc_fmm_accept_event(h, j)
        assert abs(du - dU_o.reshape(-1)[j]) <= target * scale
        st.accept(j // 6, j % 6)
        if recompute_every and (s + 1) % recompute_every == 0:
            d_phi, d_coef, d_U = k.kmc_fmm_recompute(h)
            assert d_phi < 10 * target and d_U < 10 * target, (s, d_phi, d_U)
    assert ties <= steps // 50 + 1
    assert np.array_equal(k.kmc_fmm_positions(h), workloads.site_positions(E, st.sites))
    U = k.kmc_fmm_energy(h)
    assert abs(U - st.energy()) <= 10 * target * abs(st.energy())
    print(f"{name} {precision} p={p}: worst {worst:.2e} of max|dU| over {steps} steps, near ties {ties}")
    return worst


def test_medium_fp64_meets_1e6_at_p20():
    """64^3 sites, 32768 charges, L = 4, FP64 at p = 20: every hop of a 100-step trajectory
    within 1e-6 max|dU| (measured 6.1e-7 at the first step), recompute every 50 steps."""
    _trajectory("medium", "fp64", 20, 100, FP64_TARGET, recompute_every=50)


def test_medium_mixed_meets_1e4_at_p12():
    """64^3 sites, 32768 charges, L = 4, mixed form at p = 12: every hop of a 200-step
    trajectory within 1e-4 max|dU| (measured 8.1e-5)."""
    _trajectory("medium", "mixed", 12, 200, MIXED_TARGET)


def test_large_mixed_meets_1e4_at_p14():
    """256^3 sites, 1,048,576 charges, L = 6 (the benchmark's workload), mixed form at p = 14:
    every hop of a 10-step trajectory within 1e-4 max|dU| (measured 6.3e-5)."""
    _trajectory("large", "mixed", 14, 10, MIXED_TARGET)


def test_large_fp64_meets_1e6_at_p22():
    """256^3 sites, 1,048,576 charges, L = 6, FP64 at p = 22 (FP64 CUDA-core M2L): every hop of
    one propose within 1e-6 max|dU| (measured 8.7e-7; 1.4e-5 at p = 16, 2.1e-6 at p = 20)."""
    _trajectory("large", "fp64", 22, 1, FP64_TARGET)


def test_small_fp64_p8_100_steps():
    """The 16^3 workload as its configuration states it: 1000 charges, L = 3, FP64, p = 8,
    kT = 0.1, 100 KMC steps.  No target is stated at p = 8; the bound asserted is the measured
    truncation error at that order (4.4e-4 max|dU| at the first step) with headroom."""
    _trajectory("small", "fp64", 8, 100, 1e-3)
