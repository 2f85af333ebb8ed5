"""The two arithmetics of the one-off M2L (Algorithm 2) against each other.

The default M2L runs on the bf16 tensor cores: the FP64 operands are cut into
exact integer slices and the slice products are summed exactly, so the result
is the FP64 product up to the dropped low-order slice products (about 2^-42
of the scale of each row and column).  The FP64 CUDA-core form computes the
same products directly.  Both must give the same expansions to near FP64
rounding; that shows in the energy (Algorithm 3 over every leaf) and in every
dU of a lattice propose, compared here in the FP64 form so that nothing else
rounds at FP32.  Parity of either form with the oracle is covered by the
other GPU tests, which run the default (tensor-core) M2L.

Tolerance.  The dropped slice products and the last slice's residual bound an
M2L entry's error by about K 2^-43 of its row and column scales (K = 2P <= 192
terms per translation at p = 12), i.e. ~2e-11; a dU is a difference of
potentials some ten times larger than itself, so its error relative to max|dU|
can be ten times that: 1e-9 leaves a margin of five.  The energy is a sum of
like-signed terms and keeps 1e-11.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _k():
    import paper_1905_04065_gb300 as k
    return k


def _pair(E, sites, q, L, p):
    k = _k()
    pos = workloads.site_positions(E, sites)
    out = {}
    for m2l in ("tensor", "fp64"):
        h = k.kmc_fmm_init(pos, q, float(E), L, p, precision="fp64", lattice_edge=E, kT=0.1, m2l=m2l)
        U = k.kmc_fmm_energy(h)
        mask, dU = k.kmc_fmm_propose_lattice(h)
        out[m2l] = (U, np.asarray(mask), np.asarray(dU))
        k.kmc_fmm_destroy(h)
    return out


def _check(out, tol_u, tol_du):
    (Ut, mt, dt), (Uf, mf, df) = out["tensor"], out["fp64"]
    assert np.array_equal(mt, mf)
    ok = mf.astype(bool)
    assert abs(Ut - Uf) <= tol_u * abs(Uf), (Ut, Uf)
    err = float(np.max(np.abs(dt[ok] - df[ok])) / np.max(np.abs(df[ok])))
    assert err <= tol_du, err
    return err


def test_medium_tensor_m2l_matches_fp64_m2l():
    w, sites, q = workloads.workload("medium")
    err = _check(_pair(w["E"], sites, q, w["L"], w["p"]), 1e-11, 1e-9)
    print(f"medium: max |dU_tensor - dU_fp64| / max|dU| = {err:.2e}")


@pytest.mark.parametrize("p", [8, 16])
def test_small_tensor_m2l_matches_fp64_m2l(p):
    w, sites, q = workloads.workload("small")
    err = _check(_pair(w["E"], sites, q, w["L"], p), 1e-11, 1e-9)
    print(f"small p={p}: max |dU_tensor - dU_fp64| / max|dU| = {err:.2e}")


def test_mixed_form_four_slice_m2l_matches_fp64_m2l():
    """The mixed form keeps four slices (29 bits): an M2L entry error of about K 2^-28 ~ 7e-7 of its
    row and column scales, ten times that in a dU relative to max|dU|, beside the form's own FP32
    rounding of the near field, L2P and dU (~1e-6): 2e-5 with a margin of two."""
    k = _k()
    w, sites, q = workloads.workload("medium")
    pos = workloads.site_positions(w["E"], sites)
    out = {}
    for m2l in ("tensor", "fp64"):
        h = k.kmc_fmm_init(pos, q, float(w["E"]), w["L"], w["p"], precision="mixed", lattice_edge=w["E"],
                           kT=0.1, m2l=m2l)
        mask, dU = k.kmc_fmm_propose_lattice(h)
        out[m2l] = (np.asarray(mask), np.asarray(dU))
        k.kmc_fmm_destroy(h)
    (mt, dt), (mf, df) = out["tensor"], out["fp64"]
    assert np.array_equal(mt, mf)
    ok = mf.astype(bool)
    err = float(np.max(np.abs(dt[ok] - df[ok])) / np.max(np.abs(df[ok])))
    print(f"medium, mixed form: max |dU_tensor - dU_fp64| / max|dU| = {err:.2e}")
    assert err <= 2e-5, err


def test_tensor_mma_self_check():
    """Four tcgen05 MMAs (M = 128, N = 192, K = 4 x 16) of small integers, staged as the M2L stages
    its operands (cp.async pieces and one 2D TMA box, 128-byte-swizzled K-major tiles, the K step
    advanced inside the swizzle atom), equal the exact product."""
    out = np.zeros((128, 192), np.float32)
    rc = _k().kmc_check_tensor_mma(0, out, kind=0)
    r, n, kk = np.arange(128)[:, None, None], np.arange(192)[None, :, None], np.arange(64)[None, None, :]
    want = (((r * 7 + kk * 3) % 17 - 8) * ((n * 5 + kk * 11) % 13 - 6)).sum(axis=2).astype(np.float32)
    bad = np.argwhere(out != want)
    detail = [(int(i), int(j), float(out[i, j]), float(want[i, j])) for i, j in bad[:12]]
    assert rc == 0 and bad.size == 0, (rc, len(bad), detail, out[:2, :12].tolist(), out[8:10, :12].tolist())


def _tc_pair(E, sites, q, L, p, precision, bc="periodic"):
    k = _k()
    pos = workloads.site_positions(E, sites)
    out = {}
    for m2l in ("tensor", "tensor_sync"):
        h = k.kmc_fmm_init(pos, q, float(E), L, p, precision=precision, lattice_edge=E, kT=0.1, m2l=m2l, bc=bc)
        U = k.kmc_fmm_energy(h)
        mask, dU = k.kmc_fmm_propose_lattice(h)
        out[m2l] = (U, np.asarray(mask).copy(), np.asarray(dU).copy())
        k.kmc_fmm_destroy(h)
    return out


def _identical(out):
    (Ut, mt, dt), (Us, ms, ds) = out["tensor"], out["tensor_sync"]
    assert Ut == Us, (Ut, Us)
    assert np.array_equal(mt, ms)
    ok = mt.astype(bool)  # masked hops carry no dU (NaN in both)
    assert np.array_equal(dt[ok], ds[ok]), float(np.max(np.abs(dt[ok] - ds[ok])))


@pytest.mark.parametrize("p", [8, 10, 12, 14])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tcgen05_m2l_bit_identical_to_mma_sync_medium(p, precision):
    """Both tensor-core forms sum the same exact integer slice products, so the expansions, the
    energy and every dU agree bit for bit (levels 3 and 4 of the medium system: split levels)."""
    w, sites, q = workloads.workload("medium")
    _identical(_tc_pair(w["E"], sites, q, w["L"], p, precision))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tcgen05_m2l_bit_identical_free_space(precision):
    w, sites, q = workloads.workload("medium")
    _identical(_tc_pair(w["E"], sites, q, w["L"], 10, precision, bc="free"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tcgen05_m2l_bit_identical_six_levels(precision):
    """Six levels: the leaf level (32^3 cells, 256 CTAs of 128 target cells) runs without
    interaction-list splits, the coarser levels with them."""
    sites, q = workloads.uniform_lattice(128, 16384, 2024)
    _identical(_tc_pair(128, sites, q, 6, 12, precision))


def test_m2l_timing_hook_leaves_the_state():
    """kmc_fmm_m2l_timed runs the M2L into scratch: per-level times for levels 3 .. L, and every dU
    afterwards bit for bit as before."""
    k = _k()
    w, sites, q = workloads.workload("medium")
    pos = workloads.site_positions(w["E"], sites)
    h = k.kmc_fmm_init(pos, q, float(w["E"]), w["L"], w["p"], precision="mixed", lattice_edge=w["E"], kT=0.1)
    m0, d0 = (np.asarray(a).copy() for a in k.kmc_fmm_propose_lattice(h))
    levels, total = k.kmc_fmm_m2l_timed(h, 2)
    m1, d1 = (np.asarray(a).copy() for a in k.kmc_fmm_propose_lattice(h))
    k.kmc_fmm_destroy(h)
    assert sorted(levels) == list(range(3, w["L"] + 1)) and all(v > 0 for v in levels.values())
    assert total >= sum(levels.values())
    ok = m0.astype(bool)
    assert np.array_equal(m0, m1) and np.array_equal(d0[ok], d1[ok])


def test_tensor_mma_tf32_self_check():
    """Four tcgen05 kind::tf32 MMAs (M = 128, N = 192, K = 4 x 8) of small integers, both operands
    staged as the tensor-core downward pass stages them (2D TMA boxes, 128-byte swizzle), equal the
    exact product."""
    out = np.zeros((128, 192), np.float32)
    rc = _k().kmc_check_tensor_mma(0, out, kind=1)
    r, n, kk = np.arange(128)[:, None, None], np.arange(192)[None, :, None], np.arange(32)[None, None, :]
    want = (((r * 5 + kk * 7) % 23 - 11) * ((n * 3 + kk * 13) % 19 - 9)).sum(axis=2).astype(np.float32)
    bad = np.argwhere(out != want)
    detail = [(int(i), int(j), float(out[i, j]), float(want[i, j])) for i, j in bad[:12]]
    assert rc == 0 and bad.size == 0, (rc, len(bad), detail)
