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
