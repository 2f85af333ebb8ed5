"""The mixed form's per-step downward pass on the tensor cores against its CUDA-core form.

On the finest level, when it has at least 4096 parents, the L2L translations of the accumulated
local expansions run as tcgen05 kind::tf32 MMAs with every FP32 operand split into two TF32
parts, each rounded to nearest (hi hi + hi lo + lo hi, FP32 accumulation): about 3 2^-22 = 7e-7
relative error per product, against 2^-24 = 6e-8 per FP32 operation of the CUDA-core form, whose
expansions are themselves FP32 values.  Both mixed forms are compared with the FP64 form on the
same system and order (the same truncation, so the difference is the arithmetic alone): the
tensor-core form's largest dU error may exceed the CUDA-core form's by at most a quarter plus
2e-6 of max|dU|, and the two mixed forms agree within 1e-5 of max|dU| (measured 4e-6 on the
six-level system, 7e-6 on the 1M-charge workload, whose potentials are larger sums)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _run(E, sites, q, L, p, precision, l2l="tensor"):
    import paper_1905_04065_gb300 as k
    pos = workloads.site_positions(E, sites)
    h = k.kmc_fmm_init(pos, q, float(E), L, p, precision=precision, lattice_edge=E, kT=0.05, l2l=l2l)
    mask, dU = (np.asarray(a).copy() for a in k.kmc_fmm_propose_lattice(h))
    k.kmc_fmm_destroy(h)
    return mask, dU


def _compare(E, sites, q, L, p, label):
    m64, d64 = _run(E, sites, q, L, p, "fp64")
    mt, dt = _run(E, sites, q, L, p, "mixed", "tensor")
    mc, dc = _run(E, sites, q, L, p, "mixed", "cuda")
    assert np.array_equal(mt, mc) and np.array_equal(mt, m64)
    ok = mt.astype(bool)
    scale = np.max(np.abs(d64[ok]))
    e_t = float(np.max(np.abs(dt[ok] - d64[ok])) / scale)
    e_c = float(np.max(np.abs(dc[ok] - d64[ok])) / scale)
    e_tc = float(np.max(np.abs(dt[ok] - dc[ok])) / scale)
    print(f"{label}: vs FP64 form: tensor {e_t:.2e}, cuda {e_c:.2e}; tensor vs cuda {e_tc:.2e}")
    assert e_t <= 1.25 * e_c + 2e-6, (e_t, e_c)
    assert e_tc < 1e-5, e_tc


def test_tensor_core_downward_pass_six_levels():
    sites, q = workloads.uniform_lattice(128, 16384, 2024)
    _compare(128, sites, q, 6, 12, "six levels, p = 12")


def test_tensor_core_downward_pass_large_workload():
    w, sites, q = workloads.workload("large")
    _compare(w["E"], sites, q, w["L"], w["p"], "large")


@pytest.mark.parametrize("p", [8, 10, 14])
def test_tensor_core_downward_pass_orders(p):
    sites, q = workloads.uniform_lattice(128, 16384, 2025)
    _compare(128, sites, q, 6, p, f"six levels, p = {p}")
