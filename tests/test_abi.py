"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/kmcfmm.h declares (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kmcfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(kmc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("kmc_fmm_init", "kmc_fmm_propose", "kmc_fmm_accept", "kmc_step", "kmc_fmm_destroy",
              "kmc_fmm_propose_lattice", "kmc_run", "kmc_fmm_recompute", "kmc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1905_04065_gb300 import EXPORTS, build_library
    lib = ctypes.CDLL(build_library())
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(EXPORTS) == _declared()


def test_binding_loads_without_device():
    import paper_1905_04065_gb300 as k
    lib = k.load_library()
    opts = k.kmc_opts()
    lib.kmc_opts_default(ctypes.byref(opts))  # pure host function
    assert opts.precision == k.KMC_PREC_FP64 and opts.lattice_h == 1.0 and opts.mem == k.KMC_MEM_HOST
    assert opts.m2l == k.KMC_M2L_TENSOR
    assert lib.kmc_last_error(None) is not None


def test_null_handle_is_rejected():
    import paper_1905_04065_gb300 as k
    lib = k.load_library()
    U = ctypes.c_double()
    assert lib.kmc_fmm_energy(None, ctypes.byref(U)) == k.KMC_ERR_ARG
    lib.kmc_fmm_destroy(None)


def test_proposal_tuples_flatten_in_order():
    """The tuple-list form of the proposals (Sec. 4.2) flattens charge by charge, targets in
    their given order, with offsets that split the energy changes back per charge."""
    import paper_1905_04065_gb300 as k
    P = ((3, [[0.11, 0.13, 0.09], [0.90, 0.10, 0.08]]), (7, [[0.45, 0.28, 0.89]]), (3, np.zeros((0, 3))))
    part, tgt, off = k.flatten_proposals(P)
    assert part.dtype == np.int32 and part.tolist() == [3, 3, 7]
    assert tgt.shape == (3, 3) and tgt[1].tolist() == [0.90, 0.10, 0.08] and tgt[2].tolist() == [0.45, 0.28, 0.89]
    assert off.tolist() == [0, 2, 3, 3]
    part, tgt, off = k.flatten_proposals(())
    assert part.shape == (0,) and tgt.shape == (0, 3) and off.tolist() == [0]


def test_options_struct_layout_matches_the_header():
    """kmc_opts_default fills exactly the binding's kmc_opts: the bytes after it stay untouched
    (a C struct larger than the binding's would overwrite them), and every field, the last one
    included, gets its documented default."""
    import paper_1905_04065_gb300 as k
    lib = k.load_library()
    n = ctypes.sizeof(k.kmc_opts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    lib.kmc_opts_default(ctypes.cast(buf, ctypes.c_void_p))
    assert bytes(buf[n:]) == b"\xab" * 64
    opts = k.kmc_opts.from_buffer_copy(bytes(buf[:n]))
    assert opts.kT == 1.0 and opts.lattice_edge == 0 and opts.hops == k.KMC_HOPS_6
    assert opts.bc == k.KMC_BC_PERIODIC and opts.field_z == 0.0 and opts.near_cache == 0


def test_checkpoint_round_trip_host_logic(tmp_path, monkeypatch):
    """kmc_checkpoint stores positions, charges, the creation arguments and the step counter;
    kmc_resume re-creates the handle from exactly those (the device calls are faked here)."""
    import paper_1905_04065_gb300 as k

    class Fake:
        n = 3
        init_args = dict(charges=np.array([1.0, -1.0, 0.0]), box=4.0, levels=3, order=8, precision="mixed",
                         lattice_edge=4, lattice_h=1.0, kT=0.1, leaf_capacity=0, m2l="tensor", hops=14,
                         bc="free", field_z=0.0, near_cache=True)
    pos = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5], [2.5, 3.5, 1.5]])
    monkeypatch.setattr(k, "kmc_fmm_positions", lambda h: pos)
    seen = {}

    def fake_init(positions, charges, **kw):
        seen.update(positions=np.array(positions), charges=np.array(charges), **kw)
        return "handle"
    monkeypatch.setattr(k, "kmc_fmm_init", fake_init)
    path = str(tmp_path / "state.npz")
    k.kmc_checkpoint(Fake(), path, step=123, seed=np.array([7, 8]))
    h, step, extra = k.kmc_resume(path)
    assert h == "handle" and step == 123 and extra["seed"].tolist() == [7, 8]
    assert np.array_equal(seen["positions"], pos) and seen["charges"].tolist() == [1.0, -1.0, 0.0]
    for key, v in Fake.init_args.items():
        if key != "charges":
            assert seen[key] == v, key
