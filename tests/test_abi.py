"""The C-ABI library builds, loads and exports every symbol include/vf.h
declares (no GPU needed: nothing here launches device work)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(vf_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf
    return vf.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("vf_mesh_create", "vf_partition", "vf_assemble", "vf_apply", "vf_solve", "vf_solve_batched",
                 "vf_mesh_insolation", "vf_hmat_save", "vf_hmat_load"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_the_header():
    from paper_2209_07632_gb300 import vf
    assert set(vf.declared_symbols()) <= _declared()


def test_host_side_errors_without_gpu(lib):
    """Argument checks happen before any device call."""
    import ctypes
    out = ctypes.c_void_p()
    assert lib.vf_mesh_create(None, 0, None, 0, None, ctypes.byref(out)) == 1  # VF_E_INVAL
    assert b"null" in lib.vf_last_error()
    assert lib.vf_apply(None, 0, None, 0, 1, None, 0, None) == 1
    assert lib.vf_hmat_load(b"/nonexistent/file.vfh", 0, ctypes.byref(out)) == 7  # VF_E_IO


def test_static_scratch_limits_match_header():
    from paper_2209_07632_gb300 import vf
    txt = open(os.path.join(ROOT, "include", "vf.h")).read()
    for name in ("VF_STATIC_T_FLOATS", "VF_STATIC_PART_FLOATS"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", txt)
        assert m and int(m.group(1)) == getattr(vf, name)


def test_predictor_sizes_match_header():
    from oracle import mlp
    from paper_2209_07632_gb300 import vf
    txt = open(os.path.join(ROOT, "include", "vf.h")).read()
    for name in ("VF_PRED_NFEAT", "VF_PRED_NCLASS", "VF_PRED_NPARAM"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", txt)
        assert m and int(m.group(1)) == getattr(vf, name)
    assert vf.VF_PRED_NPARAM == mlp.NPARAM and vf.VF_PRED_NFEAT == mlp.NF and vf.VF_PRED_NCLASS == mlp.NC


@pytest.mark.parametrize("fn", ["vf_apply_tree", "vf_apply_tree_static"])
def test_tree_multiply_rejects_a_mismatched_output(fn):
    """Yt must have Xt's shape: the binding refuses before the library is called
    (a smaller Yt would otherwise receive R x N floats)."""
    import torch

    from paper_2209_07632_gb300 import vf
    h = vf.HMat(None)  # never reached: the shape check comes first
    Xt = torch.zeros((8, 10))
    for Yt in (torch.zeros(10), torch.zeros((2, 10)), torch.zeros((8, 11))):
        with pytest.raises(vf.VFError) as ei:
            getattr(vf, fn)(h, Xt, Yt)
        assert ei.value.status == vf.VF_E_INVAL
        assert "shape" in str(ei.value)
