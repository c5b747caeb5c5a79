"""vf_apply_tree_static: the multiply with the library's fixed static scratch.

Collected last on purpose (file name), and independent of every other test:
it builds its own problem, so it passes alone and after the rest.  It checks
that the call gives the same bits as vf_apply_tree on two calls in a row,
that it leaves device memory untouched once the module is loaded, and that a
shape needing more than the static scratch is rejected before any launch.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def terrain():
    import torch

    import synth
    from paper_2209_07632_gb300 import vf
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    v, f = synth.fbm_dem_mesh(n=48, seed=5)
    prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=1e-3, precisions=("fp32", "bf16"))
    return prob


@pytest.mark.parametrize("R,precision", [(1, "fp32"), (3, "fp32"), (8, "bf16")])
def test_static_matches_workspace_path(terrain, R, precision):
    import torch

    from paper_2209_07632_gb300 import vf
    h = terrain.hmat
    n = h.n
    g = torch.Generator(device="cpu").manual_seed(100 + R)
    Xt = torch.rand((R, n), generator=g).cuda()
    Y_ws = [torch.empty_like(Xt) for _ in range(2)]
    Y_st = [torch.full_like(Xt, float("nan")) for _ in range(2)]
    for k in range(2):
        vf.vf_apply_tree(h, Xt, Y_ws[k], precision=precision)
    torch.cuda.synchronize()
    for k in range(2):  # two calls in a row through the static scratch
        vf.vf_apply_tree_static(h, Xt, Y_st[k], precision=precision)
    assert torch.equal(Y_ws[0], Y_ws[1])
    assert torch.equal(Y_st[0], Y_ws[0])
    assert torch.equal(Y_st[1], Y_ws[0])


def test_static_allocates_nothing(terrain):
    import torch

    from paper_2209_07632_gb300 import vf
    h = terrain.hmat
    Xt = torch.rand((2, h.n)).cuda()
    Yt = torch.empty_like(Xt)
    vf.vf_apply_tree_static(h, Xt, Yt)  # first call: module and kernel attributes already set up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        vf.vf_apply_tree_static(h, Xt, Yt)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_rejects_oversize(terrain):
    import torch

    from paper_2209_07632_gb300 import vf
    h = terrain.hmat
    # enough columns that the T vectors exceed the static scratch
    desc = vf.vf_hmat_blocks(h)
    nT = int(desc[:, 3][desc[:, 2] == 3].sum())  # T slots: the ranks of the SVD blocks
    assert nT >= 1000, "the test terrain should have SVD blocks"
    R = vf.VF_STATIC_T_FLOATS // nT + 9
    Xt = torch.zeros((R, h.n), device="cuda")
    Yt = torch.full_like(Xt, 7.0)
    with pytest.raises(vf.VFError) as ei:
        vf.vf_apply_tree_static(h, Xt, Yt)
    assert ei.value.status == vf.VF_E_INVAL
    assert "limit" in str(ei.value)
    assert bool((Yt == 7.0).all())  # nothing was launched
