"""FP8 E4M3 on the tensor cores (kind::f8f6f4 MMAs on K-major FP8 panels
and pages, FP32 accumulation in tensor memory; power-of-two scales per RHS
column, per matrix row and per SVD rank column, undone in the epilogues)
against the FP32 CUDA-core multiply and the FP64 oracle, and refined FP8
solves (split-BF16 residual) against the oracle's solution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf as _vf
    return _vf


def _rel(a, b):
    return ((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-30)).max().item()


@pytest.fixture(scope="module")
def terrain(vf):
    import synth
    v, f = synth.fbm_dem_mesh(n=40, seed=8)
    return vf.build_problem(v, f, tol=1e-3, precisions=("fp32", "bf16", "fp8"))


@pytest.fixture(scope="module")
def cap(vf):
    import oracle
    import synth
    v, f = synth.cap_bowl_mesh()
    prob = vf.build_problem(v, f, tol=1e-3, precisions=("fp32", "fp8"))
    om = oracle.mesh(v, f)
    return prob, om, oracle.F_dense(om)


# E4M3 keeps 3 mantissa bits: the factors, the right-hand sides and T each
# round to at most 2^-4 relative (half that on average); sums of many
# nonnegative terms keep the product's relative error well below that
TOL_FP8 = 6e-2


@pytest.mark.parametrize("R", [16, 128, 129, 300])
def test_fp8_tensor_apply_matches_fp32(vf, terrain, R):
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    X = torch.rand((R, n), generator=torch.Generator().manual_seed(R)).cuda()
    Y32 = torch.empty_like(X)
    Y8 = torch.empty_like(X)
    vf.vf_apply(h, X, Y32, precision="fp32")
    vf.vf_apply(h, X, Y8, precision="fp8")
    assert _rel(Y8, Y32) <= TOL_FP8
    perm = torch.from_numpy(vf.vf_tree_perm(terrain.tree).astype(np.int64)).cuda()
    Xt = X[:, perm].contiguous()
    Yt = torch.empty_like(Xt)
    vf.vf_apply_tree(h, Xt, Yt, precision="fp8")
    assert torch.equal(Yt, Y8[:, perm])


def test_fp8_tensor_apply_deterministic_and_scale_free(vf, terrain):
    # the per-column scales are powers of two, so scaling a column by 2^k
    # scales its product by exactly 2^k
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    X = torch.rand((128, n), generator=torch.Generator().manual_seed(3)).cuda()
    Y = [torch.empty_like(X) for _ in range(3)]
    vf.vf_apply(h, X, Y[0], precision="fp8")
    vf.vf_apply(h, X, Y[1], precision="fp8")
    assert torch.equal(Y[0], Y[1])
    vf.vf_apply(h, X * 1024.0, Y[2], precision="fp8")
    assert torch.equal(Y[2], Y[0] * 1024.0)


def test_fp8_pages_are_smaller(vf, terrain):
    b1 = vf.vf_hmat_tensor_bytes(terrain.hmat, 1)
    b3 = vf.vf_hmat_tensor_bytes(terrain.hmat, 3)
    assert 0 < b3["total"] < b1["total"]


def test_fp8_tensor_apply_against_oracle(vf, cap):
    import torch

    import oracle
    import synth
    prob, om, F = cap
    E = oracle.insolation(om, synth.sun_directions(32, 10.0), 1365.0)  # (n, 32)
    ref = F @ E
    X = torch.tensor(np.ascontiguousarray(E.T), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    vf.vf_apply(prob.hmat, X, Y, precision="fp8")
    got = Y.cpu().numpy().T.astype(np.float64)
    live = np.linalg.norm(ref, axis=0) > 0
    err = np.linalg.norm(got - ref, axis=0)[live] / np.linalg.norm(ref, axis=0)[live]
    assert np.all(err <= 2e-3 + TOL_FP8), err.max()


def test_fp8_tensor_refined_solve_against_oracle(vf, cap):
    """FP8 sweeps on the tensor cores with the split-BF16 residual reach the
    oracle's FP64 solution of the uncompressed system to the compression
    error (2 tol), like the FP32 solve."""
    import torch

    import oracle
    import synth
    prob, om, F = cap
    dirs = synth.sun_directions(32, 25.0)
    E = torch.empty((32, om.n), device="cuda")
    vf.vf_mesh_insolation(prob.mesh, dirs, 1365.0, E)
    B = torch.empty_like(E)
    st = vf.vf_solve(prob.hmat, E, B, rho=0.5, rtol=1e-7, precision="fp8", refine=True)
    assert st["converged"] == 1 and st["refinements"] >= 1
    Bo, _, _ = oracle.jacobi(lambda X: F @ X, oracle.insolation(om, dirs, 1365.0), 0.5, rtol=1e-12)
    Bg = B.double().cpu().numpy().T
    live = np.linalg.norm(Bo, axis=0) > 0
    err = np.linalg.norm(Bg - Bo, axis=0)[live] / np.linalg.norm(Bo, axis=0)[live]
    assert np.all(err <= 2e-3), err.max()


@pytest.mark.parametrize("R", [128, 300])
def test_fp8_tensor_refined_solve_matches_fp32(vf, terrain, R):
    import torch

    import synth
    h, m = terrain.hmat, terrain.mesh
    E = torch.empty((R, m.n), device="cuda")
    vf.vf_mesh_insolation(m, synth.sun_directions(R, 6.0), 1365.0, E)
    B32, B8 = torch.empty_like(E), torch.empty_like(E)
    vf.vf_solve(h, E, B32, rho=0.12, rtol=1e-7)
    st = vf.vf_solve(h, E, B8, rho=0.12, rtol=1e-7, precision="fp8", refine=True)
    assert st["converged"] == 1 and st["refinements"] >= 1
    live = B32.norm(dim=1) > 0
    err = ((B8 - B32).norm(dim=1)[live] / B32.norm(dim=1)[live]).max().item()
    assert err <= 1e-5, err
