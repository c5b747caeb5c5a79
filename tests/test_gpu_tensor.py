"""The tensor-core multiply (BF16 factors and right-hand sides, tcgen05 MMAs,
FP32 accumulation in tensor memory) for panels of 128 columns, against the
FP32 CUDA-core multiply and the FP64 oracle."""
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
    return vf.build_problem(v, f, tol=1e-3, precisions=("fp32", "bf16"))


# BF16 rounds the factors, the right-hand sides and T (relative 2^-9 each);
# the sums of nonnegative terms keep the product's relative error near that
TOL_BF16 = 4e-3


@pytest.mark.parametrize("R", [16, 128, 129, 300])
def test_tensor_apply_matches_fp32(vf, terrain, R):
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    X = torch.rand((R, n), generator=torch.Generator().manual_seed(R)).cuda()
    Y32 = torch.empty_like(X)
    Ytc = torch.empty_like(X)
    vf.vf_apply(h, X, Y32, precision="fp32")
    vf.vf_apply(h, X, Ytc, precision="bf16")
    assert _rel(Ytc, Y32) <= TOL_BF16
    # the tree-order entry point gives the same product
    perm = torch.from_numpy(vf.vf_tree_perm(terrain.tree).astype(np.int64)).cuda()
    Xt = X[:, perm].contiguous()
    Yt = torch.empty_like(Xt)
    vf.vf_apply_tree(h, Xt, Yt, precision="bf16")
    assert torch.equal(Yt, Ytc[:, perm])


def test_tensor_apply_deterministic(vf, terrain):
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    X = torch.rand((128, n), generator=torch.Generator().manual_seed(3)).cuda()
    Y = [torch.empty_like(X) for _ in range(2)]
    for y in Y:
        vf.vf_apply(h, X, y, precision="bf16")
    assert torch.equal(Y[0], Y[1])


def test_tensor_apply_unit_columns(vf, terrain):
    # e_k columns: each output column is one column of F-hat; every block's
    # piece lands in the right rows (a misplaced block would change nonzeros)
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    cols = np.linspace(0, n - 1, 16).astype(int)
    E = torch.zeros((16, n), device="cuda")
    for i, c in enumerate(cols):
        E[i, c] = 1.0
    A = torch.empty_like(E)
    B = torch.empty_like(E)
    vf.vf_apply(h, E, A, precision="fp32")
    vf.vf_apply(h, E, B, precision="bf16")
    assert _rel(B, A) <= TOL_BF16
    assert torch.equal(A != 0, B != 0)


def test_tensor_apply_against_oracle(vf):
    import torch

    import oracle
    import synth
    v, f = synth.cap_bowl_mesh()
    prob = vf.build_problem(v, f, tol=1e-3, precisions=("fp32", "bf16"))
    om = oracle.mesh(v, f)
    F = oracle.F_dense(om)
    E = oracle.insolation(om, synth.sun_directions(32, 10.0), 1365.0)  # (n, 32)
    ref = F @ E
    X = torch.tensor(np.ascontiguousarray(E.T), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    vf.vf_apply(prob.hmat, X, Y, precision="bf16")
    got = Y.cpu().numpy().T.astype(np.float64)
    live = np.linalg.norm(ref, axis=0) > 0
    err = np.linalg.norm(got - ref, axis=0)[live] / np.linalg.norm(ref, axis=0)[live]
    assert np.all(err <= 2e-3 + TOL_BF16), err.max()


@pytest.mark.parametrize("R", [128, 300])
def test_tensor_refined_solve_matches_fp32(vf, terrain, R):
    # BF16 sweeps on the tensor cores, split-BF16 residual (pairs of 128-RHS
    # panels where there are two): within 1e-5 of the FP32 CUDA-core solve
    import torch

    import synth
    h, m = terrain.hmat, terrain.mesh
    E = torch.empty((R, m.n), device="cuda")
    vf.vf_mesh_insolation(m, synth.sun_directions(R, 6.0), 1365.0, E)
    B32, Bt = torch.empty_like(E), torch.empty_like(E)
    vf.vf_solve(h, E, B32, rho=0.12, rtol=1e-7)
    st = vf.vf_solve(h, E, Bt, rho=0.12, rtol=1e-7, precision="bf16", refine=True)
    assert st["converged"] == 1 and st["refinements"] >= 1
    live = B32.norm(dim=1) > 0
    err = ((Bt - B32).norm(dim=1)[live] / B32.norm(dim=1)[live]).max().item()
    assert err <= 1e-5, err


def test_tensor_bytes_and_trim(vf, terrain):
    # the tensor pages' bytes add up by record kind; trimming the handle's
    # caches and rebuilding them gives the same product bit for bit
    import torch
    h, n = terrain.hmat, terrain.mesh.n
    b1 = vf.vf_hmat_tensor_bytes(h, 1)
    b2 = vf.vf_hmat_tensor_bytes(h, 2)
    recs = sum(b1[k] for k in ("dense", "csr", "svd_u", "svd_v", "empty"))
    # the total adds a 16-byte header per page (pages hold 12 KB)
    assert 0 < recs <= b1["total"] <= recs + 16 * (b1["total"] // 1000 + 1)
    assert b2["total"] > 1.5 * b1["total"]
    X = torch.rand((128, n), generator=torch.Generator().manual_seed(4)).cuda()
    Y0, Y1 = torch.empty_like(X), torch.empty_like(X)
    vf.vf_apply(h, X, Y0, precision="bf16")
    vf.vf_hmat_trim(h)
    vf.vf_apply(h, X, Y1, precision="bf16")
    assert torch.equal(Y0, Y1)
    assert vf.vf_hmat_tensor_bytes(h, 1) == b1
