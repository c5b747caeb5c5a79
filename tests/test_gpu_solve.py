"""GPU parity: assembly (Algorithms 3-4), multiply (Algorithm 5) and the
Jacobi solve of libvf against the oracle's dense FP64 F.

Tolerances:
* block structure: identical except near-ties of the rank rule (the GPU's
  FP32 randomized probe against exact FP64 singular values); the mismatch
  fraction is bounded and every GPU block meets its own invariant;
* dense / CSR entries: the same sparsity pattern, values to FP32 evaluation
  error (1e-6 of A_j / (pi r^2) plus 2e-6 relative);
* SVD blocks: ||F_hat_IJ - F_IJ||_2 <= tol sigma_1(F_IJ) (5% slack for
  FP32 entries and the probe);
* multiply and solve in FP32: relative error per column <= 2 tol;
* BF16/FP8 sweeps with FP64-residual refinement: within 1e-5 of the FP32
  solve on the same compressed F, hence within 2 tol of the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf as _vf
    return _vf


def _dense_from_gpu(vf, h, n):
    """F_hat in face order, by applying it to the identity."""
    import torch
    I = torch.eye(n, device="cuda", dtype=torch.float32)
    Y = torch.empty_like(I)
    vf.vf_apply(h, I, Y)
    return Y.double().cpu().numpy().T  # Y[r] = F_hat e_r -> column r


CASES = {
    "cap_1e-3": (lambda: synth.cap_bowl_mesh(), "quad", 1e-3),
    "cap_1e-2": (lambda: synth.cap_bowl_mesh(), "quad", 1e-2),
    "dem30_1e-3": (lambda: synth.fbm_dem_mesh(n=30, seed=3, crater_diameter=120.0), "quad", 1e-3),
    "sphere3_1e-3": (lambda: synth.gaussian_sphere_mesh(level=3, sigma=0.3, seed=4), "oct", 1e-3),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, vf):
    mk, kind, tol = CASES[request.param]
    v, f = mk()
    om = oracle.mesh(v, f)
    V = oracle.visibility_rows(om, np.arange(om.n))
    F = oracle.F_rows(om, np.arange(om.n), V)
    tree = oracle.partition(om, kind, 64)
    Ft = F[np.ix_(tree.perm, tree.perm)]
    top = oracle.assemble(Ft, tree, tol)
    prob = vf.build_problem(v, f, kind=kind, leaf_size=64, tol=tol, precisions=("fp32", "bf16", "fp8"))
    Fh = _dense_from_gpu(vf, prob.hmat, om.n)
    return dict(name=request.param, v=v, f=f, om=om, F=F, tree=tree, Ft=Ft, top=top, prob=prob, Fh=Fh, tol=tol)


def test_block_structure_matches_oracle(vf, case):
    desc = vf.vf_hmat_blocks(case["prob"].hmat)
    gpu = {(int(d[0]), int(d[1])): (int(d[2]), int(d[3])) for d in desc}
    ora = {(b.I, b.J): (b.kind, b.q) for b in oracle.leaf_blocks(case["top"]) if b.kind != oracle.ZERO}
    same = sum(1 for k, v in ora.items() if gpu.get(k) == v)
    frac = same / max(len(ora), 1)
    # near-ties of the rank rule can flip a block's representation
    assert frac >= 0.9, f"{case['name']}: only {frac:.3f} of blocks identical"
    # the stored blocks tile the matrix exactly once
    tree = case["tree"]
    cover = np.zeros((case["om"].n, case["om"].n), dtype=np.int32)
    for d in desc:
        r0, m = tree.first[d[0]], tree.count[d[0]]
        c0, n = tree.first[d[1]], tree.count[d[1]]
        cover[r0:r0 + m, c0:c0 + n] += 1
    # zero blocks are not stored: uncovered entries must be zero in F
    assert cover.max() == 1
    assert np.all(case["Ft"][cover == 0] == 0)


def _entry_scale(om, rows, cols):
    """A_j / (pi r_ij^2): the size of F_ij's terms before the two cosines, so
    FP32 cancellation in a cosine is bounded by a few ulps of this."""
    d = om.cent[cols][None, :, :] - om.cent[rows][:, None, :]
    r2 = np.maximum((d * d).sum(-1), 1e-300)
    return om.area[cols][None, :] / (np.pi * r2)


def test_blocks_meet_their_invariants(vf, case):
    tree, Ft, tol = case["tree"], case["Ft"], case["tol"]
    perm = tree.perm
    Fht = case["Fh"][np.ix_(perm, perm)]
    for d in vf.vf_hmat_blocks(case["prob"].hmat):
        r0, m = tree.first[d[0]], tree.count[d[0]]
        c0, n = tree.first[d[1]], tree.count[d[1]]
        A = Ft[r0:r0 + m, c0:c0 + n]
        Ah = Fht[r0:r0 + m, c0:c0 + n]
        if d[2] in (1, 2):  # dense, CSR: the entries themselves, to FP32 evaluation error
            rows, cols = perm[r0:r0 + m], perm[c0:c0 + n]
            assert np.array_equal(Ah != 0, A != 0)
            assert np.all(np.abs(Ah - A) <= 1e-6 * _entry_scale(case["om"], rows, cols) + 2e-6 * np.abs(A))
        else:
            s1 = np.linalg.norm(A, 2)
            err = np.linalg.norm(Ah - A, 2)
            assert err <= 1.05 * tol * s1, f"block {tuple(d[:2])}: {err / s1:.3e} > tol"


def test_apply_fp32_within_two_tol(vf, case):
    import torch
    om, F, tol = case["om"], case["F"], case["tol"]
    rng_cols = synth.uniform_columns(om.n, 13, seed=11)
    for R in (1, 3, 8, 13):
        X = rng_cols[:, :R]
        Xt = torch.tensor(X.T.copy(), device="cuda", dtype=torch.float32)
        Y = torch.empty_like(Xt)
        vf.vf_apply(case["prob"].hmat, Xt, Y)
        Yg = Y.double().cpu().numpy().T
        Yo = F @ X
        err = np.linalg.norm(Yg - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
        assert np.all(err <= 2 * tol), (R, err)


@pytest.mark.parametrize("prec,bound", [("bf16", 1.2e-2), ("fp8", 1.5e-1)])
def test_apply_low_precision(vf, case, prec, bound):
    """BF16 (8-bit mantissa) and FP8 E4M3 (3-bit mantissa, per-block scale)
    factors against the FP32 factors of the same matrix."""
    import torch
    om = case["om"]
    X = synth.uniform_columns(om.n, 4, seed=5)
    Xt = torch.tensor(X.T.copy(), device="cuda", dtype=torch.float32)
    Y32 = torch.empty_like(Xt)
    Ylp = torch.empty_like(Xt)
    vf.vf_apply(case["prob"].hmat, Xt, Y32, precision="fp32")
    vf.vf_apply(case["prob"].hmat, Xt, Ylp, precision=prec)
    a = Y32.double().cpu().numpy()
    b = Ylp.double().cpu().numpy()
    err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(a, axis=1)
    assert np.all(err < bound), err


def test_solve_fp32_matches_oracle(vf, case):
    import torch
    om, F, tol = case["om"], case["F"], case["tol"]
    dirs = synth.sun_directions(4, 15.0)
    E = torch.empty((4, om.n), device="cuda")
    vf.vf_mesh_insolation(case["prob"].mesh, dirs, 1365.0, E)
    B = torch.empty_like(E)
    st = vf.vf_solve(case["prob"].hmat, E, B, rho=0.12, rtol=1e-7)
    assert st["converged"] == 1
    Eo = oracle.insolation(om, dirs, 1365.0)
    Bo, iters, _ = oracle.jacobi(lambda X: F @ X, Eo, 0.12, rtol=1e-12)
    Bg = B.double().cpu().numpy().T
    err = np.linalg.norm(Bg - Bo, axis=0) / np.linalg.norm(Bo, axis=0)
    assert np.all(err <= 2 * tol), err


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_solve_refined_low_precision(vf, case, prec):
    import torch
    om = case["om"]
    dirs = synth.sun_directions(3, 25.0)
    E = torch.empty((3, om.n), device="cuda")
    vf.vf_mesh_insolation(case["prob"].mesh, dirs, 1365.0, E)
    B32 = torch.empty_like(E)
    Blp = torch.empty_like(E)
    vf.vf_solve(case["prob"].hmat, E, B32, rho=0.5, rtol=1e-7)
    st = vf.vf_solve(case["prob"].hmat, E, Blp, rho=0.5, rtol=1e-6, precision=prec, refine=True)
    assert st["converged"] == 1
    a, b = B32.double().cpu().numpy(), Blp.double().cpu().numpy()
    err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(a, axis=1)
    assert np.all(err < 1e-5), err


def test_solve_edge_cases(vf, case):
    import torch
    om, h = case["om"], case["prob"].hmat
    E = torch.zeros((2, om.n), device="cuda")
    E[1] = 1.0
    B = torch.full_like(E, 7.0)
    st = vf.vf_solve(h, E, B, rho=0.12, rtol=1e-7, clamp=True)
    assert torch.all(B[0] == 0)
    assert torch.all(B[1] >= 0.999)
    st = vf.vf_solve(h, E, B, rho=0.9, rtol=1e-12, max_iter=1)
    assert st["converged"] == 0 and st["sweeps"] == 1


def test_save_load_roundtrip(vf, case, tmp_path):
    import torch
    p = str(tmp_path / "f.vfh")
    vf.vf_hmat_save(case["prob"].hmat, p)
    h2 = vf.vf_hmat_load(p)
    X = torch.rand((5, case["om"].n), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    Y1 = torch.empty_like(X)
    Y2 = torch.empty_like(X)
    vf.vf_apply(case["prob"].hmat, X, Y1)
    vf.vf_apply(h2, X, Y2)
    assert torch.equal(Y1, Y2)
    # a flipped byte in the payload is caught by the section CRC
    raw = bytearray(open(p, "rb").read())
    raw[-40] ^= 0x5A
    bad = str(tmp_path / "bad.vfh")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(vf.VFError) as e:
        vf.vf_hmat_load(bad)
    assert e.value.status == vf.VF_E_CORRUPT


def test_apply_deterministic(vf, case):
    import torch
    X = torch.rand((3, case["om"].n), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    Y1 = torch.empty_like(X)
    Y2 = torch.empty_like(X)
    vf.vf_apply(case["prob"].hmat, X, Y1)
    vf.vf_apply(case["prob"].hmat, X, Y2)
    assert torch.equal(Y1, Y2)
