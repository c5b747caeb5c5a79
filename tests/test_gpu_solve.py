"""GPU parity: assembly (Algorithms 3-4), multiply (Algorithm 5) and the
Jacobi solve of libvf against the oracle's dense FP64 F.

Tolerances:
* block structure: identical except near-ties of the rank rule (the GPU's
  FP32 randomized probe against exact FP64 singular values); the mismatch
  fraction is bounded and every GPU block meets its own invariant;
* dense / CSR entries: the same sparsity pattern, values to FP32 evaluation
  error (1e-6 of A_j / (pi r^2) plus 2e-6 relative);
* SVD blocks: ||F_hat_IJ - F_IJ||_2 <= tol sigma_1(F_IJ) (the default
  assembly checks each factorisation in FP64);
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


def _gpu_decision(gpu, anc, I, J):
    """What the GPU stored for the oracle node (I, J): ('stored', kind, q),
    'above' (a stored GPU block covers a strictly larger pair), 'HIER' (GPU
    blocks strictly inside) or 'ZERO' (nothing stored there)."""
    if (I, J) in gpu:
        return ("stored",) + gpu[(I, J)]
    for a in anc[I]:
        for b in anc[J]:
            if (a, b) != (I, J) and (a, b) in gpu:
                return "above"
    return "INSIDE"


def _near_tie(b, g, Ft, tree, tol, k_max=128, band=1.5, slack=0.02):
    """A divergence at oracle node b is a near-tie when the GPU's choice is
    one of the choices Algorithms 3-4 make under a perturbed rank rule
    (tol / band .. tol * band, the GPU probe's FP32 randomized spectrum
    against exact FP64 singular values; an SVD may carry up to 4 more ranks,
    added by the FP64 check of assembly) and byte costs within `slack`."""
    if b.sv is None or b.hier_bytes < 0:
        return False, "leaf block: dense / CSR costs are exact integers"
    r0, m = tree.first[b.I], tree.count[b.I]
    c0, n = tree.first[b.J], tree.count[b.J]
    A = Ft[r0:r0 + m, c0:c0 + n] != 0
    m1, n1 = int(A.any(1).sum()), int(A.any(0).sum())
    qs = sorted({oracle.numerical_rank(b.sv, tol * f) for f in (1 / band, 1.0, band)})
    cost = {oracle.DENSE: oracle.nbytes_dense(m, n), oracle.CSR: oracle.nbytes_csr(m, b.nnz),
            oracle.HIER: b.hier_bytes}
    svd = [oracle.nbytes_svd(q, m1, n1) for q in qs if q <= k_max]
    best = min(list(cost.values()) + svd)
    if g[0] == "stored":
        kind, q = g[1], g[2]
        if kind == oracle.SVD:
            # the FP64 check may add up to 4 ranks to a factorisation that
            # sits at the threshold; the SVD must still beat the other kinds
            other = min(cost.values())
            ok = qs[0] <= q <= qs[-1] + 4 and oracle.nbytes_svd(q, m1, n1) <= (1 + slack) * other
            return ok, f"GPU SVD q={q}, oracle ranks {qs} in the band, kind {b.kind} q={b.q}"
        ok = cost[kind] <= (1 + slack) * best
        return ok, f"GPU kind {kind} ({cost[kind]} B) vs best {best} B in the band (oracle kind {b.kind} q={b.q})"
    ok = cost[oracle.HIER] <= (1 + slack) * best
    return ok, f"GPU hierarchical ({cost[oracle.HIER]} B) vs best {best} B (oracle kind {b.kind} q={b.q})"


def test_block_structure_matches_oracle(vf, case):
    """The stored blocks equal the oracle's Algorithm 4 except where the two
    diverge at a near-tie of the rank rule or the byte comparison (reading
    R11: the GPU probe's randomized FP32 spectrum against exact FP64 SVDs);
    every divergence is listed and checked to be such a near-tie."""
    tree = case["tree"]
    desc = vf.vf_hmat_blocks(case["prob"].hmat)
    gpu = {(int(d[0]), int(d[1])): (int(d[2]), int(d[3])) for d in desc}
    anc = []
    for k in range(len(tree.count)):
        a, x = [], k
        while x >= 0:
            a.append(x)
            x = int(tree.parent[x])
        anc.append(a)
    div = []

    def walk(b):
        g = _gpu_decision(gpu, anc, b.I, b.J)
        if g == "above":
            return
        if g == "INSIDE":
            if b.kind == oracle.HIER:
                for c in b.children:
                    walk(c)
                return
            if b.kind == oracle.ZERO:
                return
            g = ("hier",)
        elif (b.kind, b.q if b.kind == oracle.SVD else 0) == (g[1], g[2] if g[1] == oracle.SVD else 0):
            return
        div.append((b, g))

    for b in case["top"]:
        walk(b)
    nstored = sum(1 for b in oracle.leaf_blocks(case["top"]) if b.kind != oracle.ZERO)
    report = []
    for b, g in div:
        ok, why = _near_tie(b, g, case["Ft"], tree, case["tol"])
        report.append((ok, (b.I, b.J), why))
    print(f"{case['name']}: {len(div)} divergences from the oracle's {nstored} stored blocks")
    for ok, ij, why in report:
        print(f"  {'near-tie' if ok else 'NOT A TIE'} at {ij}: {why}")
    assert all(ok for ok, _, _ in report), [r for r in report if not r[0]]
    # the check's extra rank at the threshold is the usual divergence; the
    # rest of the structure is identical
    assert len(div) <= 0.5 * nstored
    # the stored blocks tile the matrix exactly once
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
            # the default assembly checks every factorisation in FP64 (verify on)
            assert err <= tol * s1, f"block {tuple(d[:2])}: {err / s1:.3e} > tol"


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


@pytest.mark.parametrize("prec,bound", [("bf16", 1.2e-2), ("fp8", 1.5e-1)])
def test_apply_low_precision_against_oracle(vf, case, prec, bound):
    """BF16 / FP8 E4M3 (per-block scale) multiplies against the oracle's
    FP64 F: compression (2 tol, reading R8) plus the factors' rounding."""
    import torch
    om, F, tol = case["om"], case["F"], case["tol"]
    X = synth.uniform_columns(om.n, 4, seed=6)
    Xt = torch.tensor(X.T.copy(), device="cuda", dtype=torch.float32)
    Y = torch.empty_like(Xt)
    vf.vf_apply(case["prob"].hmat, Xt, Y, precision=prec)
    Yo = F @ X
    err = np.linalg.norm(Y.double().cpu().numpy().T - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
    assert np.all(err <= 2 * tol + bound), err


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_solve_refined_low_precision_against_oracle(vf, case, prec):
    """BF16 / FP8 sweeps with FP64-residual refinement reach the oracle's
    FP64 solution of the uncompressed system to the compression error
    (2 tol), like the FP32 solve."""
    import torch
    om, F, tol = case["om"], case["F"], case["tol"]
    dirs = synth.sun_directions(3, 25.0)
    E = torch.empty((3, om.n), device="cuda")
    vf.vf_mesh_insolation(case["prob"].mesh, dirs, 1365.0, E)
    B = torch.empty_like(E)
    st = vf.vf_solve(case["prob"].hmat, E, B, rho=0.5, rtol=1e-7, precision=prec, refine=True)
    assert st["converged"] == 1
    Bo, _, _ = oracle.jacobi(lambda X: F @ X, oracle.insolation(om, dirs, 1365.0), 0.5, rtol=1e-12)
    err = np.linalg.norm(B.double().cpu().numpy().T - Bo, axis=0) / np.linalg.norm(Bo, axis=0)
    assert np.all(err <= 2 * tol), err


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
