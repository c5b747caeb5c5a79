"""Many meshes in one launch per phase: the block-diagonal stack of several
compressed matrices multiplies and solves exactly like its meshes one by
one, and the batched solve judges convergence per mesh and column."""
import numpy as np
import pytest

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


MESHES = [(lambda: synth.cap_bowl_mesh(), "quad"),
          (lambda: synth.fbm_dem_mesh(n=30, seed=3, crater_diameter=120.0), "quad"),
          (lambda: synth.fbm_dem_mesh(n=44, seed=5), "quad"),
          (lambda: synth.gaussian_sphere_mesh(level=3, sigma=0.3, seed=4), "oct")]


@pytest.fixture(scope="module")
def meshes():
    return [(mk(), kind) for mk, kind in MESHES]


@pytest.fixture(scope="module")
def probs(vf, meshes):
    return [vf.build_problem(v, f, kind=k, tol=1e-3, precisions=("fp32", "bf16")) for (v, f), k in meshes]


@pytest.fixture(scope="module")
def oracle_F(meshes):
    """Each mesh's dense FP64 F (Eq. FF-def, the oracle's own visibility)."""
    import oracle
    out = []
    for (v, f), _ in meshes:
        om = oracle.mesh(v, f)
        out.append((om, oracle.F_rows(om, np.arange(om.n))))
    return out


@pytest.mark.parametrize("prec,R", [("fp32", 3), ("bf16", 128)])
def test_batched_solve_against_the_oracle(vf, probs, oracle_F, prec, R):
    """One vf_solve_batched over the stack of all meshes against the oracle's
    per-mesh FP64 Jacobi solution of the uncompressed system: within the
    compression error (2 tol) for every mesh and column."""
    import oracle
    import torch
    Es, Bs, dirs = [], [], []
    for k, p in enumerate(probs):
        d = synth.sun_directions(R, 9.0 + 3 * k)
        E = torch.empty((R, p.mesh.n), device="cuda")
        vf.vf_mesh_insolation(p.mesh, d, 1365.0, E)
        Es.append(E)
        Bs.append(torch.empty_like(E))
        dirs.append(d)
    kw = dict(rho=0.12, rtol=1e-7)
    if prec != "fp32":
        kw.update(precision=prec, refine=True)
    stats = vf.vf_solve_batched([p.hmat for p in probs], Es, Bs, **kw)
    for (om, F), B, d, st in zip(oracle_F, Bs, dirs, stats):
        assert st["converged"] == 1
        Bo, _, _ = oracle.jacobi(lambda X: F @ X, oracle.insolation(om, d, 1365.0), 0.12, rtol=1e-12)
        nb = np.linalg.norm(Bo, axis=0)
        live = nb > 0
        assert live.sum() >= R // 2
        err = np.linalg.norm(B.double().cpu().numpy().T - Bo, axis=0)[live] / nb[live]
        assert np.all(err <= 2e-3), (om.n, err.max())


def _rel(a, b):
    return ((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-30)).max().item()


@pytest.mark.parametrize("prec,R", [("fp32", 3), ("bf16", 8), ("bf16", 130)])
def test_stacked_apply_equals_per_mesh(vf, probs, prec, R):
    import torch
    S = vf.vf_hmat_stack([p.hmat for p in probs])
    assert vf.vf_hmat_nsegments(S) == len(probs)
    ns = [p.mesh.n for p in probs]
    assert S.n == sum(ns)
    X = torch.rand((R, S.n), generator=torch.Generator().manual_seed(R)).cuda()
    Y = torch.empty_like(X)
    vf.vf_apply(S, X, Y, precision=prec)
    o = 0
    for p, n in zip(probs, ns):
        Xk = X[:, o:o + n].contiguous()
        Yk = torch.empty_like(Xk)
        vf.vf_apply(p.hmat, Xk, Yk, precision=prec)
        # FP32: the same records in the same order per row tile, equal to
        # rounding.  BF16 on the tensor cores: K chunks start at other
        # columns once the mesh is shifted, so FP32 partial sums of T round
        # differently before T is rounded to BF16 (2^-9); both products are
        # equally close to the exact one.
        bound = 1e-6 if (prec == "fp32" or R < 16) else 1e-4
        assert _rel(Y[:, o:o + n], Yk) <= bound, (p.mesh.n, prec, R)
        o += n


def test_batched_solve_matches_single_solves(vf, probs):
    import torch
    Rs = [3, 5, 1, 2]
    Es, Bs = [], []
    for k, (p, R) in enumerate(zip(probs, Rs)):
        E = torch.empty((R, p.mesh.n), device="cuda")
        vf.vf_mesh_insolation(p.mesh, synth.sun_directions(R, 10.0 + 5 * k), 1365.0, E)
        Es.append(E)
        Bs.append(torch.empty_like(E))
    stats = vf.vf_solve_batched([p.hmat for p in probs], Es, Bs, rho=0.12, rtol=1e-6)
    for p, E, B, st in zip(probs, Es, Bs, stats):
        assert st["converged"] == 1 and st["max_rel_residual"] <= 1e-6
        B1 = torch.empty_like(E)
        vf.vf_solve(p.hmat, E, B1, rho=0.12, rtol=1e-6)
        assert _rel(B, B1) <= 2e-6


def test_batched_convergence_is_per_mesh(vf, probs):
    # one mesh's flux a million times smaller: a criterion over all meshes
    # together would stop before that mesh meets its own tolerance
    import torch
    Es, Bs = [], []
    for k, p in enumerate(probs):
        E = torch.empty((2, p.mesh.n), device="cuda")
        vf.vf_mesh_insolation(p.mesh, synth.sun_directions(2, 12.0), 1365.0, E)
        if k == 1:
            E *= 1e-6
        Es.append(E)
        Bs.append(torch.empty_like(E))
    stats = vf.vf_solve_batched([p.hmat for p in probs], Es, Bs, rho=0.12, rtol=1e-7)
    for p, E, B, st in zip(probs, Es, Bs, stats):
        assert st["converged"] == 1 and st["max_rel_residual"] <= 1e-7
        B1 = torch.empty_like(E)
        vf.vf_solve(p.hmat, E, B1, rho=0.12, rtol=1e-7)
        assert _rel(B, B1) <= 1e-6


def test_batched_tensor_refined_solve(vf, probs):
    import torch
    R = 128
    Es, Bs, Ref = [], [], []
    for k, p in enumerate(probs):
        E = torch.empty((R, p.mesh.n), device="cuda")
        vf.vf_mesh_insolation(p.mesh, synth.sun_directions(R, 8.0 + k), 1365.0, E)
        Es.append(E)
        Bs.append(torch.empty_like(E))
        B32 = torch.empty_like(E)
        vf.vf_solve(p.hmat, E, B32, rho=0.12, rtol=1e-6)
        Ref.append(B32)
    stats = vf.vf_solve_batched([p.hmat for p in probs], Es, Bs, rho=0.12, rtol=1e-6, precision="bf16",
                                refine=True)
    for B, B32, st in zip(Bs, Ref, stats):
        assert st["converged"] == 1
        live = B32.norm(dim=1) > 0
        err = ((B - B32).norm(dim=1)[live] / B32.norm(dim=1)[live]).max().item()
        assert err <= 1e-5, err


def test_stack_cache_follows_handles(vf):
    import torch
    ps = [vf.build_problem(*synth.fbm_dem_mesh(n=24, seed=s), tol=1e-3, precisions=("fp32",)) for s in (1, 2)]
    Es = [torch.rand((2, p.mesh.n), device="cuda") for p in ps]
    Bs = [torch.empty_like(E) for E in Es]
    vf.vf_solve_batched([p.hmat for p in ps], Es, Bs, rho=0.12, rtol=1e-6)
    first = [B.clone() for B in Bs]
    # a new handle for the second mesh: the cached stack of the old pair is not reused
    ps[1] = vf.build_problem(*synth.fbm_dem_mesh(n=24, seed=2), tol=1e-3, precisions=("fp32",))
    vf.vf_solve_batched([p.hmat for p in ps], Es, Bs, rho=0.12, rtol=1e-6)
    for a, b in zip(first, Bs):
        assert _rel(b, a) <= 1e-6


def test_autotune_records_a_valid_choice(vf, probs):
    import torch
    h, n = probs[2].hmat, probs[2].mesh.n
    X = torch.rand((40, n), generator=torch.Generator().manual_seed(7)).cuda()
    Y32 = torch.empty_like(X)
    vf.vf_apply(h, X, Y32, precision="fp32")
    t = vf.vf_autotune(h, "bf16", 40)
    assert t["rb"] in (1, 2, 4, 8) and t["tensor"] in (0, 1) and t["rhs_block"] == 0 and t["us_per_rhs"] > 0
    Y = torch.empty_like(X)
    vf.vf_apply(h, X, Y, precision="bf16")
    assert _rel(Y, Y32) <= 4e-3
    t = vf.vf_autotune(h, "fp32", 5)
    assert t["rb"] in (1, 2, 4) and t["tensor"] == 0
    X5 = X[:5].contiguous()
    Y5 = torch.empty_like(X5)
    vf.vf_apply(h, X5, Y5, precision="fp32")
    assert _rel(Y5, Y32[:5]) <= 1e-6


def test_rhs_blocks_solve_like_one_block(vf):
    import torch
    p = vf.build_problem(*synth.fbm_dem_mesh(n=36, seed=9), tol=1e-3, precisions=("fp32",))
    R = 200
    E = torch.empty((R, p.mesh.n), device="cuda")
    vf.vf_mesh_insolation(p.mesh, synth.sun_directions(R, 9.0), 1365.0, E)
    B1, B2 = torch.empty_like(E), torch.empty_like(E)
    vf.vf_solve(p.hmat, E, B1, rho=0.12, rtol=1e-8)
    vf.vf_tune_set(p.hmat, "fp32", R, rb=8, rhs_block=64)
    st = vf.vf_solve(p.hmat, E, B2, rho=0.12, rtol=1e-8)
    assert st["converged"] == 1
    assert _rel(B2, B1) <= 1e-6
    with pytest.raises(vf.VFError):
        vf.vf_tune_set(p.hmat, "fp32", R, rb=3)
