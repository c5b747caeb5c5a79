"""The FP64 truncation check of assembly (Algorithm 3's criterion
sigma_{q+1} < tol sigma_1, checked on the accepted factors in FP64 on the
GPU): with it on, every SVD block of the assembled matrix meets the
criterion against the oracle's dense FP64 F, and when no block fails the
check the matrix is the one assembled without it."""
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


def _dense(vf, h, n):
    import torch
    I = torch.eye(n, device="cuda", dtype=torch.float32)
    Y = torch.empty_like(I)
    vf.vf_apply(h, I, Y)
    return Y.double().cpu().numpy().T


CASES = {
    "cap_1e-2": (lambda: synth.cap_bowl_mesh(), 1e-2),
    "dem30_1e-3": (lambda: synth.fbm_dem_mesh(n=30, seed=3, crater_diameter=120.0), 1e-3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_verified_svd_blocks_meet_the_criterion(vf, name):
    mk, tol = CASES[name]
    v, f = mk()
    om = oracle.mesh(v, f)
    F = oracle.F_dense(om)
    m = vf.vf_mesh_create(v, f)
    t = vf.vf_partition(m, "quad", 64)
    nodes = vf.vf_tree_nodes(t)
    perm = vf.vf_tree_perm(t).astype(np.int64)
    Ft = F[np.ix_(perm, perm)]
    # no power iterations: the weakest probe, so the check has the most to catch
    h, st = vf.vf_assemble(m, t, tol=tol, power_iters=0, verify=True, precisions=("fp32",))
    assert st["verify_failed"] >= 0
    Fh = _dense(vf, h, om.n)[np.ix_(perm, perm)]
    nsvd = 0
    for d in vf.vf_hmat_blocks(h):
        if d[2] != 3:
            continue
        nsvd += 1
        r0, mm = nodes["first"][d[0]], nodes["count"][d[0]]
        c0, nn = nodes["first"][d[1]], nodes["count"][d[1]]
        A = Ft[r0:r0 + mm, c0:c0 + nn]
        err = np.linalg.norm(Fh[r0:r0 + mm, c0:c0 + nn] - A, 2)
        # the check accepts only below 0.9 tol of its power-iteration
        # estimates (which approach the norms from below): no slack here
        assert err <= tol * np.linalg.norm(A, 2), (tuple(d[:2]), err / np.linalg.norm(A, 2))
    assert nsvd > 0


def test_check_keeps_passing_blocks(vf):
    import torch
    v, f = synth.fbm_dem_mesh(n=40, seed=8)
    m = vf.vf_mesh_create(v, f)
    t = vf.vf_partition(m, "quad", 64)
    h0, s0 = vf.vf_assemble(m, t, tol=1e-3, verify=False, precisions=("fp32",))
    h1, s1 = vf.vf_assemble(m, t, tol=1e-3, verify=True, precisions=("fp32",))
    assert s0["verify_failed"] == 0
    X = torch.rand((4, m.n), generator=torch.Generator().manual_seed(1)).cuda()
    Y0, Y1 = torch.empty_like(X), torch.empty_like(X)
    vf.vf_apply(h0, X, Y0)
    vf.vf_apply(h1, X, Y1)
    if s1["verify_failed"] == 0:
        assert torch.equal(Y0, Y1)
        assert np.array_equal(vf.vf_hmat_blocks(h0), vf.vf_hmat_blocks(h1))
    else:
        # failed blocks were re-probed at a higher rank or stored another way
        assert s1["probes"] > s0["probes"] or s1["nblocks"] != s0["nblocks"]
