"""Failure paths, made on the host or by a short bound on a device wait (no
GPU fault is ever provoked):

* a bounded page wait of the CUDA-core multiply that runs out
  (vf_set_wait_limit(0)) makes vf_solve and vf_apply_tree_static return
  VF_E_TIMEOUT, the kernels exit normally and the next call, with the
  default bound, gives the same result as before;
* every device allocation of a whole pipeline (mesh, partition, assembly,
  FP32 solve, BF16 tensor-core solve with refinement, host-buffer solve)
  is made to fail in turn (vf_debug_fail_alloc): each call returns
  VF_E_NOMEM, and a fresh pipeline afterwards gives the same result.
"""
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
    yield _vf
    _vf.vf_set_wait_limit(-1)
    _vf.vf_debug_fail_alloc(0)


@pytest.fixture(scope="module")
def bowl():
    return synth.cap_bowl_mesh(n_rim=30, n_interior=140, seed=0)


def test_wait_limit_reports_timeout_and_recovers(vf):
    import torch
    v, f = synth.fbm_dem_mesh(n=40, seed=3)
    prob = vf.build_problem(v, f, tol=1e-3)
    n = prob.mesh.n
    E = torch.empty((2, n), device="cuda")
    vf.vf_mesh_insolation(prob.mesh, synth.sun_directions(2, 20.0), 1365.0, E)
    B0 = torch.empty_like(E)
    st = vf.vf_solve(prob.hmat, E, B0, rtol=1e-6)
    assert st["converged"] == 1
    Xt = torch.rand((2, n), device="cuda")
    Y0 = torch.empty_like(Xt)
    vf.vf_apply_tree_static(prob.hmat, Xt, Y0)
    try:
        vf.vf_set_wait_limit(0)  # every page wait gives up at once
        B1 = torch.empty_like(E)
        with pytest.raises(vf.VFError) as ei:
            vf.vf_solve(prob.hmat, E, B1, rtol=1e-6)
        assert ei.value.status == vf.VF_E_TIMEOUT
        Y1 = torch.empty_like(Xt)
        with pytest.raises(vf.VFError) as ei:
            vf.vf_apply_tree_static(prob.hmat, Xt, Y1)
        assert ei.value.status == vf.VF_E_TIMEOUT
    finally:
        vf.vf_set_wait_limit(-1)
    torch.cuda.synchronize()  # the context is intact: no sticky error
    B2 = torch.empty_like(E)
    st = vf.vf_solve(prob.hmat, E, B2, rtol=1e-6)
    assert st["converged"] == 1 and torch.equal(B2, B0)
    Y2 = torch.empty_like(Xt)
    vf.vf_apply_tree_static(prob.hmat, Xt, Y2)
    assert torch.equal(Y2, Y0)


def _pipeline(vf, v, f):
    """Everything from mesh to solves; returns the host results."""
    import torch
    prob = vf.build_problem(v, f, tol=1e-3, precisions=("fp32", "bf16"))
    n = prob.mesh.n
    E = torch.empty((16, n), device="cuda")
    vf.vf_mesh_insolation(prob.mesh, synth.sun_directions(16, 10.0), 1365.0, E)
    B = torch.empty_like(E)
    vf.vf_solve(prob.hmat, E[:1], B[:1], rtol=1e-6)
    vf.vf_solve(prob.hmat, E, B, rtol=1e-6, precision="bf16", refine=True)  # tensor cores, split residual
    Eh = E[:2].cpu().contiguous().numpy()
    Bh = np.empty_like(Eh)
    vf.vf_solve_host(prob.hmat, Eh, Bh, rtol=1e-6)
    torch.cuda.synchronize()
    return B.cpu().numpy(), Bh


def test_every_allocation_failure_is_reported(vf, bowl):
    v, f = bowl
    ref = _pipeline(vf, v, f)
    failed_at = []
    for k in range(1, 2000):
        vf.vf_debug_fail_alloc(k)
        try:
            _pipeline(vf, v, f)
            done = True
        except vf.VFError as e:
            assert e.status == vf.VF_E_NOMEM, (k, str(e))
            failed_at.append(k)
            done = False
        finally:
            vf.vf_debug_fail_alloc(0)
        if done:
            break
    assert done, "the pipeline never completed"
    # every allocation before the completing run failed as armed
    assert failed_at == list(range(1, k)), failed_at[:10]
    assert len(failed_at) >= 30
    again = _pipeline(vf, v, f)
    for a, b in zip(ref, again):
        assert np.array_equal(a, b)
