"""Parity at the full size of the terrain workload (79,202 facets, the
bench's mesh and tolerance), on outputs the oracle computes row by row: the
FP32 multiply in the bench's single-RHS launch configuration and at R = 4,
the BF16 tensor-core multiply of 128 columns, and the refined BF16 solve of
128 suns through the equation it solves."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module")
def vf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf as _vf
    return _vf


@pytest.fixture(scope="module")
def full(vf):
    v, f = synth.fbm_dem_mesh(n=200, spacing=10.0, hurst=0.8, seed=1, rms_slope_deg=15.0, crater_diameter=1000.0)
    prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=TOL, precisions=("fp32", "bf16"))
    om = oracle.mesh(v, f)
    assert om.n == prob.mesh.n == 79202
    rows = np.sort(np.random.default_rng(11).choice(om.n, 128, replace=False))
    Fr = oracle.F_rows(om, rows)  # (128, n), FP64, the oracle's own visibility
    return dict(prob=prob, om=om, rows=rows, Fr=Fr)


def _sampled_err(got_rows, ref_rows):
    """Per column: || got - ref || / || ref || over the sampled rows (columns with ref = 0 skipped)."""
    nr = np.linalg.norm(ref_rows, axis=0)
    live = nr > 0
    return (np.linalg.norm(got_rows - ref_rows, axis=0)[live] / nr[live]), int(live.sum())


@pytest.mark.parametrize("R", [1, 4])
def test_fp32_multiply_sampled_rows(vf, full, R):
    import torch
    om, rows, Fr = full["om"], full["rows"], full["Fr"]
    E = oracle.insolation(om, synth.sun_directions(R, 10.0), 1365.0)  # (n, R)
    X = torch.tensor(np.ascontiguousarray(E.T), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    vf.vf_apply(full["prob"].hmat, X, Y, precision="fp32")
    got = Y.double().cpu().numpy().T[rows]
    err, live = _sampled_err(got, Fr @ E)
    assert live == R
    assert np.all(err <= 2 * TOL), err


def test_bf16_tensor_multiply_sampled_rows(vf, full):
    import torch
    om, rows, Fr = full["om"], full["rows"], full["Fr"]
    E = oracle.insolation(om, synth.sun_directions(128, 10.0), 1365.0)
    X = torch.tensor(np.ascontiguousarray(E.T), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    vf.vf_apply(full["prob"].hmat, X, Y, precision="bf16")
    got = Y.double().cpu().numpy().T[rows]
    err, live = _sampled_err(got, Fr @ E)
    assert live > 100
    # compression (2 tol) plus BF16 factors and right-hand sides (4e-3 against FP32)
    assert np.all(err <= 2 * TOL + 4e-3), err.max()


def test_refined_bf16_solve_satisfies_the_system_on_sampled_rows(vf, full):
    # B from BF16 tensor-core sweeps with split-BF16 refinement solves
    # (I - rho F_hat) B = E to rtol; with the oracle's exact F rows the
    # residual E - B + rho F B on the sampled rows is then rho (F - F_hat) B,
    # bounded by rho x 2 tol of F B
    import torch
    prob, rows, Fr = full["prob"], full["rows"], full["Fr"]
    rho = 0.12
    E = torch.empty((128, prob.mesh.n), device="cuda")
    vf.vf_mesh_insolation(prob.mesh, synth.sun_directions(128, 10.0), 1365.0, E)
    B = torch.empty_like(E)
    st = vf.vf_solve(prob.hmat, E, B, rho=rho, rtol=1e-6, precision="bf16", refine=True)
    assert st["converged"] == 1
    Bd = B.double().cpu().numpy().T  # (n, 128)
    Ed = E.double().cpu().numpy().T
    FB = Fr @ Bd
    r = Ed[rows] - Bd[rows] + rho * FB
    nfb = np.linalg.norm(FB, axis=0)
    live = nfb > 0
    assert live.sum() > 100
    rel = np.linalg.norm(r, axis=0)[live] / (rho * nfb[live])
    assert np.all(rel <= 2 * TOL + 1e-4), rel.max()
