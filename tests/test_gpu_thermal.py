"""The thermal layer on the GPU against the oracle: Section 5.1 equilibrium
temperatures (vf_equilibrium), the Algorithm 6 flux updates (vf_flux_step)
and the finite solar disk (vf_mesh_insolation_disk), on the 1,196-facet
spherical-cap bowl with the oracle's dense FP64 F, and the analytic
shadowed-bowl temperature of Section 6.1."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-3
ALB, EPS = 0.12, 0.95


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
def bowl(vf, cap_full, cap_full_F):
    v, f = synth.cap_bowl_mesh()
    prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=TOL, precisions=("fp32", "bf16"))
    return prob, cap_full, cap_full_F[0]


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float32, device="cuda")


def _host(t):
    return t.double().cpu().numpy().T


def _rel(got, ref):
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


def test_equilibrium_matches_the_oracle_and_the_bowl(vf, bowl):
    import torch
    prob, om, F = bowl
    dirs = synth.sun_directions(4, 10.0)
    Eo = oracle.insolation(om, dirs, 1365.0)
    E = _dev(Eo)
    T = torch.empty_like(E)
    Qvis = torch.empty_like(E)
    Qir = torch.empty_like(E)
    st = vf.vf_equilibrium(prob.hmat, E, T, albedo=ALB, emissivity=EPS, Qvis=Qvis, Qir=Qir, rtol=1e-7)
    assert st[0]["converged"] == 1 and st[1]["converged"] == 1
    To, Qvo, Qio = oracle.equilibrium_temperature(lambda X: F @ X, Eo, ALB, EPS)
    assert _rel(_host(Qvis), Qvo).max() <= 2 * TOL
    assert _rel(_host(Qir), Qio).max() <= 3 * TOL
    Tg = _host(T)
    assert _rel(Tg, To).max() <= TOL
    # Section 6.1: the analytic temperature of the bowl's shadowed part
    T_exact = oracle.bowl_shadow_temperature(1365.0, 10.0, ALB, EPS, 0.2)
    sh = Eo[:, 0] == 0
    assert sh.sum() > 50
    assert np.abs(Tg[sh, 0] - T_exact).max() / T_exact < 0.02


def test_equilibrium_per_facet_albedo_emissivity_heat_flux(vf, bowl):
    import torch
    prob, om, F = bowl
    rng = np.random.default_rng(9)
    alb = rng.uniform(0.05, 0.3, size=om.n)
    eps = rng.uniform(0.9, 1.0, size=om.n)
    H = rng.uniform(0.0, 0.05, size=om.n)
    Eo = oracle.insolation(om, synth.sun_directions(2, 25.0), 1365.0)
    E = _dev(Eo)
    T = torch.empty_like(E)
    Qvis = torch.empty_like(E)
    Qir = torch.empty_like(E)
    tv = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    vf.vf_equilibrium(prob.hmat, E, T, albedo=tv(alb), emissivity=tv(eps), H=tv(H), Qvis=Qvis, Qir=Qir, rtol=1e-7)
    To, Qro, Qio = oracle.equilibrium_fluxes(lambda X: F @ X, Eo, alb[:, None], eps[:, None], H[:, None])
    assert _rel(_host(Qvis), Eo + Qro).max() <= 2 * TOL
    assert _rel(_host(Qir), Qio).max() <= 3 * TOL
    assert _rel(_host(T), To).max() <= TOL


@pytest.mark.parametrize("R,precision,tol", [(2, "fp32", 2 * TOL), (8, "bf16", 2 * TOL + 4e-3)])
def test_flux_step_matches_the_oracle(vf, bowl, R, precision, tol):
    import torch
    prob, om, F = bowl
    apply = lambda X: F @ X
    E0 = oracle.insolation(om, synth.sun_directions(R, 12.0), 1365.0)
    E1 = oracle.insolation(om, synth.sun_directions(R, 12.5), 1365.0)
    Qr, Qi, Qa, Qd = oracle.flux_init(E0, ALB)
    Qr, Qi, Qa = oracle.flux_step(apply, E0, Qr, Qi, Qd, ALB, EPS)  # a state with every flux nonzero
    Qd = Qa
    ref = oracle.flux_step(apply, E1, Qr, Qi, Qd, ALB, EPS)
    gQr, gQi, gQd = _dev(Qr), _dev(Qi), _dev(Qd)
    gQa = torch.empty_like(gQr)
    vf.vf_flux_step(prob.hmat, _dev(E1), gQr, gQi, gQd, gQa, albedo=ALB, emissivity=EPS, precision=precision)
    for got, want in zip((gQr, gQi, gQa), ref):
        assert _rel(_host(got), want).max() <= tol


def test_flux_steps_with_instantaneous_equilibrium_converge(vf, bowl):
    """Algorithm 6 with Q_rad = Q_abs and a fixed sun reaches the Section 5.1
    equilibrium (the same one vf_equilibrium and the oracle compute)."""
    import torch
    prob, om, F = bowl
    Eo = oracle.insolation(om, synth.sun_directions(2, 10.0), 1365.0)
    E = _dev(Eo)
    Qr = torch.zeros_like(E)
    Qi = torch.zeros_like(E)
    Qa = (1 - ALB) * E
    Qd = Qa.clone()
    for _ in range(120):
        vf.vf_flux_step(prob.hmat, E, Qr, Qi, Qd, Qa, albedo=ALB, emissivity=EPS)
        Qd.copy_(Qa)
    T6 = ((torch.clamp(Qa.double(), min=0) / (EPS * oracle.SIGMA_SB)) ** 0.25).cpu().numpy().T
    To, _, _ = oracle.equilibrium_temperature(lambda X: F @ X, Eo, ALB, EPS)
    assert _rel(T6, To).max() <= TOL


def test_disk_insolation_matches_the_oracle(vf, bowl):
    import torch
    prob, om, _ = bowl
    dirs = synth.sun_directions(3, 10.0)
    for radius, rings in ((math.radians(0.267), 3), (0.05, 5)):
        Eo = oracle.insolation_disk(om, dirs, 1365.0, radius, rings)
        E = torch.empty((3, om.n), device="cuda")
        vf.vf_mesh_insolation_disk(prob.mesh, dirs, 1365.0, radius, rings, E)
        Eg = _host(E)
        assert np.array_equal(Eg > 0, Eo > 0)
        assert np.abs(Eg - Eo).max() <= 1e-6 * Eo.max()
        if radius > 0.01:  # a wide disk: partly lit facets along the shadow's edge
            part = (Eo > 0) & (Eo < 0.98 * 1365.0 * np.maximum(om.nrm @ dirs.T, 0))
            assert part.sum() > 10
