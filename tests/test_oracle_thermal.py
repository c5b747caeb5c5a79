"""Pins of the oracle's time-stepping (Algorithm 6, Section 5.2) and
finite-disk sun (Section 2) against closed forms and hand values."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_flux_init_and_one_step_by_hand():
    # two facets, F = [[0, a], [b, 0]] (hand-checkable), albedo and emissivity per facet
    a, b = 0.3, 0.2
    F = np.array([[0.0, a], [b, 0.0]])
    alb = np.array([[0.1], [0.4]])
    eps = np.array([[0.9], [0.8]])
    E0 = np.array([[100.0], [50.0]])
    Qrefl, Qir, Qabs, Qrad = oracle.flux_init(E0, alb, H=2.0)
    assert np.allclose(Qabs, [[92.0], [32.0]]) and np.allclose(Qrad, Qabs)
    assert not Qrefl.any() and not Qir.any()
    E1 = np.array([[80.0], [60.0]])
    r1, i1, q1 = oracle.flux_step(lambda X: F @ X, E1, Qrefl, Qir, Qrad, alb, eps)
    # Q_refl' = F (alb * E1) = [a * 0.4 * 60, b * 0.1 * 80]
    assert np.allclose(r1, [[0.3 * 24.0], [0.2 * 8.0]])
    # Q_IR' = F Q_rad (Q_IR = 0) = [a * 32, b * 92]
    assert np.allclose(i1, [[9.6], [18.4]])
    assert np.allclose(q1, [[0.9 * (80 + 7.2) + 0.9 * 9.6], [0.6 * (60 + 1.6) + 0.8 * 18.4]])


def test_flux_steps_with_instantaneous_equilibrium_reach_section_5_1(cap_small):
    """With Q_rad = Q_abs (no subsurface storage) and a fixed sun, the
    Algorithm 6 updates converge to the two time-independent systems of
    Section 5.1: Q_refl = Q_vis - Q_direct, Q_IR, and eps sigma T^4 = Q_abs."""
    m = cap_small
    F = oracle.F_dense(m, oracle.visibility_rows(m, np.arange(m.n)))
    E = oracle.insolation(m, synth.sun_directions(2, 10.0), 1365.0)
    alb, eps = 0.12, 0.95
    T, Qvis, Qir = oracle.equilibrium_temperature(lambda X: F @ X, E, alb, eps)
    Qrefl, Qi, Qabs, Qrad = oracle.flux_init(E, alb)
    for _ in range(400):
        Qrefl, Qi, Qabs = oracle.flux_step(lambda X: F @ X, E, Qrefl, Qi, Qrad, alb, eps)
        Qrad = Qabs
    assert np.allclose(Qrefl, Qvis - E, rtol=1e-9, atol=1e-9 * E.max())
    assert np.allclose(Qi, Qir, rtol=1e-9, atol=1e-9 * E.max())
    T6 = (np.maximum(Qabs, 0) / (eps * oracle.SIGMA_SB)) ** 0.25
    assert np.allclose(T6, T, rtol=1e-9)


def test_disk_weights_and_mean_direction():
    s = np.array([0.3, -0.2, 0.8])
    s /= np.linalg.norm(s)
    th = math.radians(0.267)  # the Sun's angular radius at 1 AU
    for rings in (1, 3, 8):
        d, w = oracle.disk_sun_samples(s, th, rings)
        assert d.shape[0] == 1 + 3 * rings * (rings - 1)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
        mean = w @ d
        # symmetric sectors: the mean points along s
        assert np.linalg.norm(np.cross(mean, s)) < 1e-12
        ang = np.arccos(np.clip(d @ s, -1, 1))
        assert ang.max() <= th * (1 + 1e-12)


def test_disk_mean_cosine_converges_to_the_uniform_disk():
    # mean of cos(t) over a uniform disk of angular radius th (planar radial
    # measure 2 r dr, t = th r): 2 [(cos th - 1) / th^2 + sin th / th]
    s = np.array([0.0, 0.0, 1.0])
    th = 0.2
    exact = 2.0 * ((math.cos(th) - 1.0) / th ** 2 + math.sin(th) / th)
    errs = []
    for rings in (2, 4, 8, 16):
        d, w = oracle.disk_sun_samples(s, th, rings)
        errs.append(abs(w @ (d @ s) - exact))
    # second order in the ring width: each halving cuts the error about 4x
    assert errs[-1] < 1e-5
    assert all(3.0 < e0 / e1 < 8.0 for e0, e1 in zip(errs, errs[1:]))


def test_disk_insolation_lit_plane_and_point_limit(cap_small):
    m = cap_small
    dirs = synth.sun_directions(3, 30.0)
    th = math.radians(0.267)
    Ed = oracle.insolation_disk(m, dirs, 1365.0, th, 4)
    Ep = oracle.insolation(m, dirs, 1365.0)
    for r, s in enumerate(dirs):
        d, w = oracle.disk_sun_samples(s, th, 4)
        lit_all = np.all(oracle.insolation(m, d, 1.0) > 0, axis=1)
        # a facet every point source lights gets S n . (sum w_k s_k) exactly
        assert np.allclose(Ed[lit_all, r], 1365.0 * m.nrm[lit_all] @ (w @ d), rtol=1e-12)
        # fully dark facets stay dark, and the disk stays within [0, max point flux]
        dark = np.all(oracle.insolation(m, d, 1.0) == 0, axis=1)
        assert np.all(Ed[dark, r] == 0)
    assert np.all(Ed >= 0) and Ed.max() <= 1365.0
    # a vanishing disk is the point sun
    E0 = oracle.insolation_disk(m, dirs, 1365.0, 1e-9, 3)
    assert np.allclose(E0, Ep, rtol=1e-6, atol=1e-6)


def test_equilibrium_fluxes_solve_the_printed_systems(cap_small):
    """Per-facet albedo, emissivity and heat flux: the outputs satisfy
    Eqs. time-indep-system-1/2 and 3d-equilbr to rounding; with uniform
    values they equal equilibrium_temperature (B = Q_direct + Q_refl)."""
    m = cap_small
    F = oracle.F_dense(m, oracle.visibility_rows(m, np.arange(m.n)))
    E = oracle.insolation(m, synth.sun_directions(2, 10.0), 1365.0)
    rng = np.random.default_rng(5)
    alb = rng.uniform(0.05, 0.3, size=(m.n, 1))
    eps = rng.uniform(0.9, 1.0, size=(m.n, 1))
    H = rng.uniform(0.0, 0.05, size=(m.n, 1))
    T, Qr, Qi = oracle.equilibrium_fluxes(lambda X: F @ X, E, alb, eps, H)
    sc = np.abs(F @ (alb * E)).max()
    assert np.abs(Qr - F @ (alb * Qr) - F @ (alb * E)).max() <= 1e-11 * sc
    r2 = Qi - F @ Qi - F @ ((1 - alb) * (E + Qr)) - F @ np.broadcast_to(H, E.shape)
    assert np.abs(r2).max() <= 1e-11 * np.abs(Qi).max()
    assert np.allclose(eps * oracle.SIGMA_SB * T ** 4, (1 - alb) * (E + Qr) + eps * Qi, rtol=1e-12)
    T0, Qvis0, Qir0 = oracle.equilibrium_temperature(lambda X: F @ X, E, 0.12, 0.95)
    T1, Qr1, Qi1 = oracle.equilibrium_fluxes(lambda X: F @ X, E, 0.12, 0.95)
    assert np.allclose(Qr1, Qvis0 - E, rtol=1e-9, atol=1e-9 * E.max())
    assert np.allclose(Qi1, Qir0, rtol=1e-9, atol=1e-9 * E.max())
    assert np.allclose(T1, T0, rtol=1e-10)
