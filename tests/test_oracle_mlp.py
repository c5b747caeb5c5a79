"""Pins of the oracle's rank-predictor network (FP64, CPU): the backward pass
against central finite differences, closed forms at special weights, and
softmax's shift invariance."""
import numpy as np

from oracle import mlp


def _case(seed=0, n=37, scale=0.5):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, scale, mlp.NPARAM)
    F = rng.normal(0.0, 1.0, (n, mlp.NF))
    y = rng.integers(0, mlp.NC, n)
    return mlp.with_flat(mlp.unpack(np.zeros(mlp.NPARAM)), w), F, y


def test_backward_matches_central_differences():
    P, F, y = _case()
    L, g = mlp.backward(P, F, y)
    w = mlp.flat(P)
    rng = np.random.default_rng(1)
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(mlp.with_flat(P, wp), F, y) - mlp.loss(mlp.with_flat(P, wm), F, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert np.isclose(L, mlp.loss(P, F, y), rtol=0, atol=1e-15)


def test_zero_weights_closed_form():
    # all weights zero: every class has probability 1/6, the loss is ln 6, the
    # hidden layers are zero so only the output bias has a gradient,
    # d loss / d b3_c = 1/6 - (fraction of labels equal to c)
    P = mlp.unpack(np.zeros(mlp.NPARAM))
    rng = np.random.default_rng(2)
    F = rng.normal(size=(60, mlp.NF))
    y = rng.integers(0, mlp.NC, 60)
    L, g = mlp.backward(P, F, y)
    assert abs(L - np.log(6.0)) < 1e-15
    frac = np.bincount(y, minlength=mlp.NC) / len(y)
    assert np.allclose(g[-mlp.NC:], 1.0 / 6.0 - frac, rtol=0, atol=1e-15)
    assert np.all(g[:-mlp.NC] == 0.0)


def test_softmax_shift_invariance_and_probabilities():
    P, F, y = _case(seed=3)
    v = mlp.forward(P, F)
    assert np.allclose(v["p"].sum(axis=1), 1.0, atol=1e-14)
    Q = dict(P)
    Q["b3"] = P["b3"] + 3.25  # the same constant on every class
    assert abs(mlp.loss(P, F, y) - mlp.loss(Q, F, y)) < 1e-12
    # the output-bias gradient sums to zero over classes (probabilities sum to 1)
    _, g = mlp.backward(P, F, y)
    assert abs(g[-mlp.NC:].sum()) < 1e-14


def test_standardisation_and_fp16_rounding():
    rng = np.random.default_rng(4)
    w = rng.normal(0.0, 0.3, mlp.NPARAM).astype(np.float32)
    mu = rng.normal(size=mlp.NF).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, mlp.NF).astype(np.float32)
    theta = np.concatenate([w, mu, sd])
    P = mlp.unpack(theta, round_fp16=True)
    # rounded weights are exactly representable in FP16 and within half an FP16 ulp
    assert np.all(P["W2"].astype(np.float16).astype(np.float64) == P["W2"])
    assert np.max(np.abs(P["W2"].ravel() - w[mlp.NF * 64 + 64:mlp.NF * 64 + 64 + 64 * 64])) <= 2.0 ** -11 * 2.0
    F = rng.normal(size=(5, mlp.NF))
    # standardising the features is the same as feeding (F - mu) / sd with mu = 0, sd = 1
    P0 = dict(P)
    P0["mu"], P0["sd"] = np.zeros(mlp.NF), np.ones(mlp.NF)
    assert np.allclose(mlp.forward(P, F)["p"], mlp.forward(P0, (F - mu) / sd)["p"], rtol=0, atol=1e-14)
