"""The rank predictor's own kernels against the FP64 oracle, its training,
and what it gains inside assembly (GPU)."""
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


def _random_model(vf, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, scale, vf.VF_PRED_NPARAM).astype(np.float32)
    mu = rng.normal(0.0, 1.0, vf.VF_PRED_NFEAT).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, vf.VF_PRED_NFEAT).astype(np.float32)
    return np.concatenate([w, mu, sd])


def test_gradient_matches_oracle_backprop(vf):
    from oracle import mlp
    theta = _random_model(vf, 0)
    p = vf.vf_predictor_create(seed=1)
    got = vf.vf_predictor_params(p, set_to=theta)
    assert np.array_equal(got, theta)
    rng = np.random.default_rng(5)
    F = rng.normal(0.0, 1.5, (300, vf.VF_PRED_NFEAT)).astype(np.float32)
    y = rng.integers(0, vf.VF_PRED_NCLASS, 300).astype(np.int32)
    L, g = vf.vf_predictor_grad(p, F, y)
    # the oracle at the same FP16-rounded weights, in FP64
    Lr, gr = mlp.backward(mlp.unpack(theta, round_fp16=True), F, y)
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    rel = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert rel <= 1e-3, rel
    # per block of parameters too (a wrong layer cannot hide in the total)
    o = 0
    for name, shape in mlp.SIZES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], gr[o:o + k]
        assert np.linalg.norm(a - b) <= 1e-3 * max(np.linalg.norm(b), 1e-8), name
        o += k


def test_training_lowers_the_loss_and_is_reproducible(vf):
    rng = np.random.default_rng(7)
    n = 4096
    F = rng.normal(0.0, 1.0, (n, vf.VF_PRED_NFEAT)).astype(np.float32) * 3 + 1
    # labels from a fixed rule of two features (learnable)
    y = (np.clip(np.floor((F[:, 0] - 1) / 3 + 3), 0, 5)).astype(np.int32)
    y[F[:, 4] > 4] = 5
    p1 = vf.vf_predictor_create(seed=11)
    L0, _ = vf.vf_predictor_grad(p1, F, y)
    L1 = vf.vf_predictor_train(p1, F, y, epochs=15, batch=256, lr=3e-3)
    assert L1 < 0.5 * L0, (L0, L1)
    p2 = vf.vf_predictor_create(seed=11)
    vf.vf_predictor_train(p2, F, y, epochs=15, batch=256, lr=3e-3)
    assert np.array_equal(vf.vf_predictor_params(p1), vf.vf_predictor_params(p2))
    cls, prob = vf.vf_predictor_predict(p1, F)
    assert np.mean(cls == y) > 0.8
    assert np.allclose(prob.sum(axis=1), 1.0, atol=1e-5)


def test_prediction_matches_oracle_argmax(vf):
    from oracle import mlp
    theta = _random_model(vf, 3, scale=0.5)
    p = vf.vf_predictor_create()
    vf.vf_predictor_params(p, set_to=theta)
    rng = np.random.default_rng(9)
    F = rng.normal(0.0, 2.0, (500, vf.VF_PRED_NFEAT)).astype(np.float32)
    cls, prob = vf.vf_predictor_predict(p, F)
    pr = mlp.forward(mlp.unpack(theta, round_fp16=True), F)["p"]
    assert np.max(np.abs(prob - pr)) < 1e-5
    top2 = np.sort(pr, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 1e-4
    assert np.array_equal(cls[clear], np.argmax(pr, axis=1)[clear])


def _problem(vf, v, f, kind="quad", predictor=None):
    return vf.build_problem(v, f, kind=kind, leaf_size=64, tol=1e-3, precisions=("fp32",), predictor=predictor)


def test_predictor_in_assembly_keeps_tolerance_and_saves_probes(vf):
    import torch

    import oracle
    import synth
    # training data: the probe logs of plain assemblies of other meshes
    Xs, ys = [], []
    for side, seed in ((40, 21), (56, 22), (64, 23)):
        v, f = synth.fbm_dem_mesh(n=side, seed=seed)
        X, y = vf.vf_hmat_probe_log(_problem(vf, v, f).hmat)
        Xs.append(X)
        ys.append(y)
    v, f = synth.cap_bowl_mesh()
    X, y = vf.vf_hmat_probe_log(_problem(vf, v, f).hmat)
    Xs.append(X)
    ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    assert len(y) > 500 and len(np.unique(y)) >= 3
    p = vf.vf_predictor_create(seed=4)
    vf.vf_predictor_train(p, X, y, epochs=40, batch=256, lr=3e-3)
    # a fresh mesh: plain path vs predictor path
    v, f = synth.fbm_dem_mesh(n=60, seed=31)
    plain = _problem(vf, v, f)
    pred = _problem(vf, v, f, predictor=p)
    sp, sq = plain.stats, pred.stats
    assert sq["probes"] < sp["probes"], (sp["probes"], sq["probes"])
    bp = vf.vf_hmat_bytes(plain.hmat, "fp32")
    bq = vf.vf_hmat_bytes(pred.hmat, "fp32")
    assert bq <= 1.10 * bp, (bp, bq)
    # both matrices meet the tolerance against the oracle's dense FP64 F on sampled rows
    om = oracle.mesh(v, f)
    rows = np.sort(np.random.default_rng(0).choice(om.n, 512, replace=False))
    Fr = oracle.F_rows(om, rows)
    E = oracle.insolation(om, synth.sun_directions(3, 10.0), 1365.0)  # (n, 3)
    ref = Fr @ E
    X = torch.tensor(np.ascontiguousarray(E.T), dtype=torch.float32, device="cuda")
    out = []
    for prob in (plain, pred):
        Y = torch.empty_like(X)
        vf.vf_apply(prob.hmat, X, Y)
        out.append(Y.cpu().numpy().T.astype(np.float64))
        got = out[-1][rows]
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.all(err <= 2e-3), err
    # the two compressed matrices each meet tol, so their products differ by <= 2 tol
    d = np.linalg.norm(out[1] - out[0], axis=0) / np.linalg.norm(out[0], axis=0)
    assert np.all(d <= 2e-3), d
