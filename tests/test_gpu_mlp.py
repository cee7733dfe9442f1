"""The learned tuner's MLP kernels (FP32, CUDA) against the FP64 oracle:
forward logits, loss and every gradient entry, the Adam update, training,
model files, and the MLP-driven choice through the C ABI."""
import os

import numpy as np
import pytest

import oracle
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu
DIMS = (8, 64, 64, (5, 4, 5, 6))


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _setup(xb, dev, seed=0, B=37):
    import torch
    model = xb.Mlp(seed=seed)
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(model.param_count()) * 0.3).astype(np.float32)
    model.set_params(P)
    X = rng.standard_normal((B, 8)).astype(np.float32)
    lab = np.stack([rng.integers(0, k, B) for k in DIMS[3]], axis=1).astype(np.int32)
    return model, P, X, lab, torch.tensor(X, device=dev), torch.tensor(lab, device=dev)


def test_forward_matches_oracle(env):
    xb, dev = env
    model, P, X, lab, Xt, _ = _setup(xb, dev)
    got = model.forward(Xt).cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(P.astype(np.float64), DIMS, X.astype(np.float64))
    assert np.max(np.abs(got - ref)) <= 1e-5 * (1 + np.max(np.abs(ref)))


def test_gradient_matches_oracle(env):
    xb, dev = env
    for seed, B in ((1, 37), (2, 300)):
        model, P, X, lab, Xt, Lt = _setup(xb, dev, seed, B)
        loss, g = model.loss_grad(Xt, Lt)
        lo, go = oracle.mlp_loss_grad(P.astype(np.float64), DIMS, X.astype(np.float64), lab)
        assert abs(loss - lo) <= 1e-5 * (1 + abs(lo))
        g = g.cpu().numpy().astype(np.float64)
        scale = np.max(np.abs(go))
        assert np.max(np.abs(g - go)) <= 1e-4 * scale, np.max(np.abs(g - go)) / scale


def test_adam_step_matches_oracle(env):
    xb, dev = env
    model, P, X, lab, Xt, Lt = _setup(xb, dev, 3)
    _, g = model.loss_grad(Xt, Lt)
    model.adam(1, lr=1e-2)
    got = model.get_params().astype(np.float64)
    Pd, M, V = P.astype(np.float64), np.zeros(P.size), np.zeros(P.size)
    oracle.adam(Pd, g.cpu().numpy().astype(np.float64), M, V, 1, lr=1e-2)
    np.testing.assert_allclose(got, Pd, rtol=1e-5, atol=1e-6)


def test_training_fits_separable_data(env):
    xb, dev = env
    import torch
    rng = np.random.default_rng(7)
    X = rng.standard_normal((512, 8)).astype(np.float32)
    lab = np.stack([(X[:, 0] > 0) * 1 + (X[:, 1] > 0) * 2, (X[:, 2] > 0) * 3,
                    (X[:, 3] > 0) * 4, (X[:, 4] > 0) * 5], axis=1).astype(np.int32)
    model = xb.Mlp(seed=1)
    Xt, Lt = torch.tensor(X, device=dev), torch.tensor(lab, device=dev)
    l0, _ = model.loss_grad(Xt, Lt)
    loss = model.train(Xt, Lt, epochs=150, batch=64, lr=3e-3, seed=0)
    assert loss < 0.15 * l0
    acc = (model.predict(Xt) == lab).mean()
    assert acc > 0.95
    # deterministic: the same seed gives the same parameters
    m2 = xb.Mlp(seed=1)
    m2.train(Xt, Lt, epochs=150, batch=64, lr=3e-3, seed=0)
    np.testing.assert_array_equal(model.get_params(), m2.get_params())


def test_save_load_roundtrip(env, tmp_path):
    xb, dev = env
    model, P, X, lab, Xt, _ = _setup(xb, dev, 4)
    model.set_norm(np.arange(8, dtype=np.float32), np.full(8, 2.0, np.float32))
    path = str(tmp_path / "m.bin")
    model.save(path)
    m2 = xb.Mlp.load(path)
    np.testing.assert_array_equal(m2.get_params(), P)
    np.testing.assert_array_equal(m2.forward(Xt).cpu().numpy(), model.forward(Xt).cpu().numpy())


def test_tune_mlp_sets_a_valid_choice(env):
    xb, dev = env
    from paper_2405_01599_gb300 import gen
    model = xb.Mlp(seed=5)
    for A, ok in ((gen.powerlaw(n=5000, seed=2), (0, 1, 2)), (gen.laplace3d(10, upper=True), (3, 4))):
        plan = xb.Plan.from_host(A, dev)
        ch, m = plan.tune_mlp(model)
        assert ch["variant"] in ok and m in xb.TUNER_RESTARTS
        if ch["variant"] == 2:
            assert ch["block"] <= 256 and ch["ipt"] in (4, 8, 16, 32)
