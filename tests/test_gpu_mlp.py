"""Surrogate network on the tensor cores (BF16 operands, FP32 accumulation)
against the FP64 reference network with the same weights."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def make(emc, n_in=4, hidden=128, layers=3, n_out=7, seed=3):
    rng = np.random.default_rng(seed)
    nrm = {"x_shift": rng.normal(size=n_in), "x_scale": rng.uniform(0.5, 2, n_in),
           "y_shift": rng.normal(size=n_out), "y_scale": rng.uniform(0.5, 2, n_out)}
    net = emc.emc.Mlp(n_in, hidden, layers, n_out, nrm["x_shift"], nrm["x_scale"], nrm["y_shift"], nrm["y_scale"],
                      seed=seed)
    sizes = [n_in] + [hidden] * layers + [n_out]
    return net, nrm, sizes, rng


def test_forward_matches_fp64_reference(emc):
    net, nrm, sizes, rng = make(emc)
    X = rng.normal(size=(1000, 4)).astype(np.float32)
    got = net.infer(X)
    want = ref.predict(net.params().astype(np.float64), sizes, X, nrm)
    err = np.abs(got - want).max() / np.abs(want - nrm["y_shift"]).max()
    assert err < 3e-2, err


def test_gradient_matches_fp64_reference(emc):
    net, nrm, sizes, rng = make(emc, seed=5)
    X = rng.normal(size=(512, 4)).astype(np.float32)
    Y = rng.normal(size=(512, 7)).astype(np.float32)
    loss, g = net.grad(X, Y)
    lref, gref = ref.loss_and_grad(net.params().astype(np.float64), sizes, X, Y, nrm)
    assert loss == pytest.approx(lref, rel=2e-2)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    rel = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
    assert cos > 0.999 and rel < 0.05, (cos, rel)


def test_training_fits_a_smooth_map(emc):
    net, nrm, sizes, rng = make(emc, n_out=3, seed=7)
    X = rng.uniform(-1, 1, size=(20000, 4)).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], np.exp(-X[:, 2] ** 2) + X[:, 3], X[:, 0] * X[:, 3]], axis=1)
    Y = (Y * nrm["y_scale"] + nrm["y_shift"]).astype(np.float32)
    hist = net.train(X, Y, steps=1500, batch=512, lr=2e-3, seed=1)
    assert hist[-100:].mean() < 0.05 * hist[:10].mean()
    Xt = rng.uniform(-1, 1, size=(2000, 4)).astype(np.float32)
    Yt = np.stack([np.sin(2 * Xt[:, 0]) * Xt[:, 1], np.exp(-Xt[:, 2] ** 2) + Xt[:, 3], Xt[:, 0] * Xt[:, 3]], axis=1)
    pred = (net.infer(Xt) - nrm["y_shift"]) / nrm["y_scale"]
    assert np.sqrt(np.mean((pred - Yt) ** 2)) < 0.05


def test_params_round_trip(emc):
    net, nrm, sizes, rng = make(emc, hidden=32, layers=2, seed=9)
    p = net.params()
    q = rng.normal(scale=0.1, size=p.size).astype(np.float32)
    net.params(q)
    assert np.array_equal(net.params(), q)
    X = rng.normal(size=(64, 4)).astype(np.float32)
    want = ref.predict(q.astype(np.float64), sizes, X, nrm)
    assert np.abs(net.infer(X) - want).max() < 3e-2 * np.abs(want - nrm["y_shift"]).max()


@pytest.mark.parametrize("hidden", [48, 256])
def test_ragged_gradient_and_widths(emc, hidden):
    """1000 rows (the last 128-row tile and the last 64-wide K block of the
    weight-gradient product are partial) at hidden widths 48 and 256 (tensor
    memory of 64 and 256 columns)."""
    net, nrm, sizes, rng = make(emc, hidden=hidden, layers=2, seed=11)
    X = rng.normal(size=(1000, 4)).astype(np.float32)
    Y = rng.normal(size=(1000, 7)).astype(np.float32)
    loss, g = net.grad(X, Y)
    lref, gref = ref.loss_and_grad(net.params().astype(np.float64), sizes, X, Y, nrm)
    assert loss == pytest.approx(lref, rel=2e-2)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos > 0.999, cos
    got = net.infer(X)
    want = ref.predict(net.params().astype(np.float64), sizes, X, nrm)
    assert np.abs(got - want).max() / np.abs(want - nrm["y_shift"]).max() < 3e-2


def test_full_size_inference_sampled(emc):
    """115,200 queries (1800 subcells x 64 bias points) in one call; sampled
    rows against the FP64 reference."""
    net, nrm, sizes, rng = make(emc, seed=13)
    X = rng.normal(size=(115_200, 4)).astype(np.float32)
    got = net.infer(X)
    idx = rng.choice(X.shape[0], 3000, replace=False)
    want = ref.predict(net.params().astype(np.float64), sizes, X[idx], nrm)
    assert np.abs(got[idx] - want).max() / np.abs(want - nrm["y_shift"]).max() < 3e-2
