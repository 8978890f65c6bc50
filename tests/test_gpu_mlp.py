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


@pytest.mark.parametrize("hidden,layers,rows", [(128, 3, 512), (48, 2, 1000)])
def test_gradient_per_tensor_elementwise(emc, hidden, layers, rows):
    """Every element of every parameter tensor (W and b of each layer) of the
    tensor-core gradient against the FP64 reference.  BF16 operands round to
    u = 2^-9 relative; an element's operands come out of the forward chain
    (activations) and the backward chain (deltas), each up to `depth` rounded
    products deep, two roundings per product, so it may err by
    2 x 2 depth x u x the sum of the absolute values of its products (from
    the FP64 reference).  The per-tensor relative error and direction are
    checked too."""
    net, nrm, sizes, rng = make(emc, hidden=hidden, layers=layers, seed=17)
    X = rng.normal(size=(rows, 4)).astype(np.float32)
    Y = rng.normal(size=(rows, 7)).astype(np.float32)
    _, g = net.grad(X, Y)
    theta = net.params().astype(np.float64)
    _, gref = ref.loss_and_grad(theta, sizes, X, Y, nrm)
    S = ref.grad_abs_products(theta, sizes, X, Y, nrm)
    depth = len(sizes) - 1
    tol = 4.0 * depth * 2.0 ** -9 * S + 1e-7 * np.abs(gref).max()
    off = 0
    for l, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        for name, cnt in (("W", a * b), ("b", b)):
            sl = slice(off, off + cnt)
            off += cnt
            err = np.abs(g[sl] - gref[sl])
            assert (err <= tol[sl]).all(), (l, name, float((err / tol[sl]).max()))
            rel = np.linalg.norm(g[sl] - gref[sl]) / np.linalg.norm(gref[sl])
            cos = float(g[sl] @ gref[sl] / (np.linalg.norm(g[sl]) * np.linalg.norm(gref[sl])))
            assert rel < 0.03 and cos > 0.999, (l, name, rel, cos)
    assert off == g.size


def test_surrogate_on_the_context_equals_the_standalone_network(emc):
    """emc_surrogate_train / emc_surrogate_infer on a Monte Carlo context run
    the same kernels as the standalone network: the same training gives the
    same loss history and predictions (to the rounding order of the split-K
    FP32 atomic sums, which may differ between runs)."""
    import workloads as W
    rng = np.random.default_rng(21)
    X = rng.uniform(-1, 1, size=(4000, 4)).astype(np.float32)
    Y = np.stack([X[:, 0] * X[:, 1], np.sin(X[:, 2]), X[:, 3] ** 2], axis=1).astype(np.float32)
    args = (4, 64, 2, 3, np.zeros(4), np.ones(4), np.zeros(3), np.ones(3))
    net = emc.emc.Mlp(*args, seed=4)
    h1 = net.train(X, Y, steps=200, batch=256, lr=2e-3, seed=8)
    with emc.Context(W.bulk(n_particles=10)) as ctx:
        with pytest.raises(emc.EmcError):
            ctx.emc_surrogate_infer(X[:5])
        h2 = ctx.emc_surrogate_train(emc.emc.mlp_config(*args, seed=4), X, Y, steps=200, batch=256, lr=2e-3, seed=8)
        np.testing.assert_allclose(h2, h1, rtol=1e-2)
        p1, p2 = net.params(), ctx.emc_surrogate_params()
        assert p1.size == p2.size and np.linalg.norm(p2 - p1) <= 1e-3 * np.linalg.norm(p1)
        y1, y2 = net.infer(X[:300]), ctx.emc_surrogate_infer(X[:300])
        assert y2.shape == y1.shape and np.abs(y2 - y1).max() <= 1e-2 * np.abs(y1).max()


def test_expired_wait_is_reported_and_the_handle_recovers(emc):
    """The reporting path of an expired tensor-core wait: with the device
    error word set (as the bounded mbarrier wait sets it; no wait is made to
    expire), the next call returns EMC_ETIMEOUT with its message, and the
    call after it runs normally with the same results."""
    net, nrm, sizes, rng = make(emc)
    X = rng.normal(size=(300, 4)).astype(np.float32)
    want = net.infer(X)
    net.debug_set_error()
    with pytest.raises(emc.EmcError) as ei:
        net.infer(X)
    assert ei.value.status == 5 and "expired" in str(ei.value)
    np.testing.assert_array_equal(net.infer(X), want)


@pytest.mark.parametrize("n_in,hidden,layers,n_out,rows", [(4, 128, 3, 7, 115_200), (4, 128, 3, 7, 1),
                                                           (16, 48, 2, 16, 1000), (3, 256, 1, 5, 333),
                                                           (5, 16, 6, 2, 129)])
def test_fused_inference_equals_layer_by_layer(emc, n_in, hidden, layers, n_out, rows):
    """The fused inference (every layer in one launch, weights and one
    activation tile in shared memory) against the layer-by-layer GEMM path
    on the same weights (the same normalisation, BF16 operands, MMA order,
    FP32 bias and SiLU): equal to FP32 rounding, ragged tiles included, and
    both against the FP64 reference network."""
    net, nrm, sizes, rng = make(emc, n_in=n_in, hidden=hidden, layers=layers, n_out=n_out, seed=17)
    X = rng.normal(size=(rows, n_in)).astype(np.float32)
    fused = net.infer(X)
    net.set_fused(False)
    layered = net.infer(X)
    net.set_fused(True)
    scale = np.abs(layered - nrm["y_shift"]).max()
    np.testing.assert_allclose(fused, layered, rtol=0, atol=1e-5 * scale)
    idx = rng.choice(rows, min(rows, 2000), replace=False)
    want = ref.predict(net.params().astype(np.float64), sizes, X[idx], nrm)
    assert np.abs(fused[idx] - want).max() / np.abs(want - nrm["y_shift"]).max() < 3e-2
