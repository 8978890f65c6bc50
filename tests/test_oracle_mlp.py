"""Pin of the FP64 reference network: analytic gradient vs central finite
differences, and a closed case (one linear layer = least squares)."""
import numpy as np

from oracle import mlp


def norms(n_in, n_out, rng):
    return {"x_shift": rng.normal(size=n_in), "x_scale": rng.uniform(0.5, 2, n_in),
            "y_shift": rng.normal(size=n_out), "y_scale": rng.uniform(0.5, 2, n_out)}


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [4, 9, 7, 3]
    nrm = norms(4, 3, rng)
    n = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    theta = rng.normal(scale=0.5, size=n)
    X = rng.normal(size=(13, 4))
    Y = rng.normal(size=(13, 3))
    _, g = mlp.loss_and_grad(theta, sizes, X, Y, nrm)
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, sizes, X, Y, nrm)[0] - mlp.loss_and_grad(theta - e, sizes, X, Y, nrm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd))


def test_linear_layer_gradient_is_least_squares_normal_equation():
    rng = np.random.default_rng(1)
    sizes = [3, 2]
    nrm = {"x_shift": np.zeros(3), "x_scale": np.ones(3), "y_shift": np.zeros(2), "y_scale": np.ones(2)}
    X = rng.normal(size=(50, 3))
    Y = rng.normal(size=(50, 2))
    A = np.hstack([X, np.ones((50, 1))])
    sol = np.linalg.lstsq(A, Y, rcond=None)[0]  # [4][2]
    W, b = sol[:3].T, sol[3]
    theta = np.concatenate([W.ravel(), b])
    _, g = mlp.loss_and_grad(theta, sizes, X, Y, nrm)
    assert np.abs(g).max() < 1e-12
