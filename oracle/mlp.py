"""FP64 reference of the surrogate network (test infrastructure only).

A fully connected network: h_0 = (x - x_shift) / x_scale; h_{l+1} =
silu(W_l h_l + b_l) for the hidden layers; z = W_L h_L + b_L; loss = mean over
rows and outputs of (z - (y - y_shift) / y_scale)^2.  The parameter vector
lists, per layer, W (out x in, row-major) then b.  Backward by the chain
rule, written out; pinned by finite differences in the tests.
"""
import numpy as np


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def unpack(theta, sizes):
    out, off = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = theta[off:off + n_in * n_out].reshape(n_out, n_in)
        off += n_in * n_out
        b = theta[off:off + n_out]
        off += n_out
        out.append((W, b))
    return out


def forward(theta, sizes, X, norm):
    h = (X - norm["x_shift"]) / norm["x_scale"]
    hs, zs = [h], []
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if l < len(layers) - 1 else z
        hs.append(h)
    return hs, zs


def loss_and_grad(theta, sizes, X, Y, norm):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    hs, zs = forward(theta, sizes, X, norm)
    t = (Y - norm["y_shift"]) / norm["y_scale"]
    d = zs[-1] - t
    n = d.size
    loss = float((d * d).sum() / n)
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    grads = [None] * len(layers)
    dz = 2.0 * d / n
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (dz.T @ hs[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * dsilu(zs[l - 1])
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, g


def predict(theta, sizes, X, norm):
    _, zs = forward(theta, sizes, X, norm)
    return zs[-1] * norm["y_scale"] + norm["y_shift"]


def grad_abs_products(theta, sizes, X, Y, norm):
    """Per parameter, the sum of absolute values of the products that make
    its gradient, carried through the chain with absolute values:
    |dz_L| = |2 d / n|, |dz_l| = (|dz_{l+1}| |W_l|) |silu'(z_l)|, and
    S_W = |dz_{l+1}|^T |h_l|, S_b = sum |dz_{l+1}|.  An element computed with
    rounded operands of relative precision u errs by at most about
    (depth) u S (the standard running-error bound of sums of products)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    hs, zs = forward(theta, sizes, X, norm)
    t = (Y - norm["y_shift"]) / norm["y_scale"]
    d = zs[-1] - t
    n = d.size
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    out = [None] * len(layers)
    dz = np.abs(2.0 * d / n)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        out[l] = (dz.T @ np.abs(hs[l]), dz.sum(axis=0))
        if l > 0:
            dz = (dz @ np.abs(W)) * np.abs(dsilu(zs[l - 1]))
    return np.concatenate([np.concatenate([sW.ravel(), sb]) for sW, sb in out])
