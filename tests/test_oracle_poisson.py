"""Pins of the oracle's Poisson solve and field on the subcell grid.

The oracle applies the 7-point operator cell by cell and solves it with CG.
These tests build the same discrete problem another way, as a Kronecker sum of
1-D operators assembled densely and solved with LAPACK, and check exact
discrete solutions (constant and linear potentials).
"""
import numpy as np
import pytest
from scipy import constants as sc

import workloads as W


def grid(nx=8, ny=3, nz=6, **kw):
    c = W.nanowire(n_particles=1, nx=nx, ny=ny, nz=nz, Lx=nx * 10e-9, **kw)
    return c


def op1d(n, h, lo, hi):
    """-d2/dx2 on n cell centres; lo/hi 'D' = Dirichlet face half a cell away,
    'N' = Neumann face."""
    A = np.zeros((n, n))
    for i in range(n):
        if i > 0:
            A[i, i] += 1; A[i, i - 1] -= 1
        elif lo == "D":
            A[i, i] += 2
        if i < n - 1:
            A[i, i] += 1; A[i, i + 1] -= 1
        elif hi == "D":
            A[i, i] += 2
    return A / (h * h)


def kron3(Ax, Ay, Az):
    Ix, Iy, Iz = (np.eye(a.shape[0]) for a in (Ax, Ay, Az))
    return np.kron(np.kron(Ax, Iy), Iz) + np.kron(np.kron(Ix, Ay), Iz) + np.kron(np.kron(Ix, Iy), Az)


def test_constant_potential_is_exact(oracle_mod):
    c = grid(Vs=0.7, Vd=0.7, Vg=0.7)
    phi = oracle_mod.poisson(c, None)
    assert np.allclose(phi, 0.7, rtol=0, atol=1e-12)


def test_linear_potential_without_gate(oracle_mod):
    c = grid(nx=10, Vs=-0.4, Vd=3.0, gate_on=0)
    phi = oracle_mod.poisson(c, None).reshape(c["nx"], c["ny"], c["nz"])
    xc = (np.arange(c["nx"]) + 0.5) * c["Lx"] / c["nx"]
    want = c["Vs"] + (c["Vd"] - c["Vs"]) * xc / c["Lx"]
    assert np.allclose(phi, want[:, None, None], rtol=0, atol=1e-11)
    Ef = oracle_mod.field(c, phi.ravel())
    assert np.allclose(Ef[:, 0], -(c["Vd"] - c["Vs"]) / c["Lx"], rtol=1e-10)
    assert np.allclose(Ef[:, 1:], 0.0, atol=1e-3)


@pytest.mark.parametrize("gate_all", [False, True])
def test_matches_kronecker_assembly(oracle_mod, gate_all):
    nx, ny, nz = 12, 3, 6
    kw = dict(Vs=0.2, Vd=1.7, Vg=-0.5)
    if gate_all:
        c = grid(nx, ny, nz, gate_on=1, **kw)
        c.update(gate_x0=0.0, gate_x1=c["Lx"])
    else:
        c = grid(nx, ny, nz, gate_on=0, **kw)
    hx, hy, hz = c["Lx"] / nx, c["Ly"] / ny, c["Lz"] / nz
    top = "D" if gate_all else "N"
    A = kron3(op1d(nx, hx, "D", "D"), op1d(ny, hy, "N", top), op1d(nz, hz, "N", top))
    rng = np.random.default_rng(7)
    rho = sc.e * 1e24 * rng.uniform(-1, 1, nx * ny * nz)
    b = rho / (c["eps_s"] * sc.epsilon_0)
    b = b.reshape(nx, ny, nz)
    b[0] += 2 * c["Vs"] / hx ** 2
    b[-1] += 2 * c["Vd"] / hx ** 2
    if gate_all:
        b[:, -1, :] += 2 * c["Vg"] / hy ** 2
        b[:, :, -1] += 2 * c["Vg"] / hz ** 2
    want = np.linalg.solve(A, b.ravel())
    got = oracle_mod.poisson(c, rho)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    # the operator itself, applied to a random vector
    x = rng.normal(size=nx * ny * nz)
    assert np.allclose(oracle_mod.poisson_apply(c, x), A @ x, rtol=1e-12, atol=1e-12 * np.abs(A @ x).max())


def test_partial_gate_symmetric_positive(oracle_mod):
    c = grid(nx=16)
    n = c["nx"] * c["ny"] * c["nz"]
    A = np.stack([oracle_mod.poisson_apply(c, e) for e in np.eye(n)], axis=1)
    assert np.allclose(A, A.T, rtol=1e-12, atol=0)
    assert np.linalg.eigvalsh(A).min() > 0


def test_field_central_and_one_sided(oracle_mod):
    c = grid(nx=5, ny=4, nz=6)
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    hy = c["Ly"] / ny
    yc = (np.arange(ny) + 0.5) * hy
    phi = np.broadcast_to((yc ** 2)[None, :, None], (nx, ny, nz)).ravel().copy()
    Ef = oracle_mod.field(c, phi).reshape(nx, ny, nz, 3)
    # central difference of y^2 is exact (2y); edges use the one-sided slope
    assert np.allclose(Ef[:, 1:-1, :, 1], -2 * yc[None, 1:-1, None], rtol=1e-12)
    assert np.allclose(Ef[:, 0, :, 1], -(yc[1] ** 2 - yc[0] ** 2) / hy, rtol=1e-12)
    assert np.allclose(Ef[:, -1, :, 1], -(yc[-1] ** 2 - yc[-2] ** 2) / hy, rtol=1e-12)
    assert np.allclose(Ef[..., 0], 0) and np.allclose(Ef[..., 2], 0)
