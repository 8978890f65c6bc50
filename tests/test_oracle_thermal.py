"""Pins of the reference thermal side: kappa(T) of GaN from Table II against
the independently computed values, the T^-1-like fall with temperature, the
boundary term, discrete energy conservation and a 1-D closed form."""
import numpy as np
import pytest

import workloads as W
from oracle import thermal


def test_kappa_gan_matches_independent_quadrature():
    # 228 W/m/K at 300 K and 143 at 415 K were obtained separately from
    # Table II with the same kinetic formula (parameters fitted to measured
    # bulk GaN; the measured value is ~230 W/m/K)
    assert thermal.kappa(300.0, W.TABLE_II_GAN) == pytest.approx(228.0, rel=0.01)
    assert thermal.kappa(415.0, W.TABLE_II_GAN) == pytest.approx(143.0, rel=0.01)
    assert thermal.kappa(300.0, W.TABLE_II_SIC) == pytest.approx(350.0, rel=0.02)


def test_kappa_boundary_scattering_reduces():
    k_bulk = thermal.kappa(300.0, W.TABLE_II_GAN)
    k_120 = thermal.kappa(300.0, W.TABLE_II_GAN, L_b=120e-9)
    k_1um = thermal.kappa(300.0, W.TABLE_II_GAN, L_b=1e-6)
    assert k_120 < k_1um < k_bulk


def grid(nx=20):
    return W.nanowire(n_particles=1, nx=nx, Lx=nx * 10e-9)


def test_heat_balance_and_symmetry():
    c = grid()
    n = c["nx"] * c["ny"] * c["nz"]
    rng = np.random.default_rng(0)
    q = rng.uniform(0, 1e18, n)
    h_b = 2e8
    T = thermal.solve(c, q, W.TABLE_II_GAN, h_bottom=h_b, L_b=120e-9)
    # every watt generated leaves through the contacts or the bottom face
    kap = np.array([thermal.kappa(t, W.TABLE_II_GAN, 120e-9) for t in T])
    A, b = thermal.operator(c, kap, 300.0, h_b)
    Vc = c["Lx"] * c["Ly"] * c["Lz"] / n
    out = (A @ T - b + A.diagonal() * 0)  # residual form: A T - b = q
    assert np.allclose(out, q, rtol=1e-8, atol=1e-8 * q.max())
    assert (T > 300.0).all()


def test_one_dimensional_closed_form():
    # uniform q, kappa fixed (tiny temperature rise), adiabatic sides and no
    # bottom loss: T(x) = T_s + q x (L - x) / (2 kappa) up to the discrete
    # half-cell boundary treatment, which is exact for a parabola sampled at
    # the cell centres except for a constant offset of q h^2 / (8 kappa)
    c = grid(40)
    n = c["nx"] * c["ny"] * c["nz"]
    q = np.full(n, 1e12)
    T = thermal.solve(c, q, W.TABLE_II_GAN, h_bottom=1e-30, L_b=0.0)
    k = thermal.kappa(300.0, W.TABLE_II_GAN)
    L = c["Lx"]
    h = L / c["nx"]
    x = (np.arange(c["nx"]) + 0.5) * h
    want = 300.0 + q[0] * x * (L - x) / (2 * k) + q[0] * h * h / (8 * k)
    got = T.reshape(c["nx"], -1)[:, 0]
    assert np.allclose(got - 300.0, want - 300.0, rtol=2e-3)
