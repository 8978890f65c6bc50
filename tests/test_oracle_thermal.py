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


# ---- phonon-electron scattering, Eq. (1)
def test_fermi_half_closed_form_at_zero():
    # F_1/2(0) = (1 - 2^(-1/2)) zeta(3/2)
    from scipy.special import zeta
    assert thermal.fermi_half(0.0) == pytest.approx((1 - 2 ** -0.5) * zeta(1.5), rel=1e-10)


def test_fermi_level_limits():
    m = W.ELECTRON_PHONON_GAN["m_rel"]
    # non-degenerate: n = N_c exp(E_F / kT)
    n = 1e18
    Nc = 2.0 * (m * 9.1093837015e-31 * 1.380649e-23 * 300.0 / (2 * np.pi * 1.054571817e-34 ** 2)) ** 1.5
    assert thermal.fermi_level(n, 300.0, m) == pytest.approx(1.380649e-23 * 300.0 * np.log(n / Nc), rel=1e-9)
    # degenerate (T -> 0): E_F = hbar^2 (3 pi^2 n)^(2/3) / 2 m*
    n = 1e26
    ef0 = 1.054571817e-34 ** 2 * (3 * np.pi ** 2 * n) ** (2 / 3) / (2 * m * 9.1093837015e-31)
    assert thermal.fermi_level(n, 20.0, m) == pytest.approx(ef0, rel=1e-4)


def test_tau_e_non_degenerate_limit():
    # for E_F far below the band edge the braces of Eq. (1) reduce to
    # exp(-(m v^2/2 - E_F)/kT - (hbar w)^2 / 8 m v^2 kT) * 2 sinh(hbar w / 2kT),
    # and exp(E_F / kT) = n / N_c
    el = W.ELECTRON_PHONON_GAN
    kB, hb, me, e = 1.380649e-23, 1.054571817e-34, 9.1093837015e-31, 1.602176634e-19
    T, n = 300.0, 1e16
    m, v = el["m_rel"] * me, el["vg_m_s"]
    Nc = 2.0 * (m * kB * T / (2 * np.pi * hb ** 2)) ** 1.5
    half = 0.5 * m * v * v
    pre = (el["Da_eV"] * e) ** 2 * m ** 3 * v / (4 * np.pi * hb ** 4 * el["rho_kg_m3"]) * kB * T / half
    for w in (1e11, 1e12, 3e12):
        want = pre * (n / Nc) * np.exp(-half / (kB * T) - (hb * w) ** 2 / (8 * m * v * v * kB * T)) \
            * 2 * np.sinh(hb * w / (2 * kB * T))
        assert thermal.tau_e_inv(w, T, n, el) == pytest.approx(want, rel=1e-6)


def test_electron_scattering_kappa_reduction():
    # the paper: free electrons reduce the room-temperature conductivity of
    # Si-doped GaN by ~13% at 7.0e18 cm^-3 (its ref. [16]); this reading of
    # Eq. (1) gives 16%
    el = W.ELECTRON_PHONON_GAN
    k0 = thermal.kappa(300.0, W.TABLE_II_GAN)
    k7 = thermal.kappa(300.0, W.TABLE_II_GAN, n_e=7e24, elec=el)
    assert 0.10 < 1.0 - k7 / k0 < 0.20
    # more electrons scatter more; no electrons, no change
    k1 = thermal.kappa(300.0, W.TABLE_II_GAN, n_e=1e24, elec=el)
    assert k7 < k1 < k0
    assert thermal.kappa(300.0, W.TABLE_II_GAN, n_e=0.0, elec=el) == k0


# ---------------------------------------- diffuse mismatch model, Eqs. (2)-(3)
KB, HB = 1.380649e-23, 1.054571817e-34


def sound_speed(mat):
    """Long-wavelength group velocity of the sine branch, omega_max pi / 2 q0."""
    return mat["omega_max_rad_s"] * np.pi / (2.0 * mat["k0_per_m"])


def test_dmm_transmissivities_are_complementary_and_reciprocal():
    """tau_12 + tau_21 = 1 where both sides have states, the detailed balance
    of the diffuse mismatch model (sum v D)_1 tau_12 = (sum v D)_2 tau_21,
    one half between identical materials, and nothing transmitted into
    material 2 above its highest frequency."""
    gan, sic = W.TABLE_II_GAN, W.TABLE_II_SIC
    for w in np.linspace(1e11, 0.999 * gan["omega_max_rad_s"], 23):
        t12, t21 = thermal.tau12(w, gan, sic), thermal.tau12(w, sic, gan)
        assert t12 + t21 == pytest.approx(1.0, abs=1e-14)
        _, v1, D1 = thermal.branch(gan, w)
        _, v2, D2 = thermal.branch(sic, w)
        assert v1 * D1 * t12 == pytest.approx(v2 * D2 * t21, rel=1e-12)
        assert thermal.tau12(w, gan, gan) == pytest.approx(0.5, abs=1e-15)
    for w in np.linspace(1.001 * gan["omega_max_rad_s"], 0.999 * sic["omega_max_rad_s"], 7):
        assert thermal.tau12(w, sic, gan) == 0.0
        assert thermal.tau12(w, gan, sic) == 1.0  # Eq. (2) with no states on the wire's side
    # long waves: tau_12 -> v_1^2 / (v_1^2 + v_2^2) (linear dispersion)
    v1, v2 = sound_speed(gan), sound_speed(sic)
    assert thermal.tau12(1e9, gan, sic) == pytest.approx(v1 ** 2 / (v1 ** 2 + v2 ** 2), rel=1e-6)


def test_interface_conductance_low_temperature_limit():
    """Only long waves are excited at low T: Eq. (3) becomes
    1/R_K = pi^2 k^4 T^3 tau_12(0) / (10 hbar^3 v_1^2) (three branches,
    integral of x^4 e^x / (e^x - 1)^2 = 4 pi^4 / 15)."""
    gan, sic = W.TABLE_II_GAN, W.TABLE_II_SIC
    v1, v2 = sound_speed(gan), sound_speed(sic)
    t0 = v1 ** 2 / (v1 ** 2 + v2 ** 2)
    for T in (0.05, 0.1):
        want = np.pi ** 2 * KB ** 4 * T ** 3 * t0 / (10.0 * HB ** 3 * v1 ** 2)
        assert thermal.interface_conductance(T, gan, sic) == pytest.approx(want, rel=1e-5)


def test_interface_conductance_classical_limit():
    """At high T every mode holds k: between identical materials (tau = 1/2)
    Eq. (3) becomes (3/8) (k / 2 pi^2) (2 q0 / pi)^2 omega_max (pi^2/4 - 2),
    the integral of arcsin^2 over [0, 1] being pi^2/4 - 2."""
    gan = W.TABLE_II_GAN
    q0, wm = gan["k0_per_m"], gan["omega_max_rad_s"]
    want = 3.0 / 8.0 * KB / (2 * np.pi ** 2) * (2 * q0 / np.pi) ** 2 * wm * (np.pi ** 2 / 4 - 2)
    assert thermal.interface_conductance(1e7, gan, gan) == pytest.approx(want, rel=1e-8)


def test_interface_conductance_gan_on_sic():
    """GaN -> SiC at 300 K: R_K = 2.32e-8 m^2 K/W from Eqs. (2)-(3) with the
    Table II dispersions (context: measured GaN/SiC boundary resistances are
    of order 1e-8); it saturates with temperature as the modes fill."""
    g300 = thermal.interface_conductance(300.0, W.TABLE_II_GAN, W.TABLE_II_SIC)
    assert 1.0 / g300 == pytest.approx(2.32e-8, rel=0.01)
    g600 = thermal.interface_conductance(600.0, W.TABLE_II_GAN, W.TABLE_II_SIC)
    g50 = thermal.interface_conductance(50.0, W.TABLE_II_GAN, W.TABLE_II_SIC)
    assert g50 < g300 < g600 < 1.01 * thermal.interface_conductance(1e5, W.TABLE_II_GAN, W.TABLE_II_SIC)


def test_fourier_bottom_boundary_puts_the_interface_in_series():
    """The operator's bottom boundary with an interface conductance G per
    area equals the lumped boundary with 1/h = 1/h_lumped + 1/G (the half
    cell, the lumped part and the interface in series)."""
    cfg = grid(6)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    kap = np.full(n, 100.0)
    g_if = np.full(n, 4.0e7)
    A1, b1 = thermal.operator(cfg, kap, 300.0, 5e8, g_if)
    A2, b2 = thermal.operator(cfg, kap, 300.0, 1.0 / (1.0 / 5e8 + 1.0 / 4.0e7))
    np.testing.assert_allclose(A1.toarray(), A2.toarray(), rtol=1e-13)
    np.testing.assert_allclose(b1, b2, rtol=1e-13)
