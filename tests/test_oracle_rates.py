"""Pins of the oracle's random numbers, scattering rates and angle samplers.

The oracle's rates are closed forms; these tests reach the same numbers by a
different route: the Fermi golden rule integrated numerically over the final
states (matrix element x delta function, with the density of states taken by
numerical differentiation of the Kane dispersion), detailed balance between
absorption and emission, and the exact inversion of the angular CDFs checked
by quadrature.  Constants come from scipy.constants, not from the oracle.
"""
import math
import os

import numpy as np
import pytest
from scipy import constants as sc
from scipy import integrate

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
Q, HB, KB, M0, E0 = sc.e, sc.hbar, sc.k, sc.m_e, sc.epsilon_0


def read_kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(x, 16) for x in line.split()]
                rows.append((tuple(v[:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


def test_philox_known_answers(oracle_mod):
    for ctr, key, out in read_kat():
        assert oracle_mod.philox(ctr, key) == out


def test_uniform_map_exact(oracle_mod):
    # (2 (x >> 9) + 1) 2^-24: odd multiples of 2^-24 in (0, 1)
    assert oracle_mod.u01(0) == 2.0 ** -24
    assert oracle_mod.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle_mod.u01(0x80000000) == 0.5 + 2.0 ** -24
    assert oracle_mod.u01(511) == oracle_mod.u01(0)


# ----------------------------------------------------------- golden rule
class Band:
    def __init__(self, m_rel, alpha_eV):
        self.m = m_rel * M0
        self.a = alpha_eV / Q

    def k_of_E(self, E):
        return math.sqrt(2 * self.m * E * (1 + self.a * E)) / HB

    def dk_dE(self, E):
        h = max(E * 1e-5, 1e-26)
        return (self.k_of_E(E + h) - self.k_of_E(E - h)) / (2 * h)

    def dos(self, E):
        """states per unit volume and energy, one spin: k^2 dk/dE / (2 pi^2)"""
        k = self.k_of_E(E)
        return k * k * self.dk_dE(E) / (2 * math.pi ** 2)


def golden_rule(k, kp, dk_dE_p, M2_of_q2):
    """(2 pi / hbar) int d^3k' / (2 pi)^3 |M|^2 delta(E' - Ef), angle by quad."""
    ang = integrate.quad(lambda c: M2_of_q2(k * k + kp * kp - 2 * k * kp * c), -1, 1,
                         epsabs=0, epsrel=1e-12, limit=200)[0]
    return (2 * math.pi / HB) * kp * kp * dk_dE_p * 2 * math.pi * ang / (2 * math.pi) ** 3


def cfg(**kw):
    return W.bulk(n_particles=1, **kw)


def occupations(T, hw_eV):
    x = hw_eV * Q / (KB * T)
    return 1.0 / math.expm1(x)


@pytest.mark.parametrize("E_eV", [0.005, 0.05, 0.2, 0.9, 2.5])
@pytest.mark.parametrize("v", [0, 1, 2])
def test_pop_rate_golden_rule(oracle_mod, v, E_eV):
    c = cfg(T=300.0)
    s = oracle_mod.Sim(c)
    b = Band(c["m_rel"][v], c["alpha_per_eV"][v])
    hw = c["hw_lo_eV"] * Q
    w0 = hw / HB
    N0 = occupations(c["T"], c["hw_lo_eV"])
    E = E_eV * Q
    pref = Q * Q * hw / (2 * E0) * (1 / c["eps_inf"] - 1 / c["eps_s"])
    for mech, Ef, occ in ((1, E + hw, N0), (2, E - hw, N0 + 1)):
        got = s.rate(v, mech, E_eV)
        if Ef <= 0:
            assert got == 0.0
            continue
        want = golden_rule(b.k_of_E(E), b.k_of_E(Ef), b.dk_dE(Ef), lambda q2: pref * occ / q2)
        assert got == pytest.approx(want, rel=1e-7), (mech, got, want)
    assert w0 > 0


@pytest.mark.parametrize("E_eV", [0.001, 0.02, 0.3, 1.5])
@pytest.mark.parametrize("Nd_cm3", [1e16, 1e18])
def test_impurity_rate_golden_rule(oracle_mod, E_eV, Nd_cm3):
    c = cfg(T=400.0, Nd_cm3=Nd_cm3)
    s = oracle_mod.Sim(c)
    b = Band(c["m_rel"][0], c["alpha_per_eV"][0])
    es = c["eps_s"] * E0
    beta2 = Q * Q * c["Nd"] / (es * KB * c["T"])  # Debye screening, n = Nd
    E = E_eV * Q
    k = b.k_of_E(E)
    want = c["Nd"] * golden_rule(k, k, b.dk_dE(E), lambda q2: (Q * Q / es) ** 2 / (q2 + beta2) ** 2)
    assert s.rate(0, 0, E_eV) == pytest.approx(want, rel=1e-7)


@pytest.mark.parametrize("E_eV", [0.01, 0.1, 1.0, 3.0])
@pytest.mark.parametrize("v", [0, 1, 2])
def test_acoustic_rate_golden_rule(oracle_mod, v, E_eV):
    c = cfg(T=350.0)
    s = oracle_mod.Sim(c)
    b = Band(c["m_rel"][v], c["alpha_per_eV"][v])
    Da = c["Da_eV"] * Q
    # |M|^2 V = Da^2 kT / (rho vs^2) (equipartition, elastic)
    want = 2 * math.pi / HB * Da * Da * KB * c["T"] / (c["rho_kg_m3"] * c["vs_m_s"] ** 2) * b.dos(E_eV * Q)
    assert s.rate(v, 3, E_eV) == pytest.approx(want, rel=1e-7)


@pytest.mark.parametrize("E_eV", [0.05, 1.0, 2.0, 2.3, 3.5])
def test_intervalley_rate_golden_rule(oracle_mod, E_eV):
    c = cfg(T=500.0)
    s = oracle_mod.Sim(c)
    hw = c["hw_iv_eV"] * Q
    w = hw / HB
    Niv = occupations(c["T"], c["hw_iv_eV"])
    D = c["Dij_eV_per_m"] * Q
    E = E_eV * Q
    for i in range(3):
        for j in range(3):
            bj = Band(c["m_rel"][j], c["alpha_per_eV"][j])
            Zf = c["Z"][j] - (1 if i == j else 0)
            dEc = (c["Ec_eV"][j] - c["Ec_eV"][i]) * Q
            for absorb in (1, 0):
                mech = 4 + 2 * j + (0 if absorb else 1)
                Ef = E + (hw if absorb else -hw) - dEc
                got = s.rate(i, mech, E_eV)
                if Ef <= 0 or Zf <= 0:
                    assert got == 0.0
                    continue
                occ = Niv if absorb else Niv + 1
                # |M|^2 V = hbar D^2 / (2 rho w) (N + 1/2 -+ 1/2), Zf final valleys
                want = 2 * math.pi / HB * HB * D * D / (2 * c["rho_kg_m3"] * w) * occ * Zf * bj.dos(Ef)
                assert got == pytest.approx(want, rel=1e-7), (i, j, absorb)


@pytest.mark.parametrize("E_eV", [0.0137, 0.2, 1.1, 2.6])
def test_detailed_balance(oracle_mod, E_eV):
    """Z_i g_i(E) W_abs(i->j, E) / N = Z_j g_j(E') W_em(j->i, E') / (N + 1)."""
    c = cfg(T=450.0)
    s = oracle_mod.Sim(c)
    E = E_eV * Q
    # polar optical, within one valley
    for v in range(3):
        b = Band(c["m_rel"][v], c["alpha_per_eV"][v])
        hw = c["hw_lo_eV"] * Q
        N0 = occupations(c["T"], c["hw_lo_eV"])
        lhs = b.dos(E) * s.rate(v, 1, E_eV) / N0
        rhs = b.dos(E + hw) * s.rate(v, 2, (E + hw) / Q) / (N0 + 1)
        assert lhs == pytest.approx(rhs, rel=1e-7)
    # intervalley between every pair
    hw = c["hw_iv_eV"] * Q
    Niv = occupations(c["T"], c["hw_iv_eV"])
    for i in range(3):
        for j in range(3):
            Ef = E + hw - (c["Ec_eV"][j] - c["Ec_eV"][i]) * Q
            if Ef <= 0:
                continue
            bi = Band(c["m_rel"][i], c["alpha_per_eV"][i])
            bj = Band(c["m_rel"][j], c["alpha_per_eV"][j])
            lhs = c["Z"][i] * bi.dos(E) * s.rate(i, 4 + 2 * j, E_eV) / Niv
            rhs = c["Z"][j] * bj.dos(Ef) * s.rate(j, 5 + 2 * i, Ef / Q) / (Niv + 1)
            if lhs == 0.0:
                assert rhs == 0.0
            else:
                assert lhs == pytest.approx(rhs, rel=1e-7), (i, j)


def test_mechanism_mask_and_parabolic_limit(oracle_mod):
    c = cfg(mech_mask=1 << 3, alpha_per_eV=(0.0, 0.0, 0.0))
    s = oracle_mod.Sim(c)
    for m in range(10):
        if m != 3:
            assert s.rate(0, m, 0.3) == 0.0
    # parabolic acoustic rate grows as sqrt(E)
    assert s.rate(0, 3, 0.4) / s.rate(0, 3, 0.1) == pytest.approx(2.0, rel=1e-12)


def test_tables_cumulative_and_gamma0(oracle_mod):
    c = cfg(n_bins=512)
    s = oracle_mod.Sim(c)
    t, g = s.tables()
    assert np.all(np.diff(t, axis=2) >= 0)
    assert np.all(t >= 0)
    # Gamma0 is the maximum total over the table: the largest normalised total is exactly 1
    for v in range(3):
        assert t[v, :, -1].max() == 1.0
        b = 100
        E = b * c["dE_eV"]
        tot = sum(s.rate(v, m, E) for m in range(10))
        assert t[v, b, -1] * g[v] == pytest.approx(tot, rel=1e-13)


# ------------------------------------------------------------ samplers
@pytest.mark.parametrize("k,kp", [(1e9, 1.3e9), (2e9, 1.7e9), (3e8, 9e8), (5e9, 4.9e9)])
def test_pop_angle_inverse_cdf(oracle_mod, k, kp):
    f = lambda c: 1.0 / (k * k + kp * kp - 2 * k * kp * c)
    tot = integrate.quad(f, -1, 1, epsabs=0, epsrel=1e-13, limit=200)[0]
    for u in (0.01, 0.2, 0.5, 0.77, 0.99):
        c = oracle_mod.cos_pop(k, kp, u)
        assert -1 <= c <= 1
        tail = integrate.quad(f, c, 1, epsabs=0, epsrel=1e-13, limit=200)[0] / tot
        assert tail == pytest.approx(u, rel=1e-8, abs=1e-10)


@pytest.mark.parametrize("k,beta2", [(1e9, 7.9e16), (2e8, 7.9e16), (3e9, 1e15)])
def test_impurity_angle_inverse_cdf(oracle_mod, k, beta2):
    f = lambda c: 1.0 / (2 * k * k * (1 - c) + beta2) ** 2
    tot = integrate.quad(f, -1, 1, epsabs=0, epsrel=1e-13, limit=400)[0]
    for u in (0.01, 0.3, 0.5, 0.9, 0.999):
        c = oracle_mod.cos_imp(k, beta2, u)
        assert -1 <= c <= 1
        tail = integrate.quad(f, c, 1, epsabs=0, epsrel=1e-13, limit=400)[0] / tot
        assert tail == pytest.approx(u, rel=1e-8, abs=1e-10)


def test_rotation_frame(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ct = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * np.pi)
        out = oracle_mod.rotate(n, ct, ph)
        assert np.linalg.norm(out) == pytest.approx(1.0, abs=1e-12)
        assert out @ n == pytest.approx(ct, abs=1e-12)
    # azimuth advances the right-handed way about n and covers the cone uniformly
    n = np.array([0.0, 0.0, 1.0])
    a = oracle_mod.rotate(n, 0.0, 0.0)
    b = oracle_mod.rotate(n, 0.0, np.pi / 2)
    assert np.cross(a, b) @ n == pytest.approx(1.0, abs=1e-12)
    nz = np.array([0.0, 0.0, -1.0])  # the basis must also hold on the negative pole
    assert oracle_mod.rotate(nz, 0.3, 1.0) @ nz == pytest.approx(0.3, abs=1e-12)


def test_initial_energy_is_kane_maxwellian(oracle_mod):
    """Mean of the initial draw vs quadrature of g(E) exp(-E/kT),
    g ~ sqrt(E(1+aE))(1+2aE); the parabolic 1.5 kT lies 1.2% away."""
    c = W.bulk(n_particles=400_000, T=300.0)
    s = oracle_mod.Sim(c)
    E = s.initial_energies(400_000)
    kT = KB * c["T"]
    a = c["alpha_per_eV"][0] / Q
    g = lambda e: math.sqrt(e * (1 + a * e)) * (1 + 2 * a * e) * math.exp(-e / kT)
    num = integrate.quad(lambda e: e * g(e), 0, 60 * kT, epsabs=0, epsrel=1e-12)[0]
    den = integrate.quad(g, 0, 60 * kT, epsabs=0, epsrel=1e-12)[0]
    want = num / den
    # the Kane-Maxwellian mean at 300 K with the Gamma1 nonparabolicity of
    # Table I is 1.5182 kT (above the parabolic 1.5 kT)
    assert want / kT == pytest.approx(1.5182, abs=2e-4)
    sem = E.std() / math.sqrt(E.size)
    assert abs(E.mean() - want) < 4 * sem
    assert abs(E.mean() / kT - 1.5) > 6 * sem / kT
