"""Pins of oracle parts that no other test fixes from outside the oracle:

- the nanowire position update of a free flight (reading R7), against the
  exact integral of the Kane group velocity along the flight;
- the walls (reading R8): plane A always specular; the other walls specular
  with probability p, else a cosine-weighted inward direction with |k| kept;
  contacts absorb;
- the scattering dynamics in equilibrium: the velocity autocorrelation of an
  elastic ensemble against the textbook momentum relaxation times
  (deformation-potential acoustic and Brooks-Herring impurity scattering), and
  the acoustic-only parabolic mobility 4 e tau0 / (3 sqrt(pi) m);
- the low-field drift velocity of the full physics (Table I, all
  mechanisms) against mu E with mu = e D / kT, D from the zero-field velocity
  autocorrelation (the Einstein relation of linear response).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W

# CODATA 2018 (the values the oracle states; newer tables differ in the tenth
# digit of hbar and m_e)
Q, HB, KB, M0, EPS0 = 1.602176634e-19, 1.054571817e-34, 1.380649e-23, 9.1093837015e-31, 8.8541878128e-12


def threads():
    from oracle import oracle
    return min(8, oracle.host_cores())


# ------------------------------------------------------------ free flight
def kane_v(k, m, a):
    """Group velocity hbar k / (m (1 + 2 a E)) of the Kane band, E from
    E (1 + a E) = hbar^2 k^2 / 2m (a in 1/J)."""
    g = HB ** 2 * np.dot(k, k) / (2 * m)
    E = g if a == 0 else (-1 + math.sqrt(1 + 4 * a * g)) / (2 * a)
    return HB * np.asarray(k) / (m * (1 + 2 * a * E)), E


def test_free_flight_parabolic_is_the_exact_parabola(oracle_mod):
    """alpha = 0 (Gamma3 valley): k(t) = k0 - qFt/hbar and
    r(t) = r0 + v0 t - qF t^2 / 2m, exactly (to rounding)."""
    s = oracle_mod.Sim(W.nanowire(n_particles=1, nx=4, Lx=40e-9))
    rng = np.random.default_rng(1)
    m = 0.40 * M0
    for _ in range(20):
        k0 = rng.normal(size=3) * 8e8
        r0 = rng.uniform(0, 1, 3) * 40e-9
        F = rng.normal(size=3) * 3e7
        t = rng.uniform(1e-16, 2e-15)
        k1, r1 = s.test_drift(2, k0, r0, F, t)
        np.testing.assert_allclose(k1, k0 - Q * F * t / HB, rtol=1e-13, atol=1e-13 * np.abs(k0).max())
        want = r0 + HB * k0 / m * t - Q * F * t * t / (2 * m)
        np.testing.assert_allclose(r1 - r0, want - r0, rtol=1e-10, atol=1e-12 * np.abs(want - r0).max())


def test_free_flight_nonparabolic_against_velocity_integral(oracle_mod):
    """alpha = 0.19/eV (Gamma1): the displacement along the force equals the
    exact integral of the group velocity (energy conservation), and across
    it the trapezoid of the start and end velocities errs by at most
    t^3/12 max|v''| -- third order in t (halving t divides the error by 8)."""
    s = oracle_mod.Sim(W.nanowire(n_particles=1, nx=4, Lx=40e-9))
    m, a = 0.21 * M0, 0.19 / Q
    rng = np.random.default_rng(2)
    for trial in range(8):
        k0 = rng.normal(size=3) * 1e9
        F = rng.normal(size=3) * 2e7
        Fh = F / np.linalg.norm(F)
        errs = []
        for t in (4e-15, 2e-15, 4e-14, 1e-15):
            r0 = np.zeros(3)
            _, r1 = s.test_drift(0, k0, r0, F, t)
            ex = np.array([integrate.quad(lambda u, i=i: kane_v(k0 - Q * F * u / HB, m, a)[0][i], 0, t,
                                          epsabs=0, epsrel=1e-13)[0] for i in range(3)])
            par = np.dot(r1, Fh)
            assert par == pytest.approx(np.dot(ex, Fh), rel=1e-9, abs=1e-9 * np.linalg.norm(ex)), (trial, t)
            perp = (r1 - par * Fh) - (ex - np.dot(ex, Fh) * Fh)
            # bound of the trapezoid error from the second derivative of v
            us = np.linspace(0, t, 201)
            vs = np.array([kane_v(k0 - Q * F * u / HB, m, a)[0] for u in us])
            vp = vs - np.outer(vs @ Fh, Fh)
            d2 = np.abs(np.diff(vp, 2, axis=0)).max() / (us[1] - us[0]) ** 2
            bound = t ** 3 / 12 * d2
            assert np.linalg.norm(perp) <= 1.05 * bound * math.sqrt(3) + 1e-12 * np.linalg.norm(ex), (trial, t)
            errs.append(np.linalg.norm(perp))
        assert 6.0 < errs[0] / errs[1] < 10.0, (trial, errs)  # third order once the flight is short


# ------------------------------------------------------------------ walls
def wall_cfg(p):
    return W.nanowire(n_particles=1, nx=4, Lx=40e-9, p_specular=p, seed=77)


def test_contacts_absorb_and_plane_a_reflects(oracle_mod):
    c = wall_cfg(0.5)
    s = oracle_mod.Sim(c)
    k = np.array([3e8, -2e8, 1e8])
    out, _, _, ctr = s.test_walls([-1e-10, 10e-9, 50e-9], k, 5)
    assert out and ctr == 5
    out, _, _, ctr = s.test_walls([c["Lx"] + 1e-10, 10e-9, 50e-9], k, 5)
    assert out and ctr == 5
    # plane A (y < 0): mirror position and k_y, no random draw
    out, r1, k1, ctr = s.test_walls([20e-9, -3e-9, 50e-9], k, 9)
    assert not out and ctr == 9
    np.testing.assert_array_equal(k1, [k[0], -k[1], k[2]])
    assert r1[1] == pytest.approx(3e-9, rel=1e-12)


@pytest.mark.parametrize("wall", ["side", "bottom", "top"])
def test_wall_specular_fraction_and_cosine_law(oracle_mod, wall):
    """Specular with probability p = 0.5; a diffuse reflection keeps |k|,
    points inward, has a cosine-weighted polar angle about the inward normal
    (P(cos theta <= c) = c^2: <cos> = 2/3, <cos^2> = 1/2) and a uniform
    azimuth."""
    p = 0.5
    c = wall_cfg(p)
    s = oracle_mod.Sim(c)
    n = 40_000
    if wall == "side":
        r0, ax, inward = [20e-9, c["Ly"] + 2e-9, 50e-9], 1, -1.0
    elif wall == "bottom":
        r0, ax, inward = [20e-9, 30e-9, -2e-9], 2, 1.0
    else:
        r0, ax, inward = [20e-9, 30e-9, c["Lz"] + 2e-9], 2, -1.0
    plane = c["Ly"] if wall == "side" else (0.0 if wall == "bottom" else c["Lz"])
    t1, t2 = [j for j in range(3) if j != ax]
    rng = np.random.default_rng(5)
    ks = rng.normal(size=(n, 3)) * 5e8
    ks[:, ax] = -inward * np.abs(ks[:, ax])  # heading out through the wall
    spec, cos_d, phi_d = 0, [], []
    for i in range(n):
        k = ks[i]
        out, r1, k1, ctr = s.test_walls(r0, k, 1000 + 3 * i)
        assert not out and ctr == 1000 + 3 * i + 1
        assert abs(r1[ax] - (2 * plane - r0[ax])) <= 1e-12 * c["Lz"]
        if k1[ax] == -k[ax] and k1[t1] == k[t1] and k1[t2] == k[t2]:
            spec += 1
            continue
        km = math.sqrt(k @ k)
        assert abs(math.sqrt(k1 @ k1) - km) <= 1e-13 * km
        ct = inward * k1[ax] / km
        assert ct > 0
        cos_d.append(ct)
        phi_d.append(math.atan2(k1[t2], k1[t1]))
    frac = spec / n
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n), frac
    cd = np.array(cos_d)
    nd = cd.size
    assert cd.mean() == pytest.approx(2 / 3, abs=4 * math.sqrt(1 / 2 - 4 / 9) / math.sqrt(nd))
    assert (cd ** 2).mean() == pytest.approx(1 / 2, abs=4 * math.sqrt(1 / 3 - 1 / 4) / math.sqrt(nd))
    # Kolmogorov-Smirnov distance to the CDF c^2 (99.9% critical value)
    xs = np.sort(cd)
    ecdf = np.arange(1, nd + 1) / nd
    assert np.abs(ecdf - xs ** 2).max() < 1.95 / math.sqrt(nd)
    ph = np.array(phi_d)
    assert abs(np.cos(ph).mean()) < 4 / math.sqrt(2 * nd) and abs(np.sin(ph).mean()) < 4 / math.sqrt(2 * nd)


# ------------------------------------- equilibrium velocity autocorrelation
def velocities(c, p):
    """Group velocities of the oracle's particles (Kane band of each valley)."""
    v = p["valley"]
    m = np.array(c["m_rel"])[v] * M0
    a = np.array(c["alpha_per_eV"])[v] / Q
    g = HB ** 2 * (p["k"] ** 2).sum(1) / (2 * m)
    E = 2 * g / (1 + np.sqrt(1 + 4 * a * g))
    return HB * p["k"] / (m * (1 + 2 * a * E))[:, None]


def measure_vacf(oracle_mod, c, lags_fs):
    """C(s) = <v(0) . v(s)> / 3 of a zero-field ensemble in equilibrium, with
    the standard error of each lag."""
    s = oracle_mod.Sim(c, threads=threads())
    s.run(20)
    v0 = velocities(c, s.particles())
    out, t = [], 0
    for lag in lags_fs:
        s.run(lag - t)
        t = lag
        prod = (v0 * velocities(c, s.particles())).sum(1) / 3
        out.append((prod.mean(), prod.std() / math.sqrt(prod.size)))
    return np.array(out)


def acoustic_rate(c, E, m, a):
    """Deformation-potential acoustic scattering, elastic equipartition:
    1/tau = pi D^2 kT g(E) / (hbar rho v_s^2), g the Kane density of states
    (both spins) (2m)^{3/2} sqrt(E(1+aE)) (1+2aE) / (2 pi^2 hbar^3)."""
    g = (2 * m) ** 1.5 * np.sqrt(E * (1 + a * E)) * (1 + 2 * a * E) / (2 * math.pi ** 2 * HB ** 3)
    D = c["Da_eV"] * Q
    return math.pi * D ** 2 * KB * c["T"] * g / (HB * c["rho_kg_m3"] * c["vs_m_s"] ** 2)


def brooks_herring_momentum_rate(c, E, m):
    """Brooks-Herring momentum relaxation rate (parabolic band):
    N_I e^4 / (16 pi sqrt(2m) eps^2 E^{3/2}) [ln(1+b) - b/(1+b)],
    b = 8 m E / (hbar^2 beta^2), Debye beta^2 = e^2 N / (eps kT)."""
    eps = c["eps_s"] * EPS0
    N = c["Nd"]
    beta2 = Q * Q * N / (eps * KB * c["T"])
    b = 8 * m * E / (HB ** 2 * beta2)
    return N * Q ** 4 / (16 * math.pi * math.sqrt(2 * m) * eps ** 2 * E ** 1.5) * (np.log1p(b) - b / (1 + b))


def vacf_theory(c, rate_m, lags_s, alpha_eV=0.0):
    """<v_z(0) v_z(s)> = <v^2/3 exp(-s / tau_m(E))> over the Kane-Maxwellian
    of valley 0: elastic scattering with an isotropic band keeps the energy,
    and the mean velocity at energy E decays at the momentum relaxation rate."""
    m = c["m_rel"][0] * M0
    a = alpha_eV / Q
    kT = KB * c["T"]

    def w(E):
        return math.sqrt(E * (1 + a * E)) * (1 + 2 * a * E) * math.exp(-E / kT)

    def v2(E):
        return 2 * E * (1 + a * E) / (m * (1 + 2 * a * E) ** 2)

    top = 40 * kT
    Z = integrate.quad(w, 0, top, epsabs=0, epsrel=1e-12, limit=200)[0]
    out = []
    for s in lags_s:
        f = lambda E: w(E) * v2(E) / 3 * math.exp(-s * rate_m(E))
        out.append(integrate.quad(f, 0, top, epsabs=0, epsrel=1e-11, limit=400, points=[kT, 5 * kT])[0] / Z)
    return np.array(out)


def mobility_theory(c, rate_m):
    """mu = e/(kT) int_0^inf C(s) ds = e <v^2/3 tau_m> / kT (parabolic)."""
    m = c["m_rel"][0] * M0
    kT = KB * c["T"]
    w = lambda E: math.sqrt(E) * math.exp(-E / kT)
    f = lambda E: w(E) * (2 * E / m) / 3 / rate_m(E)
    top = 60 * kT
    return Q / kT * integrate.quad(f, 0, top, epsabs=0, epsrel=1e-12, limit=400)[0] / \
        integrate.quad(w, 0, top, epsabs=0, epsrel=1e-12, limit=400)[0]


def test_acoustic_only_mobility_closed_form():
    """The quadrature above reproduces mu = 4 e tau0 / (3 sqrt(pi) m) for
    acoustic scattering in a parabolic band, tau0 = 1/W(kT)."""
    c = W.bulk(n_particles=1)
    m = c["m_rel"][0] * M0
    kT = KB * c["T"]
    tau0 = 1.0 / acoustic_rate(c, kT, m, 0.0)
    want = 4 * Q * tau0 / (3 * math.sqrt(math.pi) * m)
    got = mobility_theory(c, lambda E: acoustic_rate(c, E, m, 0.0))
    assert got == pytest.approx(want, rel=1e-8)


@pytest.mark.parametrize("case", ["acoustic_parabolic", "acoustic_kane", "acoustic_impurity"])
def test_equilibrium_vacf_matches_momentum_relaxation(oracle_mod, case):
    """Zero field, elastic mechanisms only, exact rates: the oracle's velocity
    autocorrelation at lags up to 2 ps equals the relaxation-time integral
    (4 standard errors per lag).  Pins the rates' energy dependence, the
    Brooks-Herring angle law and rotation (through the momentum relaxation
    rate), and the group velocity."""
    alpha = 0.19 if case == "acoustic_kane" else 0.0
    mask = (1 << 3) | (1 if case == "acoustic_impurity" else 0)
    c = W.bulk(n_particles=100_000, field_V_m=0.0, mech_mask=mask, exact_rates=1,
               alpha_per_eV=(alpha, 0.1, 0.0), seed=31)
    m, a = c["m_rel"][0] * M0, alpha / Q
    if case == "acoustic_impurity":
        rate = lambda E: acoustic_rate(c, E, m, 0.0) + brooks_herring_momentum_rate(c, E, m)
    else:
        rate = lambda E: acoustic_rate(c, E, m, a)
    lags = [0, 50, 100, 200, 400, 800, 1600]
    got = measure_vacf(oracle_mod, c, lags)
    want = vacf_theory(c, rate, [1e-15 * l for l in lags], alpha_eV=alpha)
    if alpha == 0.0:
        assert want[0] == pytest.approx(KB * c["T"] / m, rel=1e-9)  # equipartition
    for (g, se), w_, lag in zip(got, want, lags):
        assert abs(g - w_) < 4 * se + 1e-3 * want[0], (case, lag, g, w_, se)


def test_einstein_relation_low_field_drift(oracle_mod):
    """Full physics (Table I, all mechanisms, exact rates), 300 K, 1e17 cm^-3:
    the drift velocity at 0.5 kV/cm equals mu E with mu = e D / kT, D the
    time integral of the zero-field velocity autocorrelation.  The drift is
    measured with antithetic fields +-E on the same random streams (their
    half difference is the odd, linear part); the allowance adds 1% for the
    warm-electron decrease of the mobility at 0.5 kV/cm (measured: mu falls
    by 2.7% at 1 kV/cm and 11% at 2 kV/cm, quadratically in E)."""
    th = threads()
    c0 = W.bulk(n_particles=100_000, field_V_m=0.0, exact_rates=1, seed=3)
    s = oracle_mod.Sim(c0, threads=th)
    s.run(100)
    v0 = velocities(c0, s.particles())
    ts, prods, t = [0.0], [(v0 * v0).sum(1) / 3], 0
    while t < 1500:
        st = 5 if t < 300 else 25
        s.run(st)
        t += st
        ts.append(t * 1e-15)
        prods.append((v0 * velocities(c0, s.particles())).sum(1) / 3)
    P, ts = np.array(prods), np.array(ts)
    groups = 20
    Dg = np.array([np.trapezoid(P[:, g::groups].mean(1), ts) for g in range(groups)])
    D = np.trapezoid(P.mean(1), ts)
    mu_gk, se_gk = Q * D / (KB * c0["T"]), Q * Dg.std(ddof=1) / math.sqrt(groups) / (KB * c0["T"])
    # drift: the odd part of +-E runs per block of 250 fs (blocks are much
    # longer than the ~0.1 ps momentum relaxation, so nearly independent)
    F, blk, nblk = 5e4, 250, 10
    mus = []
    for seed in (41, 42):
        sims = [oracle_mod.Sim(W.bulk(n_particles=32_000, field_V_m=sgn * F, exact_rates=1, seed=seed), threads=th)
                for sgn in (1, -1)]
        prev = []
        for sim in sims:
            sim.run(500)
            prev.append(sim.tallies())
        for _ in range(nblk):
            v = []
            for i, sim in enumerate(sims):
                sim.run(blk)
                cur = sim.tallies()
                v.append((cur["sum_v"][2] - prev[i]["sum_v"][2]) / (cur["n_samples"] - prev[i]["n_samples"]))
                prev[i] = cur
            mus.append(-(v[0] - v[1]) / 2 / F)
    mus = np.array(mus)
    mu_d, se_d = float(mus.mean()), float(mus.std(ddof=1) / math.sqrt(mus.size))
    assert abs(mu_d - mu_gk) <= 3 * math.hypot(se_gk, se_d) + 0.01 * mu_gk, (mu_d, mu_gk, se_gk, se_d)
    assert 0.08 < mu_gk < 0.13  # 800..1300 cm^2/Vs
