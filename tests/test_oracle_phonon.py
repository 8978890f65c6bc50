"""Pins of the phonon Monte Carlo oracle (oracle/phonon_oracle.c,
oracle/phonon.py) against what the mathematics fixes: the generator's
published known answers, the cosine law of diffuse re-emission, the binned
spectrum against the continuous kinetic integral (itself pinned at Table II)
and the classical heat capacity, the ballistic limit (solid angles and mean
flight times of a box), and the diffusive limit (Fourier's law with the
conductivity of the same spectrum and the Milne extrapolation length)."""
import os

import numpy as np
import pytest
from scipy import constants as sc

import workloads as W
from oracle import phonon as PH
from oracle import thermal as TH

HERE = os.path.dirname(__file__)
GAN = W.TABLE_II_GAN
# the Table II dispersion with the scattering of the relaxation-time model
# switched off: only the boundary term v / L_b scatters
GAN_FREE = dict(GAN, A_s3=0.0, B1_s_per_K=0.0)


def test_philox_known_answers():
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r[:6]]
        want = [int(x, 16) for x in r[6:10]]
        assert PH.philox(v[:4], v[4:6]) == want


def test_uniforms_are_odd_multiples_of_2_pow_minus_24():
    u = PH.draws(7, 3, 0, 500)
    m = u * 2 ** 24
    assert np.all(m == np.round(m)) and np.all(np.round(m) % 2 == 1)
    assert 0 < u.min() and u.max() < 1
    # counter n of bundle 3 is the same as starting at n
    assert np.array_equal(PH.draws(7, 3, 10, 5), u[10:15])


@pytest.mark.parametrize("face", range(6))
def test_diffuse_reemission_follows_the_cosine_law(face):
    """Lambert's law about the inward normal: <cos> = 2/3, <cos^2> = 1/2,
    tangential components average to zero, unit length."""
    g = (np.arange(200) + 0.5) / 200
    U1, U2 = np.meshgrid(g, g, indexing="ij")
    d = np.array([PH.lambert(face, a, b) for a, b in zip(U1.ravel(), U2.ravel())])
    ax, sign = face // 2, (1.0 if face % 2 == 0 else -1.0)
    c = sign * d[:, ax]
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    assert c.min() > 0
    assert abs(c.mean() - 2 / 3) < 1e-4 and abs((c ** 2).mean() - 0.5) < 1e-4
    for t in range(3):
        if t != ax:
            assert abs(d[:, t].mean()) < 1e-12


def test_binned_spectrum_against_the_kinetic_integral():
    """(1/3) sum C_b v_b^2 tau_b of 4000 wave-vector bins against the
    quadrature of oracle/thermal.kappa (228 W/m/K at 300 K, Table II), with
    and without the boundary term; midpoint bins converge as 1/nb^2."""
    for T, Lb in ((300.0, 0.0), (300.0, 120e-9), (450.0, 120e-9)):
        want = TH.kappa(T, GAN, Lb)
        got = PH.kappa_binned(GAN, 4000, T, Lb)
        assert abs(got / want - 1) < 2e-4, (T, Lb, got, want)


def test_binned_heat_capacity_classical_limit():
    """At T >> hbar omega_max / k every mode holds k: three branches of
    q0^3 / (6 pi^2) modes per unit volume."""
    q0 = GAN["k0_per_m"]
    want = 3 * sc.k * q0 ** 3 / (6 * np.pi ** 2)
    got = PH.heat_capacity(GAN, 2000, 1e6).sum()
    assert abs(got / want - 1) < 1e-4


def _solid_angle_rect(a, b, d):
    """Solid angle of an a x b rectangle seen from a point at height d above
    one of its corners."""
    return np.arctan(a * b / (d * np.sqrt(a * a + b * b + d * d)))


def _face_fraction(p, L, ax, high):
    """Fraction of isotropic directions from p that leave the box [0,L]^3
    through the face normal to axis ax (high: the face at L)."""
    t = [a for a in range(3) if a != ax]
    d = (L - p[ax]) if high else p[ax]
    om = 0.0
    for lo_u, hi_u in ((0.0, p[t[0]]), (p[t[0]], L)):
        for lo_v, hi_v in ((0.0, p[t[1]]), (p[t[1]], L)):
            om += _solid_angle_rect(hi_u - lo_u, hi_v - lo_v, d)
    return om / (4 * np.pi)


def _mean_exit_distance(p, L, n=20000):
    """Mean distance from p to the surface of the box [0,L]^3 over isotropic
    directions (a Fibonacci sphere of n directions)."""
    i = np.arange(n) + 0.5
    ct = 1 - 2 * i / n
    ph = np.pi * (1 + 5 ** 0.5) * i
    st = np.sqrt(1 - ct * ct)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    with np.errstate(divide="ignore"):
        t = np.where(d > 0, (L - p) / d, np.where(d < 0, -p / d, np.inf))
    return t.min(axis=1).mean()


def test_ballistic_box_solid_angles_and_flight_times():
    """No scattering (mean free path 1 km) in a 1 um cube with absorbing
    faces, heat in one subcell: each face takes the solid-angle share seen
    from the subcell, and the time spent is the mean distance to the surface
    times <1/v> of the emission spectrum (proportional to C_b v_b)."""
    n, Lm = 16, 1e-6
    grid = dict(nx=n, ny=n, nz=n, Lx=Lm, Ly=Lm, Lz=Lm)
    src = (2, 9, 7)
    q = np.zeros(n ** 3)
    q[(src[0] * n + src[1]) * n + src[2]] = 1e18
    N = 200_000
    r = PH.solve(grid, q, GAN_FREE, [PH.ISOTHERMAL] * 6, N, seed=3, nb=200, L_b=1e3)
    assert r["capped"] == 0 and int(r["absorbed"].sum()) == N
    assert int(r["scatterings"].sum()) < 5
    h = Lm / n
    g = (np.arange(4) + 0.5) / 4
    pts = [np.array([(src[0] + a) * h, (src[1] + b) * h, (src[2] + c) * h]) for a in g for b in g for c in g]
    for f in range(6):
        want = np.mean([_face_fraction(p, Lm, f // 2, f % 2 == 1) for p in pts])
        got = r["absorbed"][f] / N
        assert abs(got - want) < 4 * np.sqrt(want * (1 - want) / N) + 2e-3, (f, got, want)
    _, _, v, _ = PH.bins(GAN_FREE, 200)
    cb = PH.heat_capacity(GAN_FREE, 200, 300.0)
    inv_v = (cb * v * (1 / v)).sum() / (cb * v).sum()
    want_t = np.mean([_mean_exit_distance(p, Lm) for p in pts]) * inv_v
    got_t = r["t_res_ps"].sum() * 1e-12 / N
    assert abs(got_t / want_t - 1) < 0.01, (got_t, want_t)


def test_diffusive_slab_follows_fouriers_law():
    """A 200 nm slab between isothermal faces (the other faces specular: an
    infinite slab), heat uniform, mean free path 2 nm at every frequency:
    the temperature rise is Fourier's q (x + d)(L + d - x) / (2 kappa) with
    kappa = (1/3) sum C_b v_b^2 tau_b and the Milne extrapolation length
    d = 0.7104 lambda of isotropic scattering."""
    L, lam, n = 200e-9, 2e-9, 40
    grid = dict(nx=n, ny=1, nz=1, Lx=L, Ly=10e-9, Lz=10e-9)
    qv = 1e18
    faces = [PH.ISOTHERMAL, PH.ISOTHERMAL] + [PH.SPECULAR] * 4
    r = PH.solve(grid, np.full(n, qv), GAN_FREE, faces, 20_000, seed=11, nb=100, L_b=lam, threads=4)
    assert r["capped"] == 0 and int(r["absorbed"].sum()) == 20_000
    kap = PH.kappa_binned(GAN_FREE, 100, 300.0, lam)
    x = (np.arange(n) + 0.5) * L / n
    dlt = 0.7104 * lam
    want = qv * (x + dlt) * (L + dlt - x) / (2 * kap)
    got = r["dT"]
    mid = slice(n // 4, 3 * n // 4)
    assert np.abs(got[mid] / want[mid] - 1).max() < 0.03, (got[mid] / want[mid])
    assert abs(got[mid].mean() / want[mid].mean() - 1) < 0.01
    # the conductivity matters: a third off would show
    assert abs(got[mid].mean() / (want[mid].mean() * 1.33) - 1) > 0.2


def test_negative_heat_is_a_phonon_deficit():
    """Bundles carry the sign of their subcell's heat: reversing every sign
    reverses the temperature rise exactly (the same bundles, the same
    paths), and a mixed-sign source is the difference of its parts within
    the Monte Carlo noise."""
    n = 10
    grid = dict(nx=n, ny=2, nz=2, Lx=200e-9, Ly=40e-9, Lz=40e-9)
    faces = [PH.ISOTHERMAL, PH.ISOTHERMAL, PH.SPECULAR, PH.ROUGH, PH.SPECULAR, PH.ROUGH]
    rng = np.random.default_rng(2)
    q = rng.uniform(0.5, 1.5, n * 4) * 1e18
    q[:8] *= -1.0
    a = PH.solve(grid, q, GAN, faces, 4000, seed=5, nb=200, p_specular=[0.5] * 6)
    b = PH.solve(grid, -q, GAN, faces, 4000, seed=5, nb=200, p_specular=[0.5] * 6)
    assert np.array_equal(a["dT"], -b["dT"]) and np.array_equal(a["scatterings"], b["scatterings"])
    # superposition, in the diffusive regime (mean free path 10 nm) where a
    # bundle's time is not dominated by rare long flights; x-slab means
    pos, neg = np.where(q > 0, q, 0.0), np.where(q < 0, -q, 0.0)
    N = 60_000
    kw = dict(nb=200, p_specular=[0.5] * 6, L_b=10e-9, threads=4)
    slab = lambda r: r["dT"].reshape(n, 4).mean(axis=1)
    m = slab(PH.solve(grid, q, GAN_FREE, faces, N, seed=6, **kw))
    p = slab(PH.solve(grid, pos, GAN_FREE, faces, N, seed=7, **kw))
    g = slab(PH.solve(grid, neg, GAN_FREE, faces, N, seed=8, **kw))
    scale = np.abs(p).max()
    assert np.abs(m - (p - g)).max() < 0.03 * scale, (m, p - g, scale)
    assert np.all(m[:2] < p[:2] - 0.05 * scale)  # the deficit shows near the source
