"""The surrogate trained on Monte Carlo data generated by this library:
accuracy on held-out Monte Carlo samples, and independence of the field
angle (the band model is isotropic)."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained(emc):
    from paper_1707_09073_gb300 import surrogate as S
    base = W.bulk()
    X = S.sample_inputs(3072, seed=1)
    t0 = time.perf_counter()
    Y = S.mc_observables(X, base, n_electrons=2000, warm_steps=800, avg_steps=800, batch=1024, seed0=1)
    t_mc = time.perf_counter() - t0
    sur = S.Surrogate(X, Y, seed=2)
    hist = sur.fit(X, Y, steps=3000, batch=1024, lr=2e-3, seed=3)
    Xt = S.sample_inputs(256, seed=9)
    Yt = S.mc_observables(Xt, base, n_electrons=4000, warm_steps=800, avg_steps=800, batch=256, seed0=100000)
    return S, sur, X, Y, Xt, Yt, hist, t_mc


def test_surrogate_fits_held_out_monte_carlo(trained):
    S, sur, X, Y, Xt, Yt, hist, t_mc = trained
    assert hist[-200:].mean() < 0.2 * hist[:20].mean()
    P = sur.predict(Xt)
    for j, name in enumerate(S.OUT_NAMES):
        if name in ("f_U", "f_Gamma3"):
            continue  # tiny occupations at these fields
        r2 = 1 - np.mean((P[:, j] - Yt[:, j]) ** 2) / np.var(Yt[:, j])
        assert r2 > 0.9, (name, r2)


def test_surrogate_ignores_field_angle(trained):
    S, sur, X, Y, Xt, Yt, hist, t_mc = trained
    Xa = Xt.copy()
    Xb = Xt.copy()
    Xa[:, 1] = 0.3
    Xb[:, 1] = 2.6
    Pa, Pb = sur.predict(Xa), sur.predict(Xb)
    j = S.OUT_NAMES.index("v_drift_m_s")
    assert np.sqrt(np.mean((Pa[:, j] - Pb[:, j]) ** 2)) < 0.1 * np.std(Yt[:, j])
