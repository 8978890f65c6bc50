"""The coupled electrothermal iteration of the hybrid method and its
surrogate-corrected variant.

Plain iteration (the hybrid method's coupled loop, repeated until the
temperature field is steady): from a steady electron Monte Carlo state,
electron Monte Carlo at the current subcell temperatures -> heat generated
per subcell (net phonon emission) -> Fourier solve -> new subcell
temperatures, repeated until no subcell temperature changes by more than
max(0.1 K, the Monte Carlo noise of the iteration).
Surrogate-corrected iteration: after each Monte Carlo run the surrogate's
drift velocity v_d(E, T) predicts how the heat of every subcell changes with
its temperature at its Monte Carlo field, and the Fourier solve is iterated
with that corrected heat to a self-consistent temperature field before the
next Monte Carlo run; the Monte Carlo iteration alone decides the result.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import emc as _emc

Q_E = 1.602176634e-19


def heat_map(ctx, seconds: float) -> np.ndarray:
    """Heat generation (W/m^3) per subcell from the net phonon energy
    tallied over the last `seconds` (tallies reset before the window)."""
    c = ctx.cfgs[0]
    Vc = c["Lx"] * c["Ly"] * c["Lz"] / ctx.n_cell
    return ctx.emc_tally(_emc.TALLY_HEAT_J) / (seconds * Vc)


def peak_rise(T: np.ndarray, T_sink: float) -> np.ndarray:
    return T.max(axis=1) - T_sink


def emitted_power(ctx, q: np.ndarray) -> np.ndarray:
    """Net power handed to phonons (W) per ensemble from a heat map (W/m^3)."""
    c = ctx.cfgs[0]
    return q.sum(axis=1) * (c["Lx"] * c["Ly"] * c["Lz"] / ctx.n_cell)


def thermal_resistance(T: np.ndarray, power: np.ndarray, T_sink: float) -> np.ndarray:
    """Device thermal resistance as the paper defines it for Fig. 5: the
    largest temperature rise divided by the total energy rate of the phonons
    the electrons emit (counted by the Monte Carlo, not the Joule heat).  K/W,
    per ensemble; NaN where no power is emitted."""
    rise = T.max(axis=1) - T_sink
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(power > 0, rise / power, np.nan)


def phonon_mc_temperature(ctx, tc, pc, q: np.ndarray, n_bundles: int, passes: int = 3, first: int = 0) -> dict:
    """Temperature (K) per subcell of the first wire of a nanowire context
    from the phonon Monte Carlo (emc_phonon_solve) for the heat q [C]
    (W/m^3): each pass takes the scattering rates and heat capacity at the
    temperatures of the previous pass (the first at T_sink; the coupling
    paragraph's local temperature) and fresh bundle ids.  Returns the
    temperatures, the peak rise after each pass and the last pass."""
    T = np.full(ctx.n_cell, tc.T_sink)
    peaks, r = [], None
    for k in range(passes):
        r = _emc.phonon_solve(ctx, tc, pc, q, n_bundles, T_cells=T, first=first + k * n_bundles)
        T = tc.T_sink + r["dT"]
        peaks.append(float(r["dT"].max()))
    return {"T": T, "peak_history": peaks, "last": r}


def mc_heat_halves(ctx, T: np.ndarray, warm_steps: int, avg_steps: int):
    """Heat maps of the two halves of the averaging window after warm_steps
    at the subcell temperatures T, and their mean (W/m^3): the halves are
    independent estimates, so their spread measures the Monte Carlo noise."""
    for e in range(ctx.n_ens):
        ctx.emc_set_temperature(e, T[e])
    ctx.emc_step(warm_steps)
    ctx.emc_tally(_emc.TALLY_OBS, reset=True)
    h = avg_steps // 2
    ctx.emc_step(h)
    qa = heat_map(ctx, h * ctx.cfgs[0]["dt"])
    ctx.emc_tally(_emc.TALLY_OBS, reset=True)
    ctx.emc_step(avg_steps - h)
    qb = heat_map(ctx, (avg_steps - h) * ctx.cfgs[0]["dt"])
    return 0.5 * (qa + qb), qa, qb


def _stop(T_new, T_old, Ta, Tb, stop_K: float):
    """The stop test of the coupled iteration: the largest change of any
    subcell temperature (over every bias point) since the previous iteration
    against max(stop_K, the largest difference between the temperatures of
    the two half-window heat maps).  Both are maxima over the same subcells
    of differences of two independent noisy estimates (the half windows'
    difference has twice the variance of the iterations'), so a change within
    the second is within the Monte Carlo noise."""
    d = np.abs(T_new - T_old).max(axis=1)
    n = np.abs(Ta - Tb).max(axis=1)
    return bool(d.max() <= max(stop_K, n.max())), d, n


def _result(ctx, tc, T, q, it, converged, hist, d_hist, n_hist, t0, **extra):
    P = emitted_power(ctx, q)
    r = {"converged": converged, "iterations": it, "T": T, "peak": peak_rise(T, tc.T_sink), "history": hist,
         "max_dT_K": d_hist, "noise_K": n_hist, "power_W": P,
         "R_th_K_per_W": thermal_resistance(T, P, tc.T_sink), "seconds": time.perf_counter() - t0}
    r.update(extra)
    return r


def iterate(ctx, tc, T0: np.ndarray, warm_steps: int = 300, avg_steps: int = 1000, max_iter: int = 15,
            stop_K: float = 0.1) -> dict:
    """Monte Carlo <-> Fourier fixed point from T0 (the hybrid method's
    coupled iteration, repeated until the temperature field is steady); the
    stop test is _stop (every subcell within max(stop_K, the noise))."""
    T = np.array(T0, dtype=float)
    hist, d_hist, n_hist = [], [], []
    t0 = time.perf_counter()
    q = None
    for it in range(1, max_iter + 1):
        q, qa, qb = mc_heat_halves(ctx, T, warm_steps, avg_steps)
        Tn, _ = _emc.thermal_solve(ctx, tc, q, T)
        Ta, _ = _emc.thermal_solve(ctx, tc, qa, Tn)
        Tb, _ = _emc.thermal_solve(ctx, tc, qb, Tn)
        ok, d, n = _stop(Tn, T, Ta, Tb, stop_K)
        T = Tn
        hist.append(peak_rise(T, tc.T_sink))
        d_hist.append(float(d.max()))
        n_hist.append(float(n.max()))
        if ok and it > 1:
            return _result(ctx, tc, T, q, it, True, hist, d_hist, n_hist, t0)
    return _result(ctx, tc, T, q, max_iter, False, hist, d_hist, n_hist, t0)


def hybrid_iterate(ctx, tc, pc, T0: np.ndarray, n_bundles: int, warm_steps: int = 300, avg_steps: int = 1000,
                   max_iter: int = 15, stop_K: float = 0.1, first: int = 0) -> dict:
    """Electron Monte Carlo <-> phonon Monte Carlo fixed point from T0 (the
    hybrid method with the phonon side in the transistor region): each
    iteration takes the electrons' heat map at the current subcell
    temperatures, and the phonon Monte Carlo (emc_phonon_solve, rates at the
    current temperatures) gives the next ones, for every ensemble of the
    context.  The stop test is _stop, with the noise of both Monte Carlos:
    the two half-window heat maps each carried by their own bundles."""
    T = np.array(T0, dtype=float)
    hist, d_hist, n_hist = [], [], []
    t0 = time.perf_counter()
    q = None
    nxt = first

    def phonon_T(heat, Tc):
        nonlocal nxt
        out = np.empty_like(Tc)
        for e in range(ctx.n_ens):
            r = _emc.phonon_solve(ctx, tc, pc, heat[e], n_bundles, T_cells=Tc[e], first=nxt)
            nxt += n_bundles
            out[e] = tc.T_sink + r["dT"]
        return out

    for it in range(1, max_iter + 1):
        q, qa, qb = mc_heat_halves(ctx, T, warm_steps, avg_steps)
        Tn = phonon_T(q, T)
        Ta = phonon_T(qa, T)
        Tb = phonon_T(qb, T)
        ok, d, n = _stop(Tn, T, Ta, Tb, stop_K)
        T = Tn
        hist.append(peak_rise(T, tc.T_sink))
        d_hist.append(float(d.max()))
        n_hist.append(float(n.max()))
        if ok and it > 1:
            return _result(ctx, tc, T, q, it, True, hist, d_hist, n_hist, t0)
    return _result(ctx, tc, T, q, max_iter, False, hist, d_hist, n_hist, t0)


def referee(ctx, tc, T: np.ndarray, warm_steps: int = 300, avg_steps: int = 5000) -> dict:
    """The plain Monte Carlo's assessment of a temperature field: one long
    Monte Carlo window at the subcell temperatures T, then the Fourier solve
    of its heat.  Any loop's result is refereed this way, so loops are
    compared on the temperatures the Monte Carlo itself gives back."""
    q, qa, qb = mc_heat_halves(ctx, T, warm_steps, avg_steps)
    Tj, _ = _emc.thermal_solve(ctx, tc, q, T)
    Ta, _ = _emc.thermal_solve(ctx, tc, qa, Tj)
    Tb, _ = _emc.thermal_solve(ctx, tc, qb, Tj)
    pk = peak_rise(Tj, tc.T_sink)
    # standard error of the peak from the two halves (each has twice the
    # variance of the full window)
    se = 0.5 * np.abs(peak_rise(Ta, tc.T_sink) - peak_rise(Tb, tc.T_sink))
    P = emitted_power(ctx, q)
    return {"T": Tj, "peak": pk, "peak_se": se, "max_dT_K": np.abs(Tj - T).max(axis=1), "power_W": P,
            "R_th_K_per_W": thermal_resistance(Tj, P, tc.T_sink)}


def warm_to_steady(ctx, window_steps: int = 200, max_windows: int = 100) -> dict:
    """Advance a nanowire context until its highest-bias ensemble (the last,
    slowest to settle) is steady by the drain-current / field-profile
    detector."""
    from .steady import run_to_steady
    return run_to_steady(ctx, ens=ctx.n_ens - 1, window_steps=window_steps, max_windows=max_windows)


def _vd(sur, E: np.ndarray, T: np.ndarray, log10_nd: np.ndarray) -> np.ndarray:
    """Surrogate drift velocity at (|E|, T, N_d) per subcell (field angle 0:
    the model is isotropic)."""
    from .surrogate import BOX, OUT_NAMES
    X = np.stack([np.minimum(E, BOX["E_max"]).ravel(), np.zeros(E.size), T.ravel(), log10_nd.ravel()], axis=1)
    return sur.predict(X)[:, OUT_NAMES.index("v_drift_m_s")].reshape(E.shape)


def surrogate_step(ctx, sur, tc, q: np.ndarray, T_mc: np.ndarray, E: np.ndarray, sweeps: int = 3,
                   floor: float = 0.25) -> np.ndarray:
    """Temperatures consistent with the heat q measured by Monte Carlo at T_mc
    once the surrogate's temperature response is applied: every subcell's
    heat scales with v_d(E_i, T_i) / v_d(E_i, T_mc,i) (power per electron
    e E v_d at the subcell's Monte Carlo field E_i); iterated with the Fourier
    solve.  The ratio is kept within [floor, 1 / floor]."""
    lnd = np.repeat(np.array([[math.log10(c["Nd"])] for c in ctx.cfgs]), ctx.n_cell, axis=1)
    v0 = _vd(sur, E, T_mc, lnd)
    T, _ = _emc.thermal_solve(ctx, tc, q, T_mc)
    for _ in range(sweeps):
        v = _vd(sur, E, T, lnd)
        ratio = np.where(v0 > 0, np.clip(v / np.where(v0 > 0, v0, 1.0), floor, 1.0 / floor), 1.0)
        T, _ = _emc.thermal_solve(ctx, tc, q * ratio, T)
    return T


def surrogate_accelerated(ctx, sur, tc, T0: np.ndarray, warm_steps: int = 300, avg_steps: int = 1000,
                          max_iter: int = 15, stop_K: float = 0.1, sweeps: int = 3,
                          corrected_iters: int | None = None) -> dict:
    """The Monte Carlo <-> Fourier iteration with the surrogate-corrected
    Fourier step between Monte Carlo runs (the stop test of iterate).
    corrected_iters = n: only the first n iterations are corrected and the
    plain iteration takes over from the temperatures they give (n = 1: the
    surrogate warm-starts the plain Monte Carlo iteration); None: every one."""
    T = np.array(T0, dtype=float)
    hist, d_hist, n_hist = [], [], []
    t0 = time.perf_counter()
    t_sur = 0.0
    q = None
    for it in range(1, max_iter + 1):
        q, qa, qb = mc_heat_halves(ctx, T, warm_steps, avg_steps)
        if corrected_iters is None or it <= corrected_iters:
            E = np.linalg.norm(ctx.emc_tally(_emc.TALLY_FIELD), axis=2)
            ts = time.perf_counter()
            Tn = surrogate_step(ctx, sur, tc, q, T, E, sweeps)
            t_sur += time.perf_counter() - ts
        else:
            Tn, _ = _emc.thermal_solve(ctx, tc, q, T)
        # the noise of the iteration: plain solves of the two half windows
        Ta, _ = _emc.thermal_solve(ctx, tc, qa, Tn)
        Tb, _ = _emc.thermal_solve(ctx, tc, qb, Tn)
        ok, d, n = _stop(Tn, T, Ta, Tb, stop_K)
        T = Tn
        hist.append(peak_rise(T, tc.T_sink))
        d_hist.append(float(d.max()))
        n_hist.append(float(n.max()))
        if ok and it > 1:
            return _result(ctx, tc, T, q, it, True, hist, d_hist, n_hist, t0, surrogate_seconds=t_sur)
    return _result(ctx, tc, T, q, max_iter, False, hist, d_hist, n_hist, t0, surrogate_seconds=t_sur)


def surrogate_heat_start(ctx, sur, tc) -> np.ndarray:
    """An initial temperature field from the surrogate alone: its heat per
    electron at each subcell's present field (and the sink temperature),
    times the subcell's electron density from the last charge count, is the
    predicted heat map; one Fourier solve of it gives the start of the plain
    iteration."""
    from .surrogate import OUT_NAMES
    c0 = ctx.cfgs[0]
    Vc = c0["Lx"] * c0["Ly"] * c0["Lz"] / ctx.n_cell
    E = np.linalg.norm(ctx.emc_tally(_emc.TALLY_FIELD), axis=2)
    w = np.array([c["Nd"] * c["Lx"] * c["Ly"] * c["Lz"] / c["n_particles"] for c in ctx.cfgs])[:, None]
    n_e = ctx.emc_tally(_emc.TALLY_CHARGE) * w / Vc
    lnd = np.repeat(np.array([[math.log10(c["Nd"])] for c in ctx.cfgs]), ctx.n_cell, axis=1)
    from .surrogate import BOX
    X = np.stack([np.minimum(E, BOX["E_max"]).ravel(), np.zeros(E.size), np.full(E.size, tc.T_sink), lnd.ravel()],
                 axis=1)
    heat = sur.predict(X)[:, OUT_NAMES.index("heat_W_per_electron")].reshape(E.shape)
    q = np.maximum(heat, 0.0) * n_e
    T, _ = _emc.thermal_solve(ctx, tc, q, np.full(E.shape, tc.T_sink))
    return T
