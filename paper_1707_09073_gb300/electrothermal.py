"""The coupled electrothermal iteration of the hybrid method and its
surrogate-corrected variant.

Plain iteration (the paragraph ending "until the steady-state temperature
distribution is obtained"): from a steady electron Monte Carlo state,
electron Monte Carlo at the current subcell temperatures -> heat generated
per subcell (net phonon emission) -> Fourier solve -> new subcell
temperatures, repeated until the peak temperature rise stops changing.
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


def mc_heat(ctx, T: np.ndarray, warm_steps: int, avg_steps: int) -> np.ndarray:
    for e in range(ctx.n_ens):
        ctx.emc_set_temperature(e, T[e])
    ctx.emc_step(warm_steps)
    ctx.emc_tally(_emc.TALLY_OBS, reset=True)
    ctx.emc_step(avg_steps)
    return heat_map(ctx, avg_steps * ctx.cfgs[0]["dt"])


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


def iterate(ctx, tc, T0: np.ndarray, warm_steps: int = 300, avg_steps: int = 1000, max_iter: int = 12,
            rtol: float = 0.01, atol: float = 0.5, relax: float = 1.0, prev_peak=None) -> dict:
    """Monte Carlo <-> Fourier fixed point from T0; converged when the peak
    temperature rise of the device (the largest over all bias points and
    subcells) changes by less than max(rtol * rise, atol kelvin) between
    iterations."""
    T = np.array(T0, dtype=float)
    hist = []
    t0 = time.perf_counter()
    prev = prev_peak
    for it in range(1, max_iter + 1):
        q = mc_heat(ctx, T, warm_steps, avg_steps)
        Tn, _ = _emc.thermal_solve(ctx, tc, q, T)
        T = T + relax * (Tn - T)
        pk = peak_rise(T, tc.T_sink)
        hist.append(pk.copy())
        if prev is not None and abs(pk.max() - prev.max()) <= max(rtol * abs(pk.max()), atol):
            P = emitted_power(ctx, q)
            return {"converged": True, "iterations": it, "T": T, "peak": pk, "history": hist, "power_W": P,
                    "R_th_K_per_W": thermal_resistance(T, P, tc.T_sink), "seconds": time.perf_counter() - t0}
        prev = pk
    P = emitted_power(ctx, q)
    return {"converged": False, "iterations": max_iter, "T": T, "peak": peak_rise(T, tc.T_sink), "history": hist,
            "power_W": P, "R_th_K_per_W": thermal_resistance(T, P, tc.T_sink), "seconds": time.perf_counter() - t0}


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
                          max_iter: int = 12, rtol: float = 0.01, atol: float = 0.5, sweeps: int = 3) -> dict:
    """The Monte Carlo <-> Fourier iteration with the surrogate-corrected
    Fourier step between Monte Carlo runs (same convergence test as
    iterate)."""
    T = np.array(T0, dtype=float)
    hist = []
    t0 = time.perf_counter()
    t_sur = 0.0
    prev = None
    q = None
    for it in range(1, max_iter + 1):
        q = mc_heat(ctx, T, warm_steps, avg_steps)
        E = np.linalg.norm(ctx.emc_tally(_emc.TALLY_FIELD), axis=2)
        ts = time.perf_counter()
        T = surrogate_step(ctx, sur, tc, q, T, E, sweeps)
        t_sur += time.perf_counter() - ts
        pk = peak_rise(T, tc.T_sink)
        hist.append(pk.copy())
        if prev is not None and abs(pk.max() - prev.max()) <= max(rtol * abs(pk.max()), atol):
            P = emitted_power(ctx, q)
            return {"converged": True, "iterations": it, "T": T, "peak": pk, "history": hist, "power_W": P,
                    "R_th_K_per_W": thermal_resistance(T, P, tc.T_sink), "seconds": time.perf_counter() - t0,
                    "surrogate_seconds": t_sur}
        prev = pk
    P = emitted_power(ctx, q)
    return {"converged": False, "iterations": max_iter, "T": T, "peak": peak_rise(T, tc.T_sink), "history": hist,
            "power_W": P, "R_th_K_per_W": thermal_resistance(T, P, tc.T_sink), "seconds": time.perf_counter() - t0,
            "surrogate_seconds": t_sur}
