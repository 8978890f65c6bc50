"""The coupled electrothermal iteration of the hybrid method and its
surrogate-accelerated variant.

Plain iteration (the paragraph ending "until the steady-state temperature
distribution is obtained"): electron Monte Carlo at the current subcell
temperatures -> heat generated per subcell (net phonon emission) -> Fourier
solve -> new subcell temperatures, repeated until the peak temperature rise
stops changing.  Accelerated iteration: after the first Monte Carlo run the
surrogate's drift velocity v_d(E, T) predicts how the device current, and so
the heat, responds to the temperature field; that prediction is iterated with
the Fourier solve to a first guess of the self-consistent temperatures, and
the Monte Carlo iteration continues from there and remains the judge of the
result.
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


def _invert(v: np.ndarray, Eg: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Field at which the increasing velocity curves v[..., :] (sampled at
    Eg) reach target[...] (linear interpolation, clamped to the grid)."""
    n = v.shape[-1]
    k = np.clip((v < target[..., None]).sum(axis=-1), 1, n - 1)
    v0 = np.take_along_axis(v, (k - 1)[..., None], -1)[..., 0]
    v1 = np.take_along_axis(v, k[..., None], -1)[..., 0]
    a = np.clip((target - v0) / np.maximum(v1 - v0, 1e-30), 0.0, 1.0)
    return Eg[k - 1] + a * (Eg[k] - Eg[k - 1])


def current_ratio(ctx, sur, T: np.ndarray, E0: np.ndarray, T0: float, n_grid: int = 128) -> np.ndarray:
    """Ratio r = J(T) / J(T0) of the device current under the temperature
    field T, from the surrogate's drift velocity: every x-slice keeps the
    Monte Carlo field E0_i it had at the uniform temperature T0 as its
    operating point, its field at T solves v_d(E_i, T_i) = r v_d(E0_i, T0)
    (increasing branch of v_d(E)), and r is the value for which the voltage
    sum_i E_i dx is unchanged (current continuity along the wire)."""
    from .surrogate import BOX, OUT_NAMES
    c0 = ctx.cfgs[0]
    nx, nyz = c0["nx"], c0["ny"] * c0["nz"]
    E0 = np.minimum(E0, BOX["E_max"])
    Eg = np.concatenate([[0.0], np.geomspace(1e3, BOX["E_max"], n_grid - 1)])
    jv = OUT_NAMES.index("v_drift_m_s")
    Ts = T.reshape(ctx.n_ens, nx, nyz).mean(axis=2)
    X = np.empty((ctx.n_ens, nx, n_grid + 1, 4), dtype=np.float32)
    X[..., :n_grid, 0] = Eg[None, None, :]
    X[..., n_grid, 0] = E0
    X[..., 1] = 0.0
    X[..., :n_grid, 2] = Ts[:, :, None]
    X[..., n_grid, 2] = T0
    for e, c in enumerate(ctx.cfgs):
        X[e, ..., 3] = math.log10(c["Nd"])
    out = sur.predict(X.reshape(-1, 4))[:, jv].reshape(ctx.n_ens, nx, n_grid + 1)
    v = np.maximum.accumulate(np.maximum(out[..., :n_grid], 0.0), axis=2)
    v0 = np.minimum(np.maximum(out[..., n_grid], 0.0), v[..., -1])
    V0 = E0.sum(axis=1)
    lo, hi = np.zeros(ctx.n_ens), np.full(ctx.n_ens, 4.0)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        Vm = _invert(v, Eg, mid[:, None] * v0).sum(axis=1)
        low = Vm < V0
        lo = np.where(low, mid, lo)
        hi = np.where(low, hi, mid)
    r = 0.5 * (lo + hi)
    return np.where((V0 > 0) & (v0.max(axis=1) > 0), r, 1.0)


def surrogate_accelerated(ctx, sur, tc, T_start: float = None, warm_steps: int = 300, avg_steps: int = 1000,
                          max_iter: int = 12, rtol: float = 0.01, atol: float = 0.5, sweeps: int = 10) -> dict:
    """Electrothermal iteration accelerated by the surrogate.  Monte Carlo
    iteration 1 at the uniform start temperature gives the heat map q1 (the
    plain iteration's first step too).  The surrogate then predicts how the
    device current responds to the temperature field, J(T) / J(T_start)
    (current_ratio), and q = q1 J(T) / J(T_start) is iterated with the Fourier
    solve to a predicted self-consistent temperature field -- the step the
    plain fixed-point iteration takes many Monte Carlo runs to make.  Monte
    Carlo iterations continue from there until the peak rise is stationary;
    the Monte Carlo remains the judge of the result."""
    T_start = tc.T_sink if T_start is None else T_start
    t0 = time.perf_counter()
    T = np.full((ctx.n_ens, ctx.n_cell), T_start)
    q1 = mc_heat(ctx, T, warm_steps, avg_steps)
    ts = time.perf_counter()
    c0 = ctx.cfgs[0]
    E0 = np.abs(ctx.emc_tally(_emc.TALLY_FIELD)[..., 0]).reshape(ctx.n_ens, c0["nx"], -1).mean(axis=2)
    Tp, _ = _emc.thermal_solve(ctx, tc, q1, T)
    for _ in range(sweeps):
        ratio = current_ratio(ctx, sur, Tp, E0, T_start)
        Tp, _ = _emc.thermal_solve(ctx, tc, q1 * ratio[:, None], Tp)
    t_sur = time.perf_counter() - ts
    r = iterate(ctx, tc, Tp, warm_steps, avg_steps, max_iter - 1, rtol, atol, prev_peak=peak_rise(Tp, tc.T_sink))
    r["iterations"] += 1
    r["seconds"] = time.perf_counter() - t0
    r["surrogate_seconds"] = t_sur
    r["predicted_peak"] = peak_rise(Tp, tc.T_sink)
    return r
