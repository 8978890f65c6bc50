"""The coupled electrothermal iteration of the hybrid method and its
surrogate warm start.

Plain iteration (the paragraph ending "until the steady-state temperature
distribution is obtained"): electron Monte Carlo at the current subcell
temperatures -> heat generated per subcell (net phonon emission) -> Fourier
solve -> new subcell temperatures, repeated until the peak temperature rise
stops changing.  Warm start: before the first Monte Carlo run, the surrogate
predicts the heat of every subcell from its local field, temperature and
doping (local-field approximation), iterated with the Fourier solve to a
self-consistent first guess of the temperatures; the Monte Carlo iteration
then starts there and remains the judge of the result.
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


def iterate(ctx, tc, T0: np.ndarray, warm_steps: int = 300, avg_steps: int = 600, max_iter: int = 12,
            rtol: float = 0.01, relax: float = 1.0) -> dict:
    """Monte Carlo <-> Fourier fixed point from T0; converged when every
    ensemble's peak rise changes by less than rtol between iterations."""
    T = np.array(T0, dtype=float)
    hist = []
    t0 = time.perf_counter()
    prev = None
    for it in range(1, max_iter + 1):
        q = mc_heat(ctx, T, warm_steps, avg_steps)
        Tn, _ = _emc.thermal_solve(ctx, tc, q, T)
        T = T + relax * (Tn - T)
        pk = peak_rise(T, tc.T_sink)
        hist.append(pk.copy())
        if prev is not None and np.all(np.abs(pk - prev) <= rtol * np.maximum(np.abs(pk), 1e-9)):
            return {"converged": True, "iterations": it, "T": T, "peak": pk, "history": hist,
                    "seconds": time.perf_counter() - t0}
        prev = pk
    return {"converged": False, "iterations": max_iter, "T": T, "peak": peak_rise(T, tc.T_sink), "history": hist,
            "seconds": time.perf_counter() - t0}


def surrogate_start(ctx, sur, tc, sweeps: int = 8) -> tuple[np.ndarray, float]:
    """First guess of the subcell temperatures from the surrogate: local
    |E|, field angle to the c axis, T and N_d of every subcell -> heat per
    electron, times the subcell electron density; alternated with the Fourier
    solve.  Returns the temperatures and the seconds spent."""
    t0 = time.perf_counter()
    E = ctx.emc_tally(_emc.TALLY_FIELD)                  # [E][C][3] V/m
    n_cnt = ctx.emc_tally(_emc.TALLY_CHARGE).astype(float)
    Em = np.linalg.norm(E, axis=2)
    ang = np.arccos(np.clip(np.abs(E[..., 2]) / np.maximum(Em, 1e-30), 0.0, 1.0))
    T = np.full((ctx.n_ens, ctx.n_cell), tc.T_sink)
    j_heat = 5
    for _ in range(sweeps):
        rows = []
        for e, c in enumerate(ctx.cfgs):
            rows.append(np.stack([Em[e], ang[e], T[e], np.full(ctx.n_cell, math.log10(c["Nd"]))], axis=1))
        X = np.concatenate(rows).astype(np.float32)
        h = sur.predict(X)[:, j_heat].reshape(ctx.n_ens, ctx.n_cell)
        q = np.empty_like(h)
        for e, c in enumerate(ctx.cfgs):
            Vc = c["Lx"] * c["Ly"] * c["Lz"] / ctx.n_cell
            w = c["Nd"] * c["Lx"] * c["Ly"] * c["Lz"] / c["n_particles"]
            q[e] = np.maximum(h[e], 0.0) * w * n_cnt[e] / Vc
        T, _ = _emc.thermal_solve(ctx, tc, q, T)
    return T, time.perf_counter() - t0
