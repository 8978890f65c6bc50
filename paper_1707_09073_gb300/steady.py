"""Steady-state detection for the self-consistent nanowire run.

The paper counts the heat once the current and the electric field no longer
change (the paragraph on the field update and the heat counted in steady
state).  Reading taken: over consecutive windows (default 100 time
steps), the window-mean drain current and the subcell field are compared
with the previous window's; the run is steady once, for `need` windows in a
row, the current changed by less than max(rtol |I|, 3 sigma of its window
noise) and the window-mean field profile along the wire (averaged over each
cross-section, which removes most of the subcell counting noise) by less
than ftol in relative RMS.
"""
from __future__ import annotations

import numpy as np

from . import emc as _emc

Q_E = 1.602176634e-19


class SteadyState:
    def __init__(self, rtol: float = 0.01, ftol: float = 0.01, need: int = 3):
        self.rtol, self.ftol, self.need = rtol, ftol, need
        self.prev_I = None
        self.prev_F = None
        self.streak = 0
        self.history = []

    def update(self, current: float, field: np.ndarray, current_sigma: float = 0.0) -> bool:
        """Feed one window's mean drain current (A), its standard error, and the
        subcell field at the window end; returns True once steady."""
        F = np.asarray(field, dtype=float)
        ok = False
        if self.prev_I is not None:
            dI = abs(current - self.prev_I)
            tolI = max(self.rtol * abs(current), 3.0 * np.hypot(current_sigma, self.prev_sigma))
            scale = max(np.sqrt(np.mean(F * F)), 1e-300)
            dF = float(np.sqrt(np.mean((F - self.prev_F) ** 2)) / scale)
            ok = dI <= tolI and dF <= self.ftol
            self.history.append((current, dI, tolI, dF))
        self.streak = self.streak + 1 if ok else 0
        self.prev_I, self.prev_F, self.prev_sigma = current, F.copy(), current_sigma
        return self.streak >= self.need


def window_current(cross_before: np.ndarray, cross_after: np.ndarray, weight: float, seconds: float) -> float:
    """Drain current (A, electrons flowing out through the drain) from the
    crossing tallies [source out, drain out, source in, drain in] of a window."""
    d = np.asarray(cross_after, dtype=np.int64) - np.asarray(cross_before, dtype=np.int64)
    return Q_E * weight * float(d[1] - d[3]) / seconds


def run_to_steady(ctx: "_emc.Context", ens: int = 0, window_steps: int = 100, max_windows: int = 200,
                  sub_windows: int = 5, detector: SteadyState | None = None) -> dict:
    """Advance a nanowire context window by window until ensemble `ens` is
    steady (or max_windows); returns the window history and the step count."""
    det = detector or SteadyState()
    c = ctx.cfgs[ens]
    w = c["Nd"] * c["Lx"] * c["Ly"] * c["Lz"] / c["n_particles"]
    sub = max(1, window_steps // sub_windows)
    nx, nyz = c["nx"], c["ny"] * c["nz"]
    for k in range(max_windows):
        parts, prof = [], []
        for _ in range(sub_windows):
            before = ctx.emc_tally(_emc.TALLY_CROSSINGS)[ens].copy()
            ctx.emc_step(sub)
            after = ctx.emc_tally(_emc.TALLY_CROSSINGS)[ens]
            parts.append(window_current(before, after, w, sub * c["dt"]))
            prof.append(ctx.emc_tally(_emc.TALLY_FIELD)[ens].reshape(nx, nyz, 3).mean(axis=1))
        I = float(np.mean(parts))
        sig = float(np.std(parts, ddof=1) / np.sqrt(len(parts))) if len(parts) > 1 else 0.0
        F = np.mean(prof, axis=0)
        if det.update(I, F, sig):
            return {"steady": True, "windows": k + 1, "current": I, "history": det.history}
    return {"steady": False, "windows": max_windows, "current": det.prev_I, "history": det.history}
