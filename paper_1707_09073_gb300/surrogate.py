"""The learned surrogate: local conditions -> Monte Carlo observables.

Inputs per sample: |E| (V/m), field angle to the c axis (rad), lattice
temperature T (K), log10 of the donor density N_d (m^-3); the network sees
the field as ln(1 + |E| / 1 kV/cm).  Outputs: drift
velocity along -E (m/s), mean kinetic energy (eV), Gamma1/U/Gamma3 fractions,
net phonon-emission heat per electron (W), current density q N_d v_d
(A/m^2).  Training data come from batched bulk runs of this library's own
Monte Carlo (one ensemble per sample); the network is the tensor-core MLP of
emc_mlp_* (4 -> 128 -> 128 -> 128 -> 7 by default).

The model is isotropic (spherical valleys), so the observables do not depend
on the field angle; the network is given the angle anyway and has to learn to
ignore it.
"""
from __future__ import annotations

import math

import numpy as np

from . import emc as _emc

Q_E = 1.602176634e-19
N_IN, N_OUT = 4, 7
OUT_NAMES = ("v_drift_m_s", "E_mean_eV", "f_Gamma1", "f_U", "f_Gamma3", "heat_W_per_electron", "J_A_m2")
# sampling box of the inputs: fields up to 2500 kV/cm, the range the drain
# end of the biased nanowire reaches (its mean field is at most 200 kV/cm)
BOX = {"E_max": 2.5e8, "T": (300.0, 600.0), "log10_Nd": (22.0, 25.0)}
# the network sees the field as xi = ln(1 + |E| / E_REF): low fields, where
# the mobility and its temperature dependence matter, get as much of the
# input range (and of the training samples) as the saturated high fields
E_REF = 1.0e5
XI_MAX = math.log1p(BOX["E_max"] / E_REF)


def features(X: np.ndarray) -> np.ndarray:
    """Network inputs from the physical ones (|E| -> xi, others as they are)."""
    F = np.array(X, dtype=np.float64, copy=True)
    F[:, 0] = np.log1p(np.maximum(F[:, 0], 0.0) / E_REF)
    return F


def sample_inputs(n: int, seed: int = 0) -> np.ndarray:
    """Physical inputs, uniform in xi (so log-like in |E|), angle, T and
    log10 N_d."""
    rng = np.random.default_rng(seed)
    return np.stack([
        E_REF * np.expm1(rng.uniform(0.0, XI_MAX, n)),
        rng.uniform(0.0, math.pi, n),
        rng.uniform(*BOX["T"], n),
        rng.uniform(*BOX["log10_Nd"], n),
    ], axis=1)


def bulk_config(base: dict, x: np.ndarray, n_electrons: int, seed: int) -> dict:
    E, ang, T, lnd = x
    c = dict(base)
    c.update(n_particles=int(n_electrons), capacity=int(n_electrons), T=float(T), Nd=float(10.0 ** lnd),
             field=(float(E * math.sin(ang)), 0.0, float(E * math.cos(ang))), seed=int(seed), geometry=0,
             nx=1, ny=1, nz=1, steps_per_launch=50)
    return c


def mc_observables(inputs: np.ndarray, base: dict, n_electrons: int = 2000, warm_steps: int = 1000,
                   avg_steps: int = 1000, batch: int = 1024, seed0: int = 0, stream=None) -> np.ndarray:
    """Run one bulk ensemble per input row (batched contexts) and return the
    observables [n][7] averaged over avg_steps after warm_steps."""
    out = np.zeros((inputs.shape[0], N_OUT))
    dt = base["dt"]
    hw_lo, hw_iv = base["hw_lo_eV"], base["hw_iv_eV"]
    for b0 in range(0, inputs.shape[0], batch):
        xs = inputs[b0:b0 + batch]
        cfgs = [bulk_config(base, x, n_electrons, seed0 + b0 + i) for i, x in enumerate(xs)]
        with _emc.Context(cfgs, stream=stream) as ctx:
            ctx.emc_step(warm_steps)
            ctx.emc_tally(_emc.TALLY_OBS, reset=True)
            ctx.emc_step(avg_steps)
            obs = ctx.emc_tally(_emc.TALLY_OBS)
            ev = ctx.emc_tally(_emc.TALLY_EVENTS).astype(np.int64)
        for i, (x, o) in enumerate(zip(xs, obs)):
            n = max(o["n_samples"], 1)
            E, ang = x[0], x[1]
            ehat = np.array([math.sin(ang), 0.0, math.cos(ang)])
            vd = float(-(o["sum_v"] @ ehat) / n) if E > 0 else 0.0
            e = ev[i]
            net = (e[:, 2].sum() - e[:, 1].sum()) * hw_lo + (e[:, 5::2].sum() - e[:, 4::2].sum()) * hw_iv
            heat = net * Q_E / (n * dt)
            out[b0 + i] = [vd, o["sum_E"] / n / Q_E, *(o["valley_steps"] / n), heat, Q_E * 10.0 ** x[3] * vd]
    return out


class Surrogate:
    """Tensor-core MLP fitted to Monte Carlo observables."""

    def __init__(self, X: np.ndarray, Y: np.ndarray, hidden: int = 128, layers: int = 3, seed: int = 0,
                 stream=None):
        x_shift = np.array([XI_MAX / 2, math.pi / 2, sum(BOX["T"]) / 2, sum(BOX["log10_Nd"]) / 2])
        x_scale = np.array([XI_MAX / 2, math.pi / 2, (BOX["T"][1] - BOX["T"][0]) / 2,
                            (BOX["log10_Nd"][1] - BOX["log10_Nd"][0]) / 2])
        y_shift = Y.mean(axis=0)
        y_scale = np.maximum(Y.std(axis=0), 1e-12 * np.maximum(np.abs(y_shift), 1.0))
        y_scale[y_scale == 0] = 1.0
        self.net = _emc.Mlp(N_IN, hidden, layers, N_OUT, x_shift, x_scale, y_shift, y_scale, seed=seed, stream=stream)

    def fit(self, X: np.ndarray, Y: np.ndarray, steps: int = 4000, batch: int = 1024, lr: float = 1e-3,
            seed: int = 0) -> np.ndarray:
        return self.net.train(features(X).astype(np.float32), Y, steps=steps, batch=batch, lr=lr, seed=seed)

    def predict(self, X: np.ndarray) -> np.ndarray:
        return self.net.infer(features(np.asarray(X)).astype(np.float32)).astype(np.float64)
