"""Seeded synthetic workloads for the GaN electron Monte Carlo.

This module holds inputs only: the parameters of Table I (electron side) and
Table II (phonon side) of Hao et al., arXiv:1707.09073, the readings where the
paper is silent, and the configurations of the benchmark workloads.  It holds
none of the method's arithmetic, so both the FP64 CPU oracle (``oracle/``) and
the CUDA library (``paper_1707_09073_gb300``) can be driven from it without
sharing any code path.

A configuration is a plain ``dict``.  Units are SI except where the key says
otherwise (``*_eV``, ``*_per_eV``).
"""
from __future__ import annotations

import copy
import random

# --- Table I: parameters for bulk GaN in the electron MC -------------------
# Valley order: Gamma1, U, Gamma3 (the three lowest conduction valleys).
TABLE_I = {
    "n_cm3": 4.0e18,                     # electron density of the paper's run
    "m_rel": (0.21, 0.25, 0.40),         # valley-bottom effective mass / m0
    "Ec_eV": (0.0, 1.95, 2.1),           # valley minimum energy
    "alpha_per_eV": (0.19, 0.1, 0.0),    # Kane nonparabolicity
    "eps_s": 8.9,                        # static dielectric constant
    "eps_inf": 5.35,                     # high-frequency dielectric constant
    "rho_kg_m3": 6095.0,                 # 6.095 g/cm^3
    "Da_eV": 8.3,                        # acoustic deformation potential
    "Dij_eV_per_m": 1.0e11,              # 1.0e9 eV/cm intervalley potential
}

# --- Table II (GaN column) and the phonon numbers quoted in the text --------
TABLE_II_GAN = {
    "k0_per_m": 10.94e9,
    "omega_max_rad_s": 3.50e13,
    "aD_m": 2.87e-10,
    "A_s3": 5.26e-45,
    "B1_s_per_K": 1.10e-19,
    "B2_K": 200.0,
}
# Phonon-electron scattering of Eq. (1): DOS mass of the Gamma1 valley and
# D_a, rho from Table I; the averaged phonon group velocity is the averaged
# sound velocity the text quotes for GaN (3338 m/s)
ELECTRON_PHONON_GAN = {
    "m_rel": 0.21,
    "Da_eV": 8.3,
    "rho_kg_m3": 6095.0,
    "vg_m_s": 3338.0,
}
TABLE_II_SIC = {
    "k0_per_m": 8.94e9,
    "omega_max_rad_s": 7.12e13,
    "aD_m": 3.51e-10,
    "A_s3": 1.00e-45,
    "B1_s_per_K": 0.596e-19,
    "B2_K": 235.0,
}
HW_LO_EV = 0.0912          # LO phonon energy taken by hot electrons
VS_AVG_M_S = 3338.0        # averaged acoustic sound velocity (Si-impurity estimate)
V0_M3 = 11.42e-30          # unit volume of wurtzite GaN
F_SI = 4.5e-5              # fractional Si concentration at 4e18 cm^-3
A_SI_PRINTED_S3 = 1.2e-46  # the paper's Si mass-difference A
M_GA, M_N, M_SI = 69.723, 14.007, 28.085   # standard atomic masses (u)

# --- Readings where the paper is silent (each is a config field) ------------
READINGS = {
    "Z": (1, 6, 1),            # valley degeneracies Gamma1/U/Gamma3
    "hw_lo_eV": HW_LO_EV,      # POP phonon energy
    "hw_iv_eV": HW_LO_EV,      # intervalley phonon energy, same for all pairs
    # sound velocity for electron acoustic scattering: omega_max * a_D / 2 of
    # the GaN column of Table II (3.50e13 rad/s * 2.87 A / 2)
    "vs_m_s": 5022.5,
    "n_bins": 2048,            # rate-table bins
    "dE_eV": 0.002,            # rate-table bin width (table spans 0..4.096 eV)
    "emax_init_kT": 40.0,      # truncation of the initial Kane-Maxwellian
    "p_specular": 0.5,         # specular fraction on the non-symmetry walls
}


def _base() -> dict:
    c = {}
    c.update({k: v for k, v in TABLE_I.items() if k != "n_cm3"})
    c.update(READINGS)
    c.update({
        "T": 300.0,
        "Nd": 1.0e23,                 # m^-3 (1e17 cm^-3)
        "field": (0.0, 0.0, 1.0e7),   # V/m, bulk only (100 kV/cm along c)
        "dt": 1.0e-15,
        "geometry": 0,                # 0 bulk, 1 half nanowire
        "nx": 1, "ny": 1, "nz": 1,
        "Lx": 1.0, "Ly": 1.0, "Lz": 1.0,
        "gate_on": 0, "gate_x0": 0.0, "gate_x1": 0.0,
        "Vs": 0.0, "Vd": 0.0, "Vg": 0.0,
        "steps_per_poisson": 10,
        "n_particles": 10_000,
        "capacity": 10_000,
        "seed": 0,
        "mech_mask": 0x3FF,           # all ten mechanisms enabled
    })
    return c


def bulk(n_particles: int = 10_000, field_V_m: float = 1.0e7, T: float = 300.0,
         Nd_cm3: float = 1.0e17, seed: int = 0, **over) -> dict:
    """Bulk wurtzite GaN ensemble: uniform field along the c axis (z)."""
    c = _base()
    c.update(n_particles=int(n_particles), capacity=int(n_particles),
             field=(0.0, 0.0, float(field_V_m)), T=float(T),
             Nd=float(Nd_cm3) * 1e6, seed=int(seed))
    c.update(over)
    return c


def nanowire(n_particles: int = 200_000, Vd: float = 10.0, Vg: float = 0.0,
             T: float = 300.0, Nd_cm3: float = 1.0e18, seed: int = 0,
             nx: int = 100, ny: int = 3, nz: int = 6, Lx: float = 1.0e-6,
             Ly: float = 60e-9, Lz: float = 120e-9, spare: float | None = None,
             **over) -> dict:
    """Half-nanowire FinFET domain: x along the wire (source at x=0, drain at
    x=Lx), y across the half wire (symmetry plane A at y=0), z height.  The
    gate covers the top face and the outer side face over the middle half of
    the wire."""
    c = _base()
    ncell = nx * ny * nz
    if spare is None:
        # room for contact re-injection: two contact layers refilled
        extra = max(64, 2 * ny * nz * (n_particles // max(ncell, 1) + 8))
    else:
        extra = int(spare)
    c.update(geometry=1, nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz,
             gate_on=1, gate_x0=0.25 * Lx, gate_x1=0.75 * Lx,
             Vs=0.0, Vd=float(Vd), Vg=float(Vg), field=(0.0, 0.0, 0.0),
             T=float(T), Nd=float(Nd_cm3) * 1e6,
             n_particles=int(n_particles), capacity=int(n_particles) + extra,
             seed=int(seed))
    c.update(over)
    return c


# --- The benchmark workloads ------------------------------------------------
def config_bulk_small() -> dict:
    """10,000 electrons, 1e17 cm^-3, 300 K, 100 kV/cm along c, dt = 1 fs,
    2000 steps (2 ps), Philox seed 0."""
    return bulk()


BULK_SMALL_STEPS = 2000


def config_nanowire_sweep() -> list[dict]:
    """Half nanowire 60 x 120 nm x 1 um, 3 x 6 x 100 subcells, 1e18 cm^-3,
    200,000 superparticles per bias point, Poisson every 10 fs, V_ds swept
    0..20 V in 1 V steps (21 independent bias points)."""
    return [nanowire(Vd=float(v), seed=v) for v in range(21)]


def config_bulk_large(n_particles: int = 10_000_000) -> dict:
    """Precision variant: the bulk physics with 1e7 electrons, 20 ps."""
    return bulk(n_particles=n_particles)


def config_batched(n_ens: int = 256, seed: int = 0, scale: float = 1.0) -> list[dict]:
    """Many independent ensembles in one batch: per ensemble N ~ 10^U(4, 6)
    electrons (times `scale`, at least 1), |E| ~ U(0, 400) kV/cm, T ~ U(300,
    600) K, N_d ~ 10^U(16, 19) cm^-3; every fourth ensemble is a half nanowire
    with V_d = |E| L (Poisson field), the others bulk with the field along c.
    Draws come from Python's Mersenne Twister seeded with `seed`, in ensemble
    order (N, |E|, T, N_d)."""
    rng = random.Random(seed)
    out = []
    for e in range(n_ens):
        n = max(1, int(round(10.0 ** rng.uniform(4.0, 6.0) * scale)))
        E = rng.uniform(0.0, 4.0e7)
        T = rng.uniform(300.0, 600.0)
        nd = 10.0 ** rng.uniform(16.0, 19.0)
        s = 1_000_000 * seed + e
        if e % 4 == 3:
            out.append(nanowire(n_particles=n, Vd=E * 1.0e-6, T=T, Nd_cm3=nd, seed=s))
        else:
            out.append(bulk(n_particles=n, field_V_m=E, T=T, Nd_cm3=nd, seed=s))
    return out


def heat_map(cfg: dict, peak_W_m3: float = 9.0e17, seed: int = 0) -> "np.ndarray":
    """Seeded synthetic heat generation per subcell (W/m^3) of a nanowire
    configuration, shaped like the electrons' at a high drain bias: a floor
    of 1/9 of the peak along the wire, a Gaussian bump of width 0.08 L at 0.75
    L (the drain-side gate edge), subcell-to-subcell scatter of +-50%, and a
    negative stretch (net phonon absorption) over the first 5% of the wire."""
    import numpy as _np
    rng = _np.random.default_rng(seed)
    x = (_np.arange(cfg["nx"]) + 0.5) / cfg["nx"]
    prof = (1.0 + 8.0 * _np.exp(-((x - 0.75) / 0.08) ** 2)) / 9.0
    q = _np.repeat(prof, cfg["ny"] * cfg["nz"]) * rng.uniform(0.5, 1.5, cfg["nx"] * cfg["ny"] * cfg["nz"])
    q[: max(1, cfg["nx"] // 20) * cfg["ny"] * cfg["nz"]] *= -0.2
    return q * peak_W_m3


def by_geometry(cfgs: list[dict]) -> dict[int, list[int]]:
    """Indices of the configurations of each geometry (one context each)."""
    g: dict[int, list[int]] = {}
    for i, c in enumerate(cfgs):
        g.setdefault(int(c["geometry"]), []).append(i)
    return g


def copy_config(c: dict, **over) -> dict:
    d = copy.deepcopy(c)
    d.update(over)
    return d
