"""FP64 reference of the phonon Monte Carlo (``phonon_oracle.c``) with its
spectral tables.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the ``cpu_baseline``
leg of ``bench.py``; never by the product package, and it never imports it.

The phonon model is the paper's phonon-model paragraph and Table II: three
identical acoustic branches omega = omega_max sin(pi q / 2 q0), relaxation
1/tau = A omega^4 + B1 omega^2 T exp(-B2/T), optionally the boundary term
v_g / L_b (size-modified mean free paths, the paragraph after Eq. (3)) and
the phonon-electron rate of Eq. (1); the interface transmissivity is
Eq. (2).  The spectrum is split into ``nb`` equal wave-vector bins of
(0, q0) (equal in q, so the density of states needs no frequency
integration across the band-edge singularity); a bin stands for its centre
q_b and frequency omega_b = omega_max sin(pi q_b / 2 q0):

- group velocity v_b = (pi omega_max / 2 q0) cos(pi q_b / 2 q0);
- heat capacity per unit volume of the bin, three branches:
  C_b = 3 hbar omega_b dn/dT q_b^2 dq / (2 pi^2);
- re-emission (and source) distribution after a scattering proportional to
  C_b / tau_b, which conserves the deviational energy bundle by bundle (the
  energy-based formulation of Peraud and Hadjiconstantinou, 2011).

Rates are tabulated at each subcell's temperature rounded to whole kelvin.
The steady temperature rise of subcell c is P t_c / (N C_tot V_c): P the
sum of |q| V over the subcells, t_c the signed time all N bundles spent in
it (a bundle carries the sign of the heat of the subcell it started in:
negative heat, where the electrons absorb more than they emit, is a phonon
deficit), C_tot = sum C_b at its temperature.
"""
from __future__ import annotations

import ctypes as C
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import oracle as _o
from . import thermal as TH

HB, KB = TH.HB, TH.KB
SPECULAR, ROUGH, ISOTHERMAL, INTERFACE = 0, 1, 2, 3


def bins(mat: dict, nb: int):
    """Centre wave vector q_b (1/m), frequency (rad/s), group velocity (m/s)
    and modes per branch and unit volume q_b^2 dq / (2 pi^2) of each of nb
    equal bins of (0, q0)."""
    q0, wm = mat["k0_per_m"], mat["omega_max_rad_s"]
    dq = q0 / nb
    q = (np.arange(nb) + 0.5) * dq
    w = wm * np.sin(np.pi * q / (2.0 * q0))
    v = wm * np.pi / (2.0 * q0) * np.cos(np.pi * q / (2.0 * q0))
    modes = q * q * dq / (2.0 * np.pi ** 2)
    return q, w, v, modes


def heat_capacity(mat: dict, nb: int, T: float) -> np.ndarray:
    """C_b (J/(m^3 K)) of each bin, three branches: 3 hbar omega dn/dT per
    mode times the bin's modes."""
    _, w, _, modes = bins(mat, nb)
    x = HB * w / (KB * T)
    dndT = x * np.exp(x) / np.expm1(x) ** 2 / T
    return 3.0 * HB * w * dndT * modes


def rates(mat: dict, nb: int, T: float, L_b: float = 0.0, n_e: float = 0.0, elec=None) -> np.ndarray:
    """1/tau (1/s) of each bin at temperature T."""
    _, w, v, _ = bins(mat, nb)
    r = mat["A_s3"] * w ** 4 + mat["B1_s_per_K"] * w ** 2 * T * np.exp(-mat["B2_K"] / T)
    if L_b > 0:
        r = r + v / L_b
    if n_e > 0:
        EF = TH.fermi_level(n_e, T, elec["m_rel"])
        r = r + np.array([TH.tau_e_inv(x, T, n_e, elec, EF) for x in w])
    return r


def kappa_binned(mat: dict, nb: int, T: float, L_b: float = 0.0, n_e: float = 0.0, elec=None) -> float:
    """(1/3) sum C_b v_b^2 tau_b: the conductivity the binned spectrum
    carries in the diffusive limit."""
    _, _, v, _ = bins(mat, nb)
    return float(np.sum(heat_capacity(mat, nb, T) * v * v / rates(mat, nb, T, L_b, n_e, elec)) / 3.0)


class Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nb", C.c_int32), ("nt", C.c_int32),
                ("pad_", C.c_int32), ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("vg", C.POINTER(C.c_double)), ("rate", C.POINTER(C.c_double)), ("cdf", C.POINTER(C.c_double)),
                ("tix", C.POINTER(C.c_int32)), ("cell_cdf", C.POINTER(C.c_double)),
                ("cell_sign", C.POINTER(C.c_double)),
                ("tau12", C.POINTER(C.c_double)), ("face", C.c_int32 * 6), ("p_specular", C.c_double * 6),
                ("seed", C.c_uint32), ("pad2_", C.c_uint32), ("max_segments", C.c_int64)]


class Tally(C.Structure):
    _fields_ = [("t_res", C.POINTER(C.c_double)), ("scatterings", C.POINTER(C.c_uint64)),
                ("emitted", C.POINTER(C.c_uint64)), ("absorbed", C.c_uint64 * 6), ("segments", C.c_uint64),
                ("capped", C.c_uint64)]


def _lib():
    L = _o.lib()
    if not hasattr(L, "_ph_ready"):
        L.ph_run.argtypes = [C.POINTER(Problem), C.c_int64, C.c_int64, C.POINTER(Tally)]
        L.ph_run.restype = None
        L.ph_test_lambert.argtypes = [C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.ph_test_lambert.restype = None
        L.ph_test_draw.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.POINTER(C.c_double)]
        L.ph_test_draw.restype = None
        L.ph_test_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.ph_test_philox.restype = None
        L._ph_ready = True
    return L


def lambert(f: int, u1: float, u2: float) -> np.ndarray:
    d = np.zeros(3)
    _lib().ph_test_lambert(f, u1, u2, d.ctypes.data_as(C.POINTER(C.c_double)))
    return d


def philox(ctr, key) -> list:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    _lib().ph_test_philox(c, k, o)
    return list(o)


def draws(seed: int, bundle: int, n0: int, count: int) -> np.ndarray:
    u = np.zeros((count, 4))
    _lib().ph_test_draw(seed, bundle, n0, count, u.ctypes.data_as(C.POINTER(C.c_double)))
    return u


def tables(mat, nb, T_cells, L_b=0.0, n_e=0.0, elec=None):
    """Per-subcell table index and the tables of the distinct whole-kelvin
    temperatures: (tix, rate 1/ps [nt][nb], cdf [nt][nb], C_tot [nt])."""
    keys = np.floor(np.asarray(T_cells, dtype=float) + 0.5).astype(np.int64)
    uniq = sorted(set(keys.tolist()))
    pos = {k: i for i, k in enumerate(uniq)}
    tix = np.array([pos[k] for k in keys], dtype=np.int32)
    rate = np.zeros((len(uniq), nb))
    cdf = np.zeros((len(uniq), nb))
    ctot = np.zeros(len(uniq))
    for i, k in enumerate(uniq):
        r = rates(mat, nb, float(k), L_b, n_e, elec)
        cb = heat_capacity(mat, nb, float(k))
        wgt = np.cumsum(cb * r)
        rate[i] = r * 1e-12
        cdf[i] = wgt / wgt[-1]
        cdf[i, -1] = 1.0
        ctot[i] = cb.sum()
    return tix, rate, cdf, ctot


def solve(grid: dict, q, mat, faces, n_bundles: int, seed: int = 1, nb: int = 1000, T_cells=None, T_ref=300.0,
          p_specular=None, L_b=0.0, n_e=0.0, elec=None, substrate=None, max_segments=10_000_000, first=0,
          threads: int = 1) -> dict:
    """Steady temperature rise (K) per subcell for heat q (W/m^3 per subcell,
    either sign)
    on the grid of ``grid`` (nx, ny, nz, Lx, Ly, Lz in m).  faces: six face
    kinds (x=0, x=Lx, y=0, y=Ly, z=0, z=Lz).  T_cells: the temperatures of the
    scattering rates (default T_ref everywhere)."""
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    Cn = nx * ny * nz
    q = np.asarray(q, dtype=float).reshape(Cn)
    T_cells = np.full(Cn, float(T_ref)) if T_cells is None else np.asarray(T_cells, dtype=float).reshape(Cn)
    tix, rate, cdf, ctot = tables(mat, nb, T_cells, L_b, n_e, elec)
    _, w, v, _ = bins(mat, nb)
    vg = v * 1e-3
    tau12 = np.array([TH.tau12(x, mat, substrate) for x in w]) if substrate is not None else np.zeros(nb)
    Vc = grid["Lx"] * grid["Ly"] * grid["Lz"] / Cn
    aq = np.abs(q)
    if not np.all(np.isfinite(q)) or not aq.sum() > 0:
        raise ValueError("need finite heat, not all zero")
    ccdf = np.cumsum(aq) / aq.sum()
    ccdf[-1] = 1.0
    sign = np.where(q < 0, -1.0, 1.0)
    P = Problem()
    P.nx, P.ny, P.nz, P.nb, P.nt = nx, ny, nz, nb, rate.shape[0]
    P.Lx, P.Ly, P.Lz = grid["Lx"] * 1e9, grid["Ly"] * 1e9, grid["Lz"] * 1e9
    keep = [np.ascontiguousarray(a) for a in (vg, rate, cdf, ccdf, tau12, sign)]
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    P.vg, P.rate, P.cdf, P.cell_cdf, P.tau12, P.cell_sign = [dp(a) for a in keep]
    P.tix = tix.ctypes.data_as(C.POINTER(C.c_int32))
    P.face[:] = list(faces)
    P.p_specular[:] = list(p_specular) if p_specular is not None else [0.0] * 6
    P.seed = seed & 0xFFFFFFFF
    P.max_segments = int(max_segments)
    threads = max(1, int(threads))
    parts = np.array_split(np.arange(first, first + n_bundles), threads)
    outs = []
    for part in parts:
        t = {"t_res": np.zeros(Cn), "scat": np.zeros(Cn, np.uint64), "emit": np.zeros(Cn, np.uint64)}
        T = Tally()
        T.t_res = dp(t["t_res"])
        T.scatterings = t["scat"].ctypes.data_as(C.POINTER(C.c_uint64))
        T.emitted = t["emit"].ctypes.data_as(C.POINTER(C.c_uint64))
        t["T"] = T
        t["range"] = (int(part[0]), int(part.size)) if part.size else (first, 0)
        outs.append(t)
    L = _lib()

    def work(t):
        L.ph_run(C.byref(P), t["range"][0], t["range"][1], C.byref(t["T"]))

    if threads == 1:
        work(outs[0])
    else:
        with ThreadPoolExecutor(threads) as ex:  # ctypes releases the GIL during the call
            list(ex.map(work, outs))
    t_res = sum(t["t_res"] for t in outs)
    scat = sum(t["scat"] for t in outs)
    emit = sum(t["emit"] for t in outs)
    absorbed = np.sum([np.array(t["T"].absorbed[:], dtype=np.uint64) for t in outs], axis=0)
    power = float(aq.sum() * Vc)
    dT = power * (t_res * 1e-12) / n_bundles / (ctot[tix] * Vc)
    return {"dT": dT, "t_res_ps": t_res, "scatterings": scat, "emitted": emit, "absorbed": absorbed,
            "segments": int(sum(t["T"].segments for t in outs)), "capped": int(sum(t["T"].capped for t in outs)),
            "power_W": power, "C_tot": ctot[tix]}
