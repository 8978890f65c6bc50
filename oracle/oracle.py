"""ctypes wrapper of the FP64 CPU oracle (``emc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports this module, and this module never imports the
product package; both take the plain configuration dicts of ``workloads.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "emc_oracle.c"), os.path.join(HERE, "phonon_oracle.c")]
HDR = [os.path.join(HERE, "emc_oracle.h"), os.path.join(HERE, "phonon_oracle.h")]
NV, NM = 3, 10

Q_E = 1.602176634e-19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree;
    OpenMP for the optional particle-parallel loop, one thread by default)."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in SRC + HDR)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fopenmp", "-o", tmp] + SRC + ["-lm"])
        os.replace(tmp, LIB)
    return LIB


class OrcConfig(C.Structure):
    _fields_ = [
        ("m_rel", C.c_double * 3), ("Ec_eV", C.c_double * 3), ("alpha_per_eV", C.c_double * 3),
        ("eps_s", C.c_double), ("eps_inf", C.c_double), ("rho", C.c_double),
        ("Da_eV", C.c_double), ("Dij_eV_per_m", C.c_double), ("hw_lo_eV", C.c_double),
        ("hw_iv_eV", C.c_double), ("vs", C.c_double),
        ("T", C.c_double), ("Nd", C.c_double), ("field", C.c_double * 3), ("dt", C.c_double),
        ("dE_eV", C.c_double), ("emax_init_kT", C.c_double),
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("gate_x0", C.c_double), ("gate_x1", C.c_double),
        ("Vs", C.c_double), ("Vd", C.c_double), ("Vg", C.c_double), ("p_spec", C.c_double),
        ("const_rate", C.c_double),
        ("n_particles", C.c_int64), ("capacity", C.c_int64),
        ("Z", C.c_int32 * 3), ("geometry", C.c_int32), ("n_bins", C.c_int32),
        ("steps_per_poisson", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("gate_on", C.c_int32),
        ("seed", C.c_uint32), ("mech_mask", C.c_uint32),
        ("exact_rates", C.c_int32), ("pad_", C.c_int32),
    ]


class OrcTallies(C.Structure):
    _fields_ = [
        ("self_events", C.c_uint64 * NV), ("overflow", C.c_uint64), ("rejected", C.c_uint64),
        ("crossings", C.c_int64 * 4), ("valley_steps", C.c_int64 * NV),
        ("n_samples", C.c_int64), ("steps_done", C.c_int64), ("n_alive", C.c_int64),
        ("inject_starved", C.c_int64),
        ("sum_v", C.c_double * 3), ("sum_E", C.c_double), ("sum_Etot", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_u01.argtypes = [C.c_uint32]
        L.orc_u01.restype = C.c_double
        L.orc_create.argtypes = [C.POINTER(OrcConfig)]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_ncell.argtypes = [P]
        L.orc_ncell.restype = C.c_int
        L.orc_rate.argtypes = [P, C.c_int, C.c_int, C.c_double]
        L.orc_rate.restype = C.c_double
        L.orc_get_tables.argtypes = [P, dp, dp]
        L.orc_run.argtypes = [P, C.c_int64]
        L.orc_set_threads.argtypes = [P, C.c_int]
        L.orc_test_drift.argtypes = [P, C.c_int, dp, dp, dp, C.c_double, dp, dp]
        L.orc_test_walls.argtypes = [P, dp, dp, C.c_uint64, dp, dp, C.POINTER(C.c_uint64)]
        L.orc_test_walls.restype = C.c_int
        L.orc_get_tallies.argtypes = [P, C.POINTER(OrcTallies)]
        L.orc_get_events.argtypes = [P, C.POINTER(C.c_uint64)]
        L.orc_get_charge.argtypes = [P, C.POINTER(C.c_int64)]
        L.orc_get_phi.argtypes = [P, dp, dp]
        L.orc_get_particles.argtypes = [P, dp, dp, dp, C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                        C.POINTER(C.c_uint64)]
        L.orc_set_bias.argtypes = [P, C.c_double, C.c_double, C.c_double]
        L.orc_set_temperature.argtypes = [P, dp, C.c_int]
        L.orc_sample_initial_energy.argtypes = [P, C.c_int64, dp]
        L.orc_cos_pop.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_cos_pop.restype = C.c_double
        L.orc_cos_imp.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_cos_imp.restype = C.c_double
        L.orc_rotate.argtypes = [dp, C.c_double, C.c_double, dp]
        L.orc_poisson.argtypes = [C.POINTER(OrcConfig), dp, dp, C.c_double, C.c_int]
        L.orc_poisson.restype = C.c_int
        L.orc_poisson_apply.argtypes = [C.POINTER(OrcConfig), dp, dp]
        L.orc_field.argtypes = [C.POINTER(OrcConfig), dp, dp]
        _lib = L
    return _lib


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def make_config(d: dict) -> OrcConfig:
    c = OrcConfig()
    c.m_rel[:] = d["m_rel"]
    c.Ec_eV[:] = d["Ec_eV"]
    c.alpha_per_eV[:] = d["alpha_per_eV"]
    c.eps_s, c.eps_inf, c.rho = d["eps_s"], d["eps_inf"], d["rho_kg_m3"]
    c.Da_eV, c.Dij_eV_per_m = d["Da_eV"], d["Dij_eV_per_m"]
    c.hw_lo_eV, c.hw_iv_eV, c.vs = d["hw_lo_eV"], d["hw_iv_eV"], d["vs_m_s"]
    c.T, c.Nd = d["T"], d["Nd"]
    c.field[:] = d["field"]
    c.dt, c.dE_eV, c.emax_init_kT = d["dt"], d["dE_eV"], d["emax_init_kT"]
    c.Lx, c.Ly, c.Lz = d["Lx"], d["Ly"], d["Lz"]
    c.gate_x0, c.gate_x1 = d["gate_x0"], d["gate_x1"]
    c.Vs, c.Vd, c.Vg, c.p_spec = d["Vs"], d["Vd"], d["Vg"], d["p_specular"]
    c.n_particles, c.capacity = d["n_particles"], d["capacity"]
    c.Z[:] = d["Z"]
    c.geometry, c.n_bins, c.steps_per_poisson = d["geometry"], d["n_bins"], d["steps_per_poisson"]
    c.nx, c.ny, c.nz, c.gate_on = d["nx"], d["ny"], d["nz"], d["gate_on"]
    c.seed = d["seed"] & 0xFFFFFFFF
    c.mech_mask = d.get("mech_mask", 0x3FF)
    c.const_rate = d.get("const_rate", 0.0)
    c.exact_rates = int(d.get("exact_rates", 0))
    return c


def philox(ctr, key) -> tuple:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


def u01(x: int) -> float:
    return lib().orc_u01(x)


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class Sim:
    """One ensemble simulated by the oracle.  threads > 1 runs the particle
    loop on that many threads (integer tallies are the same for any count)."""

    def __init__(self, cfg: dict, threads: int = 1):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.h = lib().orc_create(C.byref(self._c))
        self.ncell = lib().orc_ncell(self.h)
        self.nb = cfg["n_bins"]
        self.cap = max(cfg["capacity"], cfg["n_particles"])
        self.threads = 1
        if threads != 1:
            self.set_threads(threads)

    def set_threads(self, n: int):
        self.threads = max(1, int(n))
        lib().orc_set_threads(self.h, self.threads)

    def test_drift(self, valley: int, k0, r0, F, t: float):
        """One free flight of a lone electron (test hook; overwrites slot 0)."""
        k0 = np.ascontiguousarray(k0, dtype=float); r0 = np.ascontiguousarray(r0, dtype=float)
        F = np.ascontiguousarray(F, dtype=float)
        k1 = np.zeros(3); r1 = np.zeros(3)
        lib().orc_test_drift(self.h, int(valley), _ptr(k0), _ptr(r0), _ptr(F), float(t), _ptr(k1), _ptr(r1))
        return k1, r1

    def test_walls(self, r0, k0, ctr: int):
        """The walls and contacts applied to a lone electron (test hook;
        overwrites slot 0): (absorbed, r1, k1, counter after)."""
        r0 = np.ascontiguousarray(r0, dtype=float); k0 = np.ascontiguousarray(k0, dtype=float)
        r1 = np.zeros(3); k1 = np.zeros(3); c1 = C.c_uint64()
        out = lib().orc_test_walls(self.h, _ptr(r0), _ptr(k0), int(ctr), _ptr(r1), _ptr(k1), C.byref(c1))
        return bool(out), r1, k1, int(c1.value)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def rate(self, valley: int, mech: int, E_eV: float) -> float:
        return lib().orc_rate(self.h, valley, mech, E_eV * Q_E)

    def tables(self):
        t = np.zeros((NV, self.nb, NM))
        g = np.zeros(NV)
        lib().orc_get_tables(self.h, _ptr(t), _ptr(g))
        return t, g

    def run(self, n_steps: int):
        lib().orc_run(self.h, int(n_steps))

    def set_bias(self, Vs, Vd, Vg):
        lib().orc_set_bias(self.h, Vs, Vd, Vg)

    def set_temperature(self, T_cells):
        T = np.ascontiguousarray(np.atleast_1d(T_cells), dtype=np.float64)
        lib().orc_set_temperature(self.h, _ptr(T), int(T.size))

    def tallies(self) -> dict:
        t = OrcTallies()
        lib().orc_get_tallies(self.h, C.byref(t))
        ev = np.zeros((self.ncell, NV, NM), dtype=np.uint64)
        lib().orc_get_events(self.h, _ptr(ev, C.c_uint64))
        ch = np.zeros(self.ncell, dtype=np.int64)
        lib().orc_get_charge(self.h, _ptr(ch, C.c_int64))
        return {
            "events": ev,
            "self_events": np.array(t.self_events[:], dtype=np.uint64),
            "overflow": int(t.overflow), "rejected": int(t.rejected),
            "crossings": np.array(t.crossings[:], dtype=np.int64),
            "valley_steps": np.array(t.valley_steps[:], dtype=np.int64),
            "n_samples": int(t.n_samples), "steps_done": int(t.steps_done),
            "n_alive": int(t.n_alive), "inject_starved": int(t.inject_starved),
            "sum_v": np.array(t.sum_v[:]), "sum_E": float(t.sum_E), "sum_Etot": float(t.sum_Etot),
            "charge": ch,
        }

    def phi(self):
        phi = np.zeros(self.ncell)
        Ef = np.zeros((self.ncell, 3))
        lib().orc_get_phi(self.h, _ptr(phi), _ptr(Ef))
        return phi, Ef

    def particles(self) -> dict:
        n = self.cap
        k = np.zeros((n, 3)); r = np.zeros((n, 3)); tr = np.zeros(n)
        v = np.zeros(n, dtype=np.int32); a = np.zeros(n, dtype=np.uint8); ctr = np.zeros(n, dtype=np.uint64)
        lib().orc_get_particles(self.h, _ptr(k), _ptr(r), _ptr(tr), _ptr(v, C.c_int32),
                                _ptr(a, C.c_uint8), _ptr(ctr, C.c_uint64))
        return {"k": k, "r": r, "tr": tr, "valley": v, "alive": a, "ctr": ctr}

    def initial_energies(self, n: int) -> np.ndarray:
        E = np.zeros(n)
        lib().orc_sample_initial_energy(self.h, n, _ptr(E))
        return E

    def observables(self) -> dict:
        return observables(self.cfg, self.tallies())


def observables(cfg: dict, t: dict) -> dict:
    """Drift velocity along -F (bulk; m/s), mean kinetic energy (eV), valley
    fractions, all averaged over the sampled particle-steps."""
    n = max(t["n_samples"], 1)
    F = np.asarray(cfg["field"], dtype=float)
    Fm = np.linalg.norm(F)
    vd = float(-(t["sum_v"] @ F) / Fm / n) if Fm > 0 else 0.0
    return {
        "v_drift": vd,
        "v_mean": t["sum_v"] / n,
        "E_mean_eV": t["sum_E"] / n / Q_E,
        "Etot_mean_eV": t["sum_Etot"] / n / Q_E,
        "valley_frac": t["valley_steps"] / n,
    }


def poisson(cfg: dict, rho: np.ndarray | None, phi0: np.ndarray | None = None,
            tol: float = 1e-14, maxit: int = 200000) -> np.ndarray:
    c = make_config(cfg)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    phi = np.zeros(n) if phi0 is None else np.array(phi0, dtype=float).copy()
    r = None if rho is None else np.ascontiguousarray(rho, dtype=float)
    it = lib().orc_poisson(C.byref(c), _ptr(r) if r is not None else None, _ptr(phi), tol, maxit)
    if it < 0:
        raise RuntimeError("oracle Poisson CG did not converge")
    return phi


def poisson_apply(cfg: dict, phi: np.ndarray) -> np.ndarray:
    c = make_config(cfg)
    p = np.ascontiguousarray(phi, dtype=float)
    out = np.zeros_like(p)
    lib().orc_poisson_apply(C.byref(c), _ptr(p), _ptr(out))
    return out


def field(cfg: dict, phi: np.ndarray) -> np.ndarray:
    c = make_config(cfg)
    p = np.ascontiguousarray(phi, dtype=float)
    Ef = np.zeros((p.size, 3))
    lib().orc_field(C.byref(c), _ptr(p), _ptr(Ef))
    return Ef


def rotate(n, ct: float, ph: float) -> np.ndarray:
    a = np.ascontiguousarray(n, dtype=float)
    out = np.zeros(3)
    lib().orc_rotate(_ptr(a), ct, ph, _ptr(out))
    return out


def cos_pop(k: float, kp: float, u: float) -> float:
    return lib().orc_cos_pop(k, kp, u)


def cos_imp(k: float, beta2: float, u: float) -> float:
    return lib().orc_cos_imp(k, beta2, u)
