"""Thin ctypes binding of libemc (include/emc.h).

Argument marshalling only: every step of the Monte Carlo runs in the CUDA
kernels of ``libemc.so``.  The library must have been built (``build.build()``)
and a CUDA device must be present; there is no CPU fallback, and a missing
library raises at import of the context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# EMC_LIBRARY selects another build of the same library (the checked build
# of build.build(checked=True)); it must be set before the first call
LIB_PATH = os.environ.get("EMC_LIBRARY") or os.path.join(HERE, "_build", "libemc.so")

NV, NM = 3, 10
GEOM_BULK, GEOM_NANOWIRE = 0, 1
FP32, FP64 = 0, 1
TALLY_OBS, TALLY_EVENTS, TALLY_HEAT, TALLY_CHARGE = 0, 1, 2, 3
TALLY_CROSSINGS, TALLY_PHI, TALLY_FIELD, TALLY_HEAT_J = 4, 5, 6, 7
TALLY_EVENTS_CELL = 8
STATUS = {0: "EMC_OK", 1: "EMC_EINVAL", 2: "EMC_ENOMEM", 3: "EMC_ECUDA", 4: "EMC_EOVERFLOW",
          5: "EMC_ETIMEOUT", 6: "EMC_ESTATE"}


class EmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class EmcConfig(C.Structure):
    _fields_ = [
        ("m_rel", C.c_double * 3), ("Ec_eV", C.c_double * 3), ("alpha_per_eV", C.c_double * 3),
        ("eps_s", C.c_double), ("eps_inf", C.c_double), ("rho_kg_m3", C.c_double),
        ("Da_eV", C.c_double), ("Dij_eV_per_m", C.c_double),
        ("hw_lo_eV", C.c_double), ("hw_iv_eV", C.c_double), ("vs_m_s", C.c_double),
        ("T_K", C.c_double), ("Nd_m3", C.c_double), ("field_V_m", C.c_double * 3),
        ("dt_s", C.c_double), ("dE_eV", C.c_double), ("emax_init_kT", C.c_double),
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("gate_x0", C.c_double), ("gate_x1", C.c_double),
        ("Vs", C.c_double), ("Vd", C.c_double), ("Vg", C.c_double), ("p_specular", C.c_double),
        ("n_particles", C.c_int64), ("capacity", C.c_int64),
        ("shard_n_global", C.c_int64), ("shard_live_base", C.c_int64), ("shard_spare_base", C.c_int64),
        ("Z", C.c_int32 * 3), ("geometry", C.c_int32), ("n_bins", C.c_int32),
        ("steps_per_poisson", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("gate_on", C.c_int32), ("seed", C.c_uint32), ("mech_mask", C.c_uint32),
        ("precision", C.c_int32), ("sort_period", C.c_int32), ("block_size", C.c_int32),
        ("steps_per_launch", C.c_int32), ("table_smem_kb", C.c_int32),
    ]


class EmcObs(C.Structure):
    _fields_ = [
        ("sum_v", C.c_double * 3), ("sum_E", C.c_double), ("sum_Etot", C.c_double),
        ("n_samples", C.c_int64), ("valley_steps", C.c_int64 * 3), ("self_events", C.c_int64 * 3),
        ("overflow", C.c_int64), ("steps_done", C.c_int64), ("n_alive", C.c_int64),
        ("inject_starved", C.c_int64),
    ]


_lib = None


def lib():
    """Load libemc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libemc.so not built at {LIB_PATH}; run paper_1707_09073_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
        dp = C.POINTER(C.c_double)
        L.emc_init.argtypes = [C.POINTER(EmcConfig), P, C.POINTER(P)]
        L.emc_batch_init.argtypes = [C.POINTER(EmcConfig), I32, P, C.POINTER(P)]
        L.emc_step.argtypes = [P, I32]
        L.emc_tally.argtypes = [P, I32, P, C.c_size_t, I32, I32]
        L.emc_tally_async.argtypes = [P, I32, P, C.c_size_t, I32, I32]
        L.poisson_solve.argtypes = [P, dp, dp, dp]
        L.emc_poisson_solve_static.argtypes = [P, dp, dp, dp]
        L.emc_set_bias.argtypes = [P, I32, C.c_double, C.c_double, C.c_double]
        L.emc_set_bias_all.argtypes = [P, dp]
        L.emc_set_temperature.argtypes = [P, I32, dp, I32]
        L.emc_state_size.argtypes = [P, C.POINTER(C.c_size_t)]
        L.emc_get_state.argtypes = [P, P, C.c_size_t]
        L.emc_set_state.argtypes = [P, P, C.c_size_t]
        L.emc_shard_counts.argtypes = [P, P, P]
        L.emc_shard_tail.argtypes = [P, P, P, P, I32]
        L.emc_profile.argtypes = [P, I32]
        L.emc_profile_read.argtypes = [P, dp, C.POINTER(I64)]
        L.emc_debug_philox.argtypes = [P, C.POINTER(U32), C.POINTER(U32), C.POINTER(U32), I32]
        L.emc_debug_particles.argtypes = [P, dp, dp, dp, C.POINTER(I32), C.POINTER(I32), C.POINTER(U32),
                                          C.POINTER(C.c_uint64)]
        L.emc_debug_tables.argtypes = [P, I32, dp, dp]
        L.emc_shape.argtypes = [P, C.POINTER(I32), C.POINTER(I64), C.POINTER(I32)]
        L.emc_launch_count.argtypes = [P]
        L.emc_launch_count.restype = I64
        L.emc_last_error.argtypes = [P]
        L.emc_last_error.restype = C.c_char_p
        L.emc_destroy.argtypes = [P]
        for f in ("emc_init", "emc_batch_init", "emc_step", "emc_tally", "emc_tally_async", "poisson_solve",
                  "emc_poisson_solve_static", "emc_set_bias",
                  "emc_set_bias_all", "emc_set_temperature", "emc_profile", "emc_profile_read",
                  "emc_debug_philox", "emc_debug_particles", "emc_debug_tables", "emc_shape",
                  "emc_state_size", "emc_get_state", "emc_set_state", "emc_shard_counts", "emc_shard_tail"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def make_config(d: dict, precision: int = FP32) -> EmcConfig:
    """Marshal a plain configuration dict (keys of ``workloads.py``) into the C struct."""
    c = EmcConfig()
    c.m_rel[:] = d["m_rel"]
    c.Ec_eV[:] = d["Ec_eV"]
    c.alpha_per_eV[:] = d["alpha_per_eV"]
    c.eps_s, c.eps_inf, c.rho_kg_m3 = d["eps_s"], d["eps_inf"], d["rho_kg_m3"]
    c.Da_eV, c.Dij_eV_per_m = d["Da_eV"], d["Dij_eV_per_m"]
    c.hw_lo_eV, c.hw_iv_eV, c.vs_m_s = d["hw_lo_eV"], d["hw_iv_eV"], d["vs_m_s"]
    c.T_K, c.Nd_m3 = d["T"], d["Nd"]
    c.field_V_m[:] = d["field"]
    c.dt_s, c.dE_eV, c.emax_init_kT = d["dt"], d["dE_eV"], d["emax_init_kT"]
    c.Lx, c.Ly, c.Lz = d["Lx"], d["Ly"], d["Lz"]
    c.gate_x0, c.gate_x1 = d["gate_x0"], d["gate_x1"]
    c.Vs, c.Vd, c.Vg, c.p_specular = d["Vs"], d["Vd"], d["Vg"], d["p_specular"]
    c.n_particles, c.capacity = int(d["n_particles"]), int(d["capacity"])
    c.shard_n_global = int(d.get("shard_n_global", 0))
    c.shard_live_base = int(d.get("shard_live_base", 0))
    c.shard_spare_base = int(d.get("shard_spare_base", 0))
    c.Z[:] = d["Z"]
    c.geometry, c.n_bins, c.steps_per_poisson = d["geometry"], d["n_bins"], d["steps_per_poisson"]
    c.nx, c.ny, c.nz, c.gate_on = d["nx"], d["ny"], d["nz"], d["gate_on"]
    c.seed = d["seed"] & 0xFFFFFFFF
    c.mech_mask = d.get("mech_mask", 0x3FF)
    c.precision = d.get("precision", precision)
    c.sort_period = d.get("sort_period", 0)
    c.block_size = d.get("block_size", 0)
    c.steps_per_launch = d.get("steps_per_launch", 0)
    c.table_smem_kb = d.get("table_smem_kb", 0)
    return c


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


class Context:
    """One libemc context holding one or more ensembles (``emc_batch_init``).

    ``stream`` is a CUDA stream handle (int) or None for the default stream;
    with PyTorch pass ``torch.cuda.current_stream().cuda_stream``."""

    def __init__(self, cfgs, precision: int = FP32, stream=None):
        if isinstance(cfgs, dict):
            cfgs = [cfgs]
        self.cfgs = [dict(c) for c in cfgs]
        arr = (EmcConfig * len(cfgs))(*[make_config(c, precision) for c in cfgs])
        self._arr = arr
        self._pinned = []  # page-locked buffers handed out by pinned_tally
        self.h = C.c_void_p()
        st = lib().emc_batch_init(arr, len(cfgs), C.c_void_p(stream or 0), C.byref(self.h))
        if st != 0:
            msg = lib().emc_last_error(self.h).decode() if self.h else ""
            self.close()
            raise EmcError(st, msg)
        ne, cap, nc = C.c_int32(), C.c_int64(), C.c_int32()
        self._check(lib().emc_shape(self.h, C.byref(ne), C.byref(cap), C.byref(nc)))
        self.n_ens, self.capacity, self.n_cell = ne.value, cap.value, nc.value

    def _check(self, st: int):
        if st != 0:
            raise EmcError(st, lib().emc_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().emc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- C-ABI names ---------------------------------------------------------
    def emc_step(self, n_steps: int):
        self._check(lib().emc_step(self.h, int(n_steps)))

    def _tally_spec(self, kind: int):
        E, Cc = self.n_ens, self.n_cell
        return {
            TALLY_OBS: (OBS_DTYPE, (E,)),
            TALLY_EVENTS: (np.dtype(np.uint64), (E, NV, NM)),
            TALLY_HEAT: (np.dtype(np.int64), (E, Cc, 2)),
            TALLY_CHARGE: (np.dtype(np.int64), (E, Cc)),
            TALLY_CROSSINGS: (np.dtype(np.int64), (E, 4)),
            TALLY_PHI: (np.dtype(np.float64), (E, Cc)),
            TALLY_FIELD: (np.dtype(np.float64), (E, Cc, 3)),
            TALLY_HEAT_J: (np.dtype(np.float64), (E, Cc)),
            TALLY_EVENTS_CELL: (np.dtype(np.uint64), (E, Cc, NV, NM)),
        }[kind]

    def pinned_tally(self, kind: int) -> np.ndarray:
        """A page-locked host array of tally `kind`'s shape and type (OBS:
        structured array like obs_buffer) for emc_tally_async."""
        import torch
        dt, shape = self._tally_spec(kind)
        n = int(np.prod(shape)) * dt.itemsize
        t = torch.empty(n, dtype=torch.uint8).pin_memory()
        self._pinned.append(t)
        return t.numpy().view(dt).reshape(shape)

    def emc_tally_async(self, kind: int, out, reset: bool = False, device: bool = False):
        """Enqueue tally `kind` into ``out`` (page-locked host array from
        pinned_tally, or with ``device=True`` a device pointer) without
        waiting; read it after synchronising the stream (or an event recorded
        after this call)."""
        dt, shape = self._tally_spec(kind)
        nbytes = int(np.prod(shape)) * dt.itemsize
        if device:
            self._check(lib().emc_tally_async(self.h, kind, C.c_void_p(int(out)), nbytes, 1, int(reset)))
        else:
            if out.nbytes < nbytes or out.dtype != dt:
                raise ValueError("out must be pinned_tally(kind) of this context")
            self._check(lib().emc_tally_async(self.h, kind, out.ctypes.data_as(C.c_void_p), out.nbytes, 0, int(reset)))
        return out

    def obs_buffer(self) -> np.ndarray:
        """A structured array [n_ens] (fields as in emc_obs) for
        emc_tally(TALLY_OBS, out=...): the fast path for per-step reads."""
        return np.zeros(self.n_ens, dtype=OBS_DTYPE)

    def emc_tally(self, kind: int, reset: bool = False, out=None, device: bool = False):
        """Copy a tally (numpy array on the host, or into ``out`` when given:
        a numpy array, or with ``device=True`` a device pointer (int) of at
        least the tally's size in bytes)."""
        E, Cc = self.n_ens, self.n_cell
        spec = {
            TALLY_OBS: (EmcObs * E, None),
            TALLY_EVENTS: (np.uint64, (E, NV, NM)),
            TALLY_HEAT: (np.int64, (E, Cc, 2)),
            TALLY_CHARGE: (np.int64, (E, Cc)),
            TALLY_CROSSINGS: (np.int64, (E, 4)),
            TALLY_PHI: (np.float64, (E, Cc)),
            TALLY_FIELD: (np.float64, (E, Cc, 3)),
            TALLY_HEAT_J: (np.float64, (E, Cc)),
            TALLY_EVENTS_CELL: (np.uint64, (E, Cc, NV, NM)),
        }[kind]
        if device:
            nbytes = C.sizeof(spec[0]) if kind == TALLY_OBS else int(np.prod(spec[1])) * np.dtype(spec[0]).itemsize
            self._check(lib().emc_tally(self.h, kind, C.c_void_p(int(out)), nbytes, 1, int(reset)))
            return out
        if kind == TALLY_OBS:
            if out is not None:
                # preallocated structured array (obs_buffer()): filled in place,
                # no per-ensemble Python objects
                if out.dtype != OBS_DTYPE or out.size != E:
                    raise ValueError("out must be obs_buffer() of this context")
                self._check(lib().emc_tally(self.h, kind, out.ctypes.data_as(C.c_void_p), out.nbytes, 0, int(reset)))
                return out
            buf = spec[0]()
            self._check(lib().emc_tally(self.h, kind, C.byref(buf), C.sizeof(buf), 0, int(reset)))
            return [obs_dict(buf[e]) for e in range(E)]
        a = np.zeros(spec[1], dtype=spec[0]) if out is None else out
        self._check(lib().emc_tally(self.h, kind, a.ctypes.data_as(C.c_void_p), a.nbytes, 0, int(reset)))
        return a

    def poisson_solve(self, charge=None, bc_volts=(0.0, 0.0, 0.0)):
        bc = np.ascontiguousarray(bc_volts, dtype=np.float64)
        phi = np.zeros(self.n_cell)
        ch = None if charge is None else np.ascontiguousarray(charge, dtype=np.float64)
        self._check(lib().poisson_solve(self.h, _p(ch) if ch is not None else None, _p(bc), _p(phi)))
        return phi

    def emc_poisson_solve_static(self, charge=None, bc_volts=(0.0, 0.0, 0.0)):
        """poisson_solve without device allocation (library-owned static scratch,
        at most 8192 subcells; calls must not overlap on the GPU)."""
        bc = np.ascontiguousarray(bc_volts, dtype=np.float64)
        phi = np.zeros(self.n_cell)
        ch = None if charge is None else np.ascontiguousarray(charge, dtype=np.float64)
        self._check(lib().emc_poisson_solve_static(self.h, _p(ch) if ch is not None else None, _p(bc), _p(phi)))
        return phi

    def emc_set_bias(self, ens: int, Vs: float, Vd: float, Vg: float):
        self._check(lib().emc_set_bias(self.h, int(ens), Vs, Vd, Vg))

    def emc_set_bias_all(self, bias_ptr_or_array):
        """bias: host float64 [E][3] (numpy array, or an int address of pinned memory)."""
        if isinstance(bias_ptr_or_array, int):
            self._check(lib().emc_set_bias_all(self.h, C.cast(C.c_void_p(bias_ptr_or_array), C.POINTER(C.c_double))))
        else:
            b = np.ascontiguousarray(bias_ptr_or_array, dtype=np.float64).reshape(self.n_ens, 3)
            self._check(lib().emc_set_bias_all(self.h, _p(b)))

    def emc_set_temperature(self, ens: int, T_cells):
        """Lattice temperature (K) of every subcell of ensemble `ens`."""
        T = np.ascontiguousarray(np.atleast_1d(T_cells), dtype=np.float64)
        self._check(lib().emc_set_temperature(self.h, int(ens), _p(T), int(T.size)))

    def emc_get_state(self) -> np.ndarray:
        """The whole simulation state as a byte array (emc_get_state)."""
        n = C.c_size_t()
        self._check(lib().emc_state_size(self.h, C.byref(n)))
        out = np.zeros(n.value, dtype=np.uint8)
        self._check(lib().emc_get_state(self.h, out.ctypes.data_as(C.c_void_p), out.nbytes))
        return out

    def emc_set_state(self, blob):
        """Restore a state from emc_get_state of a context of the same ensembles."""
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        self._check(lib().emc_set_state(self.h, b.ctypes.data_as(C.c_void_p), b.nbytes))

    def emc_shard_counts(self):
        """(charge int32[E][C], free int64[E][2]) of a sharded context waiting
        for its exchange: its own electron count per subcell and its free ids
        among the initial-electron and the spare ids."""
        q = np.zeros((self.n_ens, self.n_cell), dtype=np.int32)
        f = np.zeros((self.n_ens, 2), dtype=np.int64)
        self._check(lib().emc_shard_counts(self.h, q.ctypes.data_as(C.c_void_p), f.ctypes.data_as(C.c_void_p)))
        return q, f

    def emc_shard_counts_ptr(self, charge_ptr: int, free_ptr: int):
        """emc_shard_counts into caller memory given by address (host or
        device: int32[E][C] and int64[E][2])."""
        self._check(lib().emc_shard_counts(self.h, C.c_void_p(int(charge_ptr)), C.c_void_p(int(free_ptr))))

    def emc_shard_tail_ptr(self, charge_ptr: int, prefix_ptr: int, total_ptr: int, lead: bool):
        """emc_shard_tail from caller memory given by address (host or device)."""
        self._check(lib().emc_shard_tail(self.h, C.c_void_p(int(charge_ptr)), C.c_void_p(int(prefix_ptr)),
                                         C.c_void_p(int(total_ptr)), int(bool(lead))))

    def emc_shard_tail(self, charge_global, free_prefix, free_total, lead: bool):
        """Refill and Poisson update of a sharded context from the wire's
        count (emc_shard_tail)."""
        q = np.ascontiguousarray(charge_global, dtype=np.int32).reshape(self.n_ens, self.n_cell)
        p = np.ascontiguousarray(free_prefix, dtype=np.int64).reshape(self.n_ens, 2)
        t = np.ascontiguousarray(free_total, dtype=np.int64).reshape(self.n_ens, 2)
        self._check(lib().emc_shard_tail(self.h, q.ctypes.data_as(C.c_void_p), p.ctypes.data_as(C.c_void_p),
                                         t.ctypes.data_as(C.c_void_p), int(bool(lead))))

    def emc_surrogate_train(self, net: "EmcMlpConfig", X, Y, steps, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999,
                            eps=1e-8, seed=0):
        """Create and train the context's surrogate (emc_surrogate_train);
        returns the loss history."""
        L = _surrogate_lib()
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        t = train_config(steps, batch, lr, beta1, beta2, eps, seed)
        hist = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(L.emc_surrogate_train(self.h, C.byref(net), _p(X, C.c_float), _p(Y, C.c_float), X.shape[0],
                                          C.byref(t), _p(hist, C.c_float)))
        self._sur_out = net.n_out
        return hist[:steps]

    def emc_surrogate_infer(self, X):
        L = _surrogate_lib()
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], getattr(self, "_sur_out", 16)), dtype=np.float32)
        self._check(L.emc_surrogate_infer(self.h, _p(X, C.c_float), _p(Y, C.c_float), X.shape[0]))
        return Y

    def emc_surrogate_params(self):
        L = _surrogate_lib()
        n = C.c_int64()
        self._check(L.emc_surrogate_params(self.h, None, C.byref(n)))
        out = np.zeros(n.value, dtype=np.float32)
        self._check(L.emc_surrogate_params(self.h, _p(out, C.c_float), C.byref(n)))
        return out

    def emc_profile(self, enable: bool):
        self._check(lib().emc_profile(self.h, int(enable)))

    def emc_profile_read(self):
        ms, n = C.c_double(), C.c_int64()
        self._check(lib().emc_profile_read(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def debug_philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
        out = np.zeros_like(ctr)
        self._check(lib().emc_debug_philox(self.h, _p(ctr, C.c_uint32), _p(key, C.c_uint32),
                                           _p(out, C.c_uint32), ctr.shape[0]))
        return out

    def debug_particles(self) -> dict:
        n = self.capacity
        k = np.zeros((n, 3)); r = np.zeros((n, 3)); tr = np.zeros(n)
        v = np.zeros(n, np.int32); e = np.zeros(n, np.int32); i = np.zeros(n, np.uint32); c = np.zeros(n, np.uint64)
        self._check(lib().emc_debug_particles(self.h, _p(k), _p(r), _p(tr), _p(v, C.c_int32), _p(e, C.c_int32),
                                              _p(i, C.c_uint32), _p(c, C.c_uint64)))
        return {"k": k, "r": r, "tr": tr, "valley": v, "ens": e, "id": i, "ctr": c}

    def debug_tables(self, ens: int = 0):
        nb = self.cfgs[ens]["n_bins"]
        t = np.zeros((NV, nb, NM)); g = np.zeros(NV)
        self._check(lib().emc_debug_tables(self.h, ens, _p(t), _p(g)))
        return t, g

    def launch_count(self) -> int:
        return int(lib().emc_launch_count(self.h))


# the observation tally as a numpy structured dtype (same layout as emc_obs)
OBS_DTYPE = np.dtype(EmcObs)


def group_step(ctxs, n_steps: int):
    """Advance one or two contexts (same stream, precision, block size) by
    n_steps together: one flight launch per chunk over both (emc_group_step)."""
    L = lib()
    if not getattr(L, "_group_ready", False):
        L.emc_group_step.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32]
        L.emc_group_step.restype = C.c_int
        L._group_ready = True
    hs = (C.c_void_p * len(ctxs))(*[c.h.value if hasattr(c.h, "value") else c.h for c in ctxs])
    ctxs[0]._check(L.emc_group_step(hs, len(ctxs), int(n_steps)))


def obs_dict(o: EmcObs) -> dict:
    return {
        "sum_v": np.array(o.sum_v[:]), "sum_E": o.sum_E, "sum_Etot": o.sum_Etot,
        "n_samples": o.n_samples, "valley_steps": np.array(o.valley_steps[:], dtype=np.int64),
        "self_events": np.array(o.self_events[:], dtype=np.int64), "overflow": o.overflow,
        "steps_done": o.steps_done, "n_alive": o.n_alive, "inject_starved": o.inject_starved,
    }


# ------------------------------------------------------------ thermal side
class EmcThermalConfig(C.Structure):
    _fields_ = [("T_sink", C.c_double), ("h_bottom", C.c_double), ("L_boundary", C.c_double), ("tol_K", C.c_double),
                ("k0_per_m", C.c_double), ("omega_max_rad_s", C.c_double), ("A_s3", C.c_double),
                ("B1_s_per_K", C.c_double), ("B2_K", C.c_double),
                ("n_e_m3", C.c_double), ("m_e_rel", C.c_double), ("Da_eV", C.c_double), ("rho_kg_m3", C.c_double),
                ("vg_e_m_s", C.c_double), ("max_picard", C.c_int32), ("max_cg", C.c_int32),
                ("interface_dmm", C.c_int32), ("pad_", C.c_int32), ("sub_k0_per_m", C.c_double),
                ("sub_omega_max_rad_s", C.c_double), ("interface_area_ratio", C.c_double)]


def thermal_config(table_ii: dict, T_sink=300.0, h_bottom=1e9, L_boundary=120e-9, tol_K=1e-6, max_picard=50,
                   max_cg=5000, n_e=0.0, elec: dict | None = None, substrate: dict | None = None,
                   area_ratio: float = 1.0) -> EmcThermalConfig:
    """Thermal-side parameters; n_e (m^-3) > 0 with elec = {m_rel, Da_eV,
    rho_kg_m3, vg_m_s} adds the phonon-electron scattering of Eq. (1);
    substrate (a Table II column) puts the diffuse-mismatch interface of
    Eqs. (2)-(3), times area_ratio, under the bottom face (in series with
    h_bottom; h_bottom <= 0: none)."""
    t = EmcThermalConfig()
    t.T_sink, t.h_bottom, t.L_boundary, t.tol_K = T_sink, h_bottom, L_boundary, tol_K
    t.k0_per_m, t.omega_max_rad_s = table_ii["k0_per_m"], table_ii["omega_max_rad_s"]
    t.A_s3, t.B1_s_per_K, t.B2_K = table_ii["A_s3"], table_ii["B1_s_per_K"], table_ii["B2_K"]
    if n_e > 0:
        if elec is None:
            raise ValueError("n_e > 0 needs the electron parameters")
        t.n_e_m3, t.m_e_rel, t.Da_eV = n_e, elec["m_rel"], elec["Da_eV"]
        t.rho_kg_m3, t.vg_e_m_s = elec["rho_kg_m3"], elec["vg_m_s"]
    t.max_picard, t.max_cg = max_picard, max_cg
    if substrate is not None:
        t.interface_dmm = 1
        t.sub_k0_per_m, t.sub_omega_max_rad_s = substrate["k0_per_m"], substrate["omega_max_rad_s"]
        t.interface_area_ratio = area_ratio
    return t


def _thermal_lib():
    L = lib()
    if not getattr(L, "_thermal_ready", False):
        dp = C.POINTER(C.c_double)
        L.emc_thermal_solve.argtypes = [C.c_void_p, C.POINTER(EmcThermalConfig), dp, dp, C.POINTER(C.c_int32)]
        L.emc_thermal_solve.restype = C.c_int
        L.emc_kappa.argtypes = [C.POINTER(EmcThermalConfig), dp, dp, C.c_int32]
        L.emc_kappa.restype = C.c_int
        for f in ("emc_dmm_transmissivity", "emc_interface_conductance"):
            getattr(L, f).argtypes = [C.POINTER(EmcThermalConfig), dp, dp, C.c_int32]
            getattr(L, f).restype = C.c_int
        L._thermal_ready = True
    return L


def kappa(tc: EmcThermalConfig, T) -> np.ndarray:
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    out = np.zeros_like(T)
    st = _thermal_lib().emc_kappa(C.byref(tc), _p(T), _p(out), T.size)
    if st != 0:
        raise EmcError(st, "emc_kappa")
    return out


def dmm_transmissivity(tc: EmcThermalConfig, omega) -> np.ndarray:
    """Eq. (2): wire -> substrate transmissivity at angular frequencies omega."""
    w = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
    out = np.zeros_like(w)
    st = _thermal_lib().emc_dmm_transmissivity(C.byref(tc), _p(w), _p(out), w.size)
    if st != 0:
        raise EmcError(st, "emc_dmm_transmissivity")
    return out


def interface_conductance(tc: EmcThermalConfig, T) -> np.ndarray:
    """Eq. (3): 1/R_K (W/m^2/K) per unit interface area at temperatures T."""
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    out = np.zeros_like(T)
    st = _thermal_lib().emc_interface_conductance(C.byref(tc), _p(T), _p(out), T.size)
    if st != 0:
        raise EmcError(st, "emc_interface_conductance")
    return out


def thermal_solve(ctx: "Context", tc: EmcThermalConfig, q, T0=None):
    """Temperature [E][C] of every ensemble of a nanowire context for heat
    generation q [E][C] (W/m^3)."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(ctx.n_ens, ctx.n_cell)
    T = np.full_like(q, tc.T_sink) if T0 is None else np.ascontiguousarray(T0, dtype=np.float64).copy()
    it = np.zeros((ctx.n_ens, 2), dtype=np.int32)
    ctx._check(_thermal_lib().emc_thermal_solve(ctx.h, C.byref(tc), _p(q), _p(T), _p(it, C.c_int32)))
    return T, it


# ------------------------------------------------------------ phonon MC
PH_SPECULAR, PH_ROUGH, PH_ISOTHERMAL, PH_INTERFACE = 0, 1, 2, 3
# the half wire: contacts isothermal, symmetry plane A specular, the outer
# side and the top rough, the bottom on the substrate's interface
WIRE_FACES = (PH_ISOTHERMAL, PH_ISOTHERMAL, PH_SPECULAR, PH_ROUGH, PH_INTERFACE, PH_ROUGH)


class EmcPhononConfig(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("face", C.c_int32 * 6), ("precision", C.c_int32),
                ("p_specular", C.c_double * 6), ("max_segments", C.c_int64), ("seed", C.c_uint32),
                ("block_size", C.c_int32)]


class EmcPhononTally(C.Structure):
    _fields_ = [("absorbed", C.c_uint64 * 6), ("segments", C.c_uint64), ("scatterings", C.c_uint64),
                ("capped", C.c_uint64), ("power_W", C.c_double), ("kernel_ms", C.c_double)]


def phonon_config(faces=WIRE_FACES, n_bins=1000, precision=FP32, p_specular=0.0, max_segments=10_000_000, seed=1,
                  block_size=0) -> EmcPhononConfig:
    pc = EmcPhononConfig()
    pc.n_bins = n_bins
    pc.face[:] = list(faces)
    pc.precision = precision
    pc.p_specular[:] = list(p_specular) if np.ndim(p_specular) else [float(p_specular)] * 6
    pc.max_segments, pc.seed, pc.block_size = int(max_segments), int(seed) & 0xFFFFFFFF, block_size
    return pc


def phonon_solve(ctx: "Context", tc: EmcThermalConfig, pc: EmcPhononConfig, q, n_bundles: int, T_cells=None,
                 first: int = 0) -> dict:
    """Phonon Monte Carlo of one wire of a nanowire context
    (emc_phonon_solve): temperature rise dT [C] (K) for heat q [C] (W/m^3),
    residence times, scatterings and emissions per subcell, the tally."""
    L = lib()
    if not getattr(L, "_phonon_ready", False):
        L.emc_phonon_solve.argtypes = [C.c_void_p, C.POINTER(EmcThermalConfig), C.POINTER(EmcPhononConfig),
                                       C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.POINTER(EmcPhononTally)]
        L.emc_phonon_solve.restype = C.c_int
        L._phonon_ready = True
    n = ctx.n_cell
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(n)
    Tc = None if T_cells is None else np.ascontiguousarray(T_cells, dtype=np.float64).reshape(n)
    dT, tr = np.zeros(n), np.zeros(n)
    sc, em = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    t = EmcPhononTally()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    ctx._check(L.emc_phonon_solve(ctx.h, C.byref(tc), C.byref(pc), vp(q), vp(Tc) if Tc is not None else None,
                                  int(n_bundles), int(first), vp(dT), vp(tr), vp(sc), vp(em), C.byref(t)))
    return {"dT": dT, "t_res_ps": tr, "scatterings": sc, "emitted": em, "absorbed": np.array(t.absorbed[:], np.uint64),
            "segments": int(t.segments), "n_scatterings": int(t.scatterings), "capped": int(t.capped),
            "power_W": t.power_W, "kernel_ms": t.kernel_ms}


# ------------------------------------------------------------ surrogate MLP
class EmcMlpConfig(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32), ("n_layers", C.c_int32), ("n_out", C.c_int32),
                ("x_shift", C.c_float * 16), ("x_scale", C.c_float * 16),
                ("y_shift", C.c_float * 16), ("y_scale", C.c_float * 16),
                ("seed", C.c_uint32), ("pad_", C.c_int32)]


class EmcTrainConfig(C.Structure):
    _fields_ = [("steps", C.c_int64), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint32), ("pad_", C.c_int32)]


def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        P, I64 = C.c_void_p, C.c_int64
        fp = C.POINTER(C.c_float)
        L.emc_mlp_create.argtypes = [C.POINTER(EmcMlpConfig), P, C.POINTER(P)]
        L.emc_mlp_train.argtypes = [P, fp, fp, I64, C.POINTER(EmcTrainConfig), fp]
        L.emc_mlp_infer.argtypes = [P, fp, fp, I64]
        L.emc_mlp_grad.argtypes = [P, fp, fp, I64, fp, fp]
        L.emc_mlp_params.argtypes = [P, fp, fp, C.POINTER(I64)]
        L.emc_mlp_last_error.argtypes = [P]
        L.emc_mlp_last_error.restype = C.c_char_p
        L.emc_mlp_destroy.argtypes = [P]
        L.emc_mlp_debug_set_error.argtypes = [P]
        L.emc_mlp_set_fused.argtypes = [P, C.c_int32]
        for f in ("emc_mlp_create", "emc_mlp_train", "emc_mlp_infer", "emc_mlp_grad", "emc_mlp_params",
                  "emc_mlp_debug_set_error", "emc_mlp_set_fused"):
            getattr(L, f).restype = C.c_int
        L._mlp_ready = True
    return L


def mlp_config(n_in, n_hidden, n_layers, n_out, x_shift, x_scale, y_shift, y_scale, seed=0) -> EmcMlpConfig:
    """The emc_mlp_config struct (unused normalisation slots: shift 0, scale 1)."""
    c = EmcMlpConfig()
    c.n_in, c.n_hidden, c.n_layers, c.n_out, c.seed = n_in, n_hidden, n_layers, n_out, seed
    for arr, vals in ((c.x_shift, x_shift), (c.x_scale, x_scale), (c.y_shift, y_shift), (c.y_scale, y_scale)):
        for i, v in enumerate(vals):
            arr[i] = float(v)
    for i in range(n_in, 16):
        c.x_scale[i] = 1.0
    for i in range(n_out, 16):
        c.y_scale[i] = 1.0
    return c


def train_config(steps, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0) -> EmcTrainConfig:
    t = EmcTrainConfig()
    t.steps, t.batch, t.lr, t.beta1, t.beta2, t.eps, t.seed = steps, batch, lr, beta1, beta2, eps, seed
    return t


def _surrogate_lib():
    L = _mlp_lib()
    if not getattr(L, "_sur_ready", False):
        P, I64 = C.c_void_p, C.c_int64
        fp = C.POINTER(C.c_float)
        L.emc_surrogate_train.argtypes = [P, C.POINTER(EmcMlpConfig), fp, fp, I64, C.POINTER(EmcTrainConfig), fp]
        L.emc_surrogate_infer.argtypes = [P, fp, fp, I64]
        L.emc_surrogate_params.argtypes = [P, fp, C.POINTER(I64)]
        for f in ("emc_surrogate_train", "emc_surrogate_infer", "emc_surrogate_params"):
            getattr(L, f).restype = C.c_int
        L._sur_ready = True
    return L


class Mlp:
    """The surrogate network of the C ABI (emc_mlp_*).  x_shift/x_scale and
    y_shift/y_scale normalise inputs and outputs inside the library."""

    def __init__(self, n_in, n_hidden, n_layers, n_out, x_shift, x_scale, y_shift, y_scale, seed=0, stream=None):
        c = mlp_config(n_in, n_hidden, n_layers, n_out, x_shift, x_scale, y_shift, y_scale, seed)
        self.cfg = c
        self.n_in, self.n_out = n_in, n_out
        self.h = C.c_void_p()
        st = _mlp_lib().emc_mlp_create(C.byref(c), C.c_void_p(stream or 0), C.byref(self.h))
        if st != 0:
            msg = _mlp_lib().emc_mlp_last_error(self.h).decode() if self.h else ""
            self.close()
            raise EmcError(st, msg)

    def _check(self, st):
        if st != 0:
            raise EmcError(st, _mlp_lib().emc_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            _mlp_lib().emc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def train(self, X, Y, steps, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        t = train_config(steps, batch, lr, beta1, beta2, eps, seed)
        hist = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(_mlp_lib().emc_mlp_train(self.h, _p(X, C.c_float), _p(Y, C.c_float), X.shape[0], C.byref(t),
                                             _p(hist, C.c_float)))
        return hist[:steps]

    def infer(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], self.n_out), dtype=np.float32)
        self._check(_mlp_lib().emc_mlp_infer(self.h, _p(X, C.c_float), _p(Y, C.c_float), X.shape[0]))
        return Y

    def set_fused(self, enable: bool = True):
        """Inference in one fused launch (default, when the network fits) or
        one launch per layer."""
        self._check(_mlp_lib().emc_mlp_set_fused(self.h, int(bool(enable))))

    def debug_set_error(self):
        """Set the device error word as an expired tensor-core wait would."""
        self._check(_mlp_lib().emc_mlp_debug_set_error(self.h))

    def grad(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.zeros(self.n_params(), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._check(_mlp_lib().emc_mlp_grad(self.h, _p(X, C.c_float), _p(Y, C.c_float), X.shape[0],
                                            _p(g, C.c_float), _p(loss, C.c_float)))
        return float(loss[0]), g

    def n_params(self) -> int:
        n = C.c_int64()
        self._check(_mlp_lib().emc_mlp_params(self.h, None, None, C.byref(n)))
        return n.value

    def params(self, new=None):
        n = self.n_params()
        out = np.zeros(n, dtype=np.float32)
        src = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
        cnt = C.c_int64()
        self._check(_mlp_lib().emc_mlp_params(self.h, _p(out, C.c_float), _p(src, C.c_float) if src is not None else None,
                                              C.byref(cnt)))
        return out
