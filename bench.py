#!/usr/bin/env python
"""Benchmark of the ensemble electron Monte Carlo (GaN half-nanowire FinFET).

Workload (default): the half-nanowire drain-bias sweep -- 21 bias points
V_ds = 0..20 V, each an ensemble of 200,000 superparticles in a 60 x 120 nm x
1 um half wire with 3 x 6 x 100 subcells, N_d = 1e18 cm^-3, 300 K, dt = 1 fs,
FP64 Poisson update every 10 fs -- all 21 ensembles advanced together by each
launch.  One benchmark step = one Poisson period (10 time steps) of every bias
point: flight/scatter/walls/tallies, contact refill, charge count, Poisson,
field.

Metric: real (non-self) electron scattering events per second, whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl emc|reference]

Under torchrun (N > 1) every rank runs its own sweep with its own seeds (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "electron scatter events/sec on 1 GB300 (% roofline); surrogate vs plain MC converge time"
UNIT = "events/s"
STEPS_PER_POISSON = 10
N_SM = 152
LANES_PER_SM = 128
# Algorithmic operation model of the flight kernel: lane operations (FP32,
# integer and special-function instructions of the method's arithmetic; no
# loads, stores, address arithmetic or loop control), counted from the
# kernel source for the nanowire geometry:
#   per particle-step 98: subcell lookup 14, drift 44 (k, Kane energy, two
#     group velocities, trapezoid + along-field correction, position), wall
#     and contact tests 10, step end 2, the compensated step sample 28;
#   per scattering (self or real) 133: another drift + wall test 54, Philox
#     4x32-10 60, four uniforms 12, energy bin 5, first table compare 2;
#   plus 6 for a self-scattering (tally, flight time) or 70 for a real one
#     (table scan, final energy and |k'|, angle law, sin/cos, orthonormal
#     basis and rotation, tallies, flight time).
OPS_STEP, OPS_SELF, OPS_REAL = 98, 133 + 6, 133 + 70
# The same kind of model for the phonon Monte Carlo kernel (FP32 build),
# counted from its source:
#   per flight segment 38: segment cap 1, the three face times from the
#     reciprocal velocity components 18, scattering time 4, the earliest 2,
#     position 6, fixed-point residence and its tally 7;
#   plus 15 per segment that ends on a subcell face (optical depth 3, the
#     face and the next subcell 12);
#   per scattering 111 + a binary search of the bin CDF: Philox 4x32-10 60,
#     four uniforms 12, tally 2, isotropic direction 13, optical depth 3, the
#     faces ahead 21;
#   per bundle 111 + two binary searches (subcell CDF, bin CDF) + 50: the
#     emission (id 5, Philox 60, uniforms 12, subcell index 24, position 9,
#     tally 2, sign 1) less the scattering tally, and its first direction;
#   5 per step of a binary search over n entries (ceil(log2 n) steps);
#   the rough and interface faces' draws are not counted (no tally counts them).
OPS_PH_SEG, OPS_PH_FACE, OPS_PH_SCAT, OPS_PH_BUNDLE, OPS_PH_SEARCH = 38, 15, 111, 111 + 50, 5


def phonon_ops(segments: int, scatterings: int, bundles: int, n_bins: int, n_cells: int) -> float:
    """Lane operations of the phonon op model for one solve."""
    sb = OPS_PH_SEARCH * math.ceil(math.log2(n_bins))
    sc = OPS_PH_SEARCH * math.ceil(math.log2(n_cells))
    return (OPS_PH_SEG * segments + OPS_PH_FACE * max(segments - scatterings, 0)
            + (OPS_PH_SCAT + sb) * scatterings + (OPS_PH_BUNDLE + sb + sc) * bundles)


def sweep_configs(rank: int, n_particles: int, **tune) -> list[dict]:
    return [W.nanowire(n_particles=n_particles, Vd=float(v), seed=1000 * rank + v, **tune) for v in range(21)]


def workload_desc(n_particles: int) -> dict:
    return {
        "workload": "half-nanowire V_ds sweep: 21 bias points 0..20 V x %d superparticles, 3x6x100 subcells "
                    "(60x120 nm x 1 um), N_d 1e18 cm^-3, 300 K, dt 1 fs, FP64 Poisson every 10 fs" % n_particles,
        "ensembles": 21,
        "particles_per_ensemble": n_particles,
        "step": "one Poisson period (10 x 1 fs) of all 21 bias points",
        "start": "timed after an untimed start-up transient (--prewarm-ps of simulated time) and the warm-up steps",
        "l2": "inputs larger than L2: particle state %.0f MB > 129 MB L2" % (21 * n_particles * 44 / 1e6),
    }


def kernel_sha() -> str:
    """Hash of the flight kernel's sources (common.cuh + kernels.cuh) with
    comments and blank lines removed: edits of comments keep a committed
    ncu measurement valid, any change of code invalidates it."""
    import re
    h = hashlib.sha256()
    for f in ("common.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1707_09073_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = [re.sub(r"//.*$", "", line).rstrip() for line in src.splitlines()]
        h.update("\n".join(line for line in code if line.strip()).encode())
    return h.hexdigest()[:16]


def committed_profile() -> dict | None:
    """The committed ncu figures of the flight kernel (DRAM bytes per launch,
    issue-slot and lane utilisation), if taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "flight_traffic.txt")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_sha") == kernel_sha():
            return d
    except (OSError, ValueError):
        pass
    return None


def committed_traffic() -> float | None:
    """DRAM bytes per flight launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    d = committed_profile()
    try:
        return float(d["dram_bytes_per_launch"]) if d else None
    except (KeyError, TypeError, ValueError):
        return None


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, gpu_index: int, path: str):
        self.path = path
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.f = open(path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        mx.append(float(parts[2]))
                    except ValueError:
                        continue
                    for n, v in zip(names, parts[5:9]):
                        if v.lower() == "active":
                            reasons.add(n)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("EMC_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def reduce_over_ranks(world: int, times: list, counts: list, device=None) -> tuple[list, list]:
    """Whole-job figures of a weak-scaling run: the slowest rank's times
    (max) and the units all ranks processed (sum).  Counts travel as int64,
    so event totals stay exact."""
    if world <= 1:
        return list(times), [int(c) for c in counts]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([int(x) for x in counts], dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [int(x) for x in c.tolist()]


# ------------------------------------------------------------------ oracle
def oracle_sample(n_particles: int, steps: int, min_seconds: float = 0.0, threads: int = 1) -> dict:
    """The FP64 oracle as it stands on one bias point of the sweep (V_d =
    10 V), its particle loop on `threads` host threads: real scattering
    events per second over `steps` Poisson periods (continuing until
    min_seconds if given)."""
    from oracle import oracle
    cfg = W.nanowire(n_particles=n_particles, Vd=10.0, seed=10)
    sim = oracle.Sim(cfg, threads=threads)
    t0 = sim.tallies()
    start = time.perf_counter()
    done = 0
    while done < steps or time.perf_counter() - start < min_seconds:
        sim.run(STEPS_PER_POISSON)
        done += 1
    el = time.perf_counter() - start
    t1 = sim.tallies()
    ev = int(t1["events"].sum()) - int(t0["events"].sum())
    return {"events": ev, "seconds": el, "periods": done, "n_particles": n_particles, "threads": threads}


def run_reference(args, world: int, rank: int):
    if rank != 0:
        return
    n_ref = 200_000 if args.steps + args.warmup <= 400 else max(20_000, int(200_000 * 400 / (args.steps + args.warmup)))
    from oracle import oracle
    oracle.build()
    cores = oracle.host_cores()
    cfg = W.nanowire(n_particles=n_ref, Vd=10.0, seed=10)
    sim = oracle.Sim(cfg, threads=cores)
    sim.run(STEPS_PER_POISSON * args.warmup)
    t0 = sim.tallies()
    start = time.perf_counter()
    sim.run(STEPS_PER_POISSON * args.steps)
    el = time.perf_counter() - start
    t1 = sim.tallies()
    ev = int(t1["events"].sum()) - int(t0["events"].sum())
    value = ev / el
    sample = ("FP64 oracle, particle loop on all %d host cores: 1 of the 21 bias points (V_d = 10 V), "
              "%d superparticles, each step one Poisson period (10 x 1 fs)" % (cores, n_ref))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_desc(200_000),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------- surrogate vs plain MC
def electrothermal_comparison(args, stream) -> dict:
    """Convergence of the coupled electrothermal iteration on the half
    nanowire at 64 drain biases (0..20 V) with 1800 subcells, four ways,
    each from the same steady 300 K electron state: the plain Monte Carlo
    iteration from a uniform 300 K start; the surrogate warm start (the
    first Fourier step corrected by the surrogate's v_d(E, T), which rescales
    each subcell's heat for the temperature it will have, then the plain
    iteration); the surrogate-corrected iteration (that correction in every
    Fourier step); and the plain iteration started from the surrogate's own
    heat map (heat per electron at each subcell's field x the subcell's
    electron density -> Fourier).  Every loop stops
    when no subcell temperature changes by more than max(0.1 K, the Monte
    Carlo noise of the iteration), and every result is then refereed by one
    long plain Monte Carlo window + Fourier solve at the temperatures the
    loop returned; the peak rises compared are the referee's."""
    import numpy as np
    import paper_1707_09073_gb300 as emc
    from paper_1707_09073_gb300 import electrothermal as ET
    from paper_1707_09073_gb300 import surrogate as S
    t0 = time.perf_counter()
    X = S.sample_inputs(args.sur_samples, seed=11)
    Y = S.mc_observables(X, W.bulk(), n_electrons=2000, warm_steps=800, avg_steps=800, seed0=7,
                         stream=stream.cuda_stream)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = S.Surrogate(X, Y, seed=5, stream=stream.cuda_stream)
    sur.fit(X, Y, steps=3000, batch=1024, lr=2e-3, seed=6)
    t_train = time.perf_counter() - t0
    # one surrogate query per subcell and bias point (1800 x 64), host arrays
    # in and out through the library call
    Xq = S.sample_inputs(1800 * 64, seed=12).astype(np.float32)
    sur.predict(Xq)
    t0 = time.perf_counter()
    for _ in range(10):
        sur.predict(Xq)
    t_infer = (time.perf_counter() - t0) / 10
    # the same queries through one GEMM launch per layer (the fused launch
    # is the default)
    sur.net.set_fused(False)
    sur.predict(Xq)
    t0 = time.perf_counter()
    for _ in range(10):
        sur.predict(Xq)
    t_infer_layered = (time.perf_counter() - t0) / 10
    sur.net.set_fused(True)
    nb = args.et_biases
    cfgs = [W.nanowire(n_particles=args.et_particles, Vd=20.0 * i / (nb - 1), seed=500 + i) for i in range(nb)]
    # kappa(T) with the phonon-electron scattering of Eq. (1) at the wire's
    # doping (1e18 cm^-3)
    tc = emc.emc.thermal_config(W.TABLE_II_GAN, h_bottom=args.h_bottom, L_boundary=120e-9, tol_K=1e-3,
                                n_e=cfgs[0]["Nd"], elec=W.ELECTRON_PHONON_GAN, substrate=W.TABLE_II_SIC,
                                area_ratio=args.interface_area_ratio)
    # the kappa and interface tables are built once per process (cached):
    # build them before any loop is timed
    emc.emc.kappa(tc, [300.0])
    emc.emc.interface_conductance(tc, [300.0])
    out = {}
    for mode in ("plain", "surrogate_warm_start", "surrogate", "surrogate_heat_start"):
        ctx = emc.Context(cfgs, stream=stream.cuda_stream)
        try:
            ss = ET.warm_to_steady(ctx)
            t0 = time.perf_counter()
            T0 = np.full((nb, ctx.n_cell), 300.0)
            if mode == "plain":
                r = ET.iterate(ctx, tc, T0, max_iter=15, stop_K=0.1)
            elif mode == "surrogate_warm_start":
                r = ET.surrogate_accelerated(ctx, sur, tc, T0, max_iter=15, stop_K=0.1, corrected_iters=1)
            elif mode == "surrogate":
                r = ET.surrogate_accelerated(ctx, sur, tc, T0, max_iter=15, stop_K=0.1)
            else:
                T0 = ET.surrogate_heat_start(ctx, sur, tc)
                r = ET.iterate(ctx, tc, T0, max_iter=15, stop_K=0.1)
            secs = time.perf_counter() - t0
            j = ET.referee(ctx, tc, r["T"], avg_steps=args.et_referee_steps)
            out[mode] = {"converged": r["converged"], "mc_iterations": r["iterations"], "seconds": secs,
                         "surrogate_seconds": r.get("surrogate_seconds", 0.0),
                         "peak_rise_K_max_bias_history": [round(float(h[-1]), 2) for h in r["history"]],
                         "max_dT_K_history": [round(x, 3) for x in r["max_dT_K"]],
                         "noise_K_history": [round(x, 3) for x in r["noise_K"]],
                         "referee_peak_rise_K_max_bias": float(j["peak"][-1]),
                         "referee_peak_se_K_max_bias": float(j["peak_se"][-1]),
                         "referee_max_dT_K": float(j["max_dT_K"].max()),
                         "steady_start": {"steady": ss["steady"], "windows_of_200_steps": ss["windows"]},
                         "_referee": j, "_r": r}
        finally:
            ctx.close()
    plain = out["plain"]["_referee"]
    hot = plain["peak"] >= 5.0
    # accuracy per Monte Carlo run: the first iteration whose peak rise at the
    # highest bias is within 2% / 1% of the refereed plain fixed point
    ref_pk = float(plain["peak"][-1])
    for m in out:
        h = [float(x[-1]) for x in out[m]["_r"]["history"]]
        for tol in (0.02, 0.01):
            it = next((i + 1 for i, x in enumerate(h) if abs(x - ref_pk) <= tol * ref_pk), None)
            out[m]["mc_runs_to_within_%dpct_of_refereed_peak" % round(100 * tol)] = it
    cmp = {}
    for mode in ("surrogate_warm_start", "surrogate", "surrogate_heat_start"):
        jm = out[mode]["_referee"]
        d = jm["peak"] - plain["peak"]
        se = np.hypot(jm["peak_se"], plain["peak_se"])
        rel = np.abs(d[hot]) / plain["peak"][hot]
        cmp[mode] = {"max_rel_diff_peak_rise": float(rel.max()), "mean_rel_diff_peak_rise": float(rel.mean()),
                     "biases_within_1pct": int((rel <= 0.01).sum()), "biases_compared": int(hot.sum()),
                     "biases_within_1pct_or_3se": int(((np.abs(d) <= np.maximum(0.01 * plain["peak"], 3 * se))[hot]).sum()),
                     "max_abs_diff_K_cool_biases": float(np.abs(d[~hot]).max()) if (~hot).any() else None,
                     "speedup_vs_plain": out["plain"]["seconds"] / max(out[mode]["seconds"], 1e-9)}
    saving = out["plain"]["seconds"] - out["surrogate_warm_start"]["seconds"]
    rth = []
    for i in range(0, nb, max(1, (nb - 1) // 8)):
        R = float(plain["R_th_K_per_W"][i])
        if R == R:
            rth.append({"Vd": cfgs[i]["Vd"], "peak_rise_K": float(plain["peak"][i]),
                        "power_W_half_wire": float(plain["power_W"][i]), "R_th_K_per_W_half_wire": R,
                        "R_th_K_per_W_array31": R / (2.0 * 31.0)})
    res = {
        "workload": "half nanowire 3x6x100, %d drain biases 0..20 V x %d superparticles, Fourier with kappa(T) "
                    "(Table II, 120 nm boundary, phonon-electron scattering of Eq. (1) at 1e18 cm^-3), "
                    "bottom face on the GaN/SiC interface of Eqs. (2)-(3) (diffuse mismatch, Table II "
                    "dispersions, R_K(300 K) = %.3g m2K/W) over %g times the wire's footprint%s; "
                    "each loop stops when no subcell temperature changes by more than "
                    "max(0.1 K, the largest difference between the temperatures of the two half-window heat maps); "
                    "every result refereed by a %d-step plain Monte Carlo window + Fourier solve"
                    % (nb, args.et_particles, 1.0 / float(emc.emc.interface_conductance(tc, [300.0])[0]),
                       args.interface_area_ratio,
                       ("" if args.h_bottom <= 0 else ", lumped %.1e W/m2/K in series" % args.h_bottom),
                       args.et_referee_steps),
        "plain_mc": {k: v for k, v in out["plain"].items() if not k.startswith("_")},
        "surrogate_warm_start": {k: v for k, v in out["surrogate_warm_start"].items() if not k.startswith("_")},
        "surrogate_corrected": {k: v for k, v in out["surrogate"].items() if not k.startswith("_")},
        "surrogate_heat_start": {k: v for k, v in out["surrogate_heat_start"].items() if not k.startswith("_")},
        "refereed_peak_rise_vs_plain": cmp,
        "speedup": out["plain"]["seconds"] / max(out["surrogate_warm_start"]["seconds"], 1e-9),
        "mc_iterations": {m: out[m]["mc_iterations"] for m in out},
        "R_th_vs_Vd": rth,
        "cost": {"surrogate_data_seconds": t_data, "surrogate_train_seconds": t_train,
                 "saving_per_run_seconds": saving,
                 "break_even_runs": (t_data + t_train) / saving if saving > 0 else None,
                 "note": "the surrogate is trained once per material and doping range and reused by every sweep"},
        "cost_to_2pct": _cost_to(out, "mc_runs_to_within_2pct_of_refereed_peak", t_data + t_train),
        "surrogate": {"samples": args.sur_samples, "train_steps": 3000, "batch": 1024,
                      "infer_ms_115200_queries": 1e3 * t_infer,
                      "infer_ms_115200_queries_layer_by_layer": 1e3 * t_infer_layered,
                      "network": "4-128-128-128-7 SiLU, BF16 tcgen05 tensor cores, FP32 accumulation in TMEM"},
    }
    return res


def _cost_to(out, key, t_surrogate):
    """Seconds to reach a peak-rise accuracy (Monte Carlo runs to it times
    the loop's mean seconds per run), plain against the surrogate warm start,
    and the sweeps after which the surrogate's data and training pay off."""
    def secs(m):
        n = out[m].get(key)
        return None if n is None else n * out[m]["seconds"] / max(out[m]["mc_iterations"], 1)
    sp, sw = secs("plain"), secs("surrogate_warm_start")
    saved = (sp - sw) if (sp is not None and sw is not None) else None
    return {"criterion": key, "plain_seconds": sp, "surrogate_warm_start_seconds": sw,
            "saving_per_sweep_seconds": saved,
            "break_even_sweeps": t_surrogate / saved if saved and saved > 0 else None}


# ------------------------------------------------- many-ensemble mixed batch
def batched_mixed(args, stream) -> dict:
    """Throughput on the 256-ensemble mixed batch (N ~ 10^U(4, 6), |E| ~
    U(0, 400) kV/cm, T ~ U(300, 600) K, N_d ~ 10^U(16, 19) cm^-3, 192 bulk +
    64 nanowire, 5.5e7 electrons): one context per geometry on the bench
    stream, one flight launch per context and Poisson period (profiled for
    the roofline); one step = 10 fs of every ensemble, CUDA-event timed.
    The same batch with both contexts in one flight launch per period
    (emc_group_step) is timed too."""
    import torch
    import paper_1707_09073_gb300 as emc
    cfgs = W.config_batched()
    groups = W.by_geometry(cfgs)
    ctxs = [emc.Context([cfgs[i] for i in idx], stream=stream.cuda_stream) for _, idx in sorted(groups.items())]

    def window(step_fn, profile=False):
        for ctx in ctxs:
            ctx.emc_tally(emc.TALLY_OBS, reset=True)
            ctx.emc_tally(emc.TALLY_EVENTS, reset=True)
            if profile:
                ctx.emc_profile(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.batched_steps):
            step_fn()
        b.record(stream)
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = [ctx.emc_profile_read() for ctx in ctxs]
            for ctx in ctxs:
                ctx.emc_profile(False)
        real = sum(int(ctx.emc_tally(emc.TALLY_EVENTS).sum()) for ctx in ctxs)
        obs = [o for ctx in ctxs for o in ctx.emc_tally(emc.TALLY_OBS)]
        return a.elapsed_time(b), real, obs, prof

    def group():
        emc.emc.group_step(ctxs, STEPS_PER_POISSON)

    def separate():
        for ctx in ctxs:
            ctx.emc_step(STEPS_PER_POISSON)

    try:
        with torch.cuda.stream(stream):
            for _ in range(3):
                separate()
            ms, real, obs, prof = window(separate, profile=True)
            ms_grp, real_grp, _, _ = window(group)
            # end to end: every step's observables of every ensemble read
            # back into page-locked host buffers (double-buffered)
            bufs = [[ctx.pinned_tally(emc.TALLY_OBS) for ctx in ctxs] for _ in range(2)]
            done = [torch.cuda.Event() for _ in range(2)]
            for ctx in ctxs:
                ctx.emc_tally(emc.TALLY_EVENTS, reset=True)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for i in range(args.batched_steps):
                separate()
                for ctx, ob in zip(ctxs, bufs[i % 2]):
                    ctx.emc_tally_async(emc.TALLY_OBS, ob)
                done[i % 2].record(stream)
                if i > 0:
                    done[(i - 1) % 2].synchronize()
            done[(args.batched_steps - 1) % 2].synchronize()
            e2e_s = time.perf_counter() - w0
            real2 = sum(int(ctx.emc_tally(emc.TALLY_EVENTS, reset=True).sum()) for ctx in ctxs)
            d2h = sum(b.nbytes for b in bufs[0])
    finally:
        for ctx in ctxs:
            ctx.close()
    selfe = sum(int(o["self_events"].sum()) for o in obs)
    psteps = sum(int(o["n_samples"]) for o in obs)
    flight_ms = sum(p[0] for p in prof)
    ops = OPS_REAL * real + OPS_SELF * selfe + OPS_STEP * psteps
    peaks = load_peaks()
    peak = N_SM * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops / (flight_ms * 1e-3) / 1e12 if flight_ms > 0 else None
    return {
        "workload": "256 independent ensembles: N ~ 10^U(4,6) (sum %d), |E| ~ U(0,400) kV/cm, T ~ U(300,600) K, "
                    "N_d ~ 10^U(16,19) cm^-3; 192 bulk (field along c) + 64 half nanowires (V_d = |E| x 1 um, "
                    "Poisson every 10 fs); one context per geometry, one flight launch per context per 10 fs"
                    % sum(c["n_particles"] for c in cfgs),
        "steps": args.batched_steps, "ms_per_step": ms / args.batched_steps,
        "events_per_s": real / (ms * 1e-3), "events_incl_self_per_s": (real + selfe) / (ms * 1e-3),
        "particle_steps_per_s": psteps / (ms * 1e-3),
        "one_launch_for_both": {"ms_per_step": ms_grp / args.batched_steps,
                                "events_per_s": real_grp / (ms_grp * 1e-3),
                                "path": "emc_group_step: both contexts' flights in one launch, blocks split by slots"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "k_flight<float, bulk> and k_flight<float, nanowire> (one launch per context and step)",
                     "flight_share_of_step": flight_ms / ms if ms > 0 else None,
                     "basis": "the op model of the headline roofline over the CUDA-event time of the flight launches"},
        "e2e": {"value": real2 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                "steps": args.batched_steps,
                "path": "emc_step of each context + emc_tally_async OBS of every ensemble into pinned host "
                        "buffers, double-buffered"},
    }


def phonon_comparison(args, stream) -> dict:
    """Phonon Monte Carlo of the transistor region for the heat the electrons
    emit at V_d = 20 V (one wire of the sweep, 200,000 superparticles, heat
    map over 5 ps after the 8 ps start-up): the FP32 kernel's throughput,
    the temperature after three passes with local-temperature rates, the
    Fourier solve of the same heat with the same boundaries (contacts at
    300 K, the GaN/SiC interface of Eqs. (2)-(3) under the bottom face; its
    kappa(T) with the mean free paths capped at the 120 nm cross-section,
    where the Monte Carlo scatters at the faces), and the oracle's rate on the host
    cores for a bounded sample of the same problem."""
    import numpy as np
    import paper_1707_09073_gb300 as emc
    from paper_1707_09073_gb300 import electrothermal as ET
    cfg = W.nanowire(n_particles=args.particles, Vd=20.0, seed=20)
    ctx = emc.Context([cfg], stream=stream.cuda_stream)
    try:
        ctx.emc_step(8000)
        ctx.emc_tally(emc.TALLY_HEAT_J, reset=True)
        win = 5000
        ctx.emc_step(win)
        q = ET.heat_map(ctx, win * cfg["dt"])[0]
        # the same phonon model on both sides (Table II, Eq. (1) at the wire's
        # doping, the interface of Eqs. (2)-(3)); the Monte Carlo scatters at
        # the faces themselves, the Fourier solve caps the mean free paths at
        # the 120 nm cross-section
        el = dict(n_e=cfg["Nd"], elec=W.ELECTRON_PHONON_GAN, substrate=W.TABLE_II_SIC)
        tc = emc.emc.thermal_config(W.TABLE_II_GAN, h_bottom=0.0, L_boundary=0.0, area_ratio=1.0, **el)
        tc_f = emc.emc.thermal_config(W.TABLE_II_GAN, h_bottom=0.0, L_boundary=120e-9, tol_K=1e-4, area_ratio=1.0, **el)
        pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=1000, precision=emc.FP32, p_specular=0.0, seed=77)
        N = args.phonon_bundles
        emc.emc.phonon_solve(ctx, tc, pc, q, 100_000)  # warm-up
        r = emc.emc.phonon_solve(ctx, tc, pc, q, N)
        mc = ET.phonon_mc_temperature(ctx, tc, pc, q, N, passes=3, first=N)
        T_f, _ = emc.emc.thermal_solve(ctx, tc_f, q[None, :])
        # the coupled fixed points from 300 K: electrons <-> phonon Monte
        # Carlo, and electrons <-> Fourier (the same electron windows)
        T0 = np.full((1, ctx.n_cell), 300.0)
        # 3000-step averaging windows: the half-window noise of one wire's
        # hot spot with 1000 steps (~20 K) let a loop stop a step early
        hy = ET.hybrid_iterate(ctx, tc, pc, T0, args.phonon_loop_bundles, avg_steps=3000, max_iter=10, first=10 * N)
        fo = ET.iterate(ctx, tc_f, T0, avg_steps=3000, max_iter=10)
    finally:
        ctx.close()
    P = r["power_W"]
    net = float(q.sum() * cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / q.size)
    peaks = load_peaks()
    peak = N_SM * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ops = phonon_ops(r["segments"], r["n_scatterings"], N, 1000, cfg["nx"] * cfg["ny"] * cfg["nz"])
    achieved = ops / (r["kernel_ms"] * 1e-3) / 1e12
    peak_mc = float(mc["T"].max() - tc.T_sink)
    peak_f = float(T_f[0].max() - tc.T_sink)
    nyz = cfg["ny"] * cfg["nz"]
    out = {
        "workload": "heat of the V_d = 20 V wire (%d superparticles, 3x6x100 subcells) carried by %d phonon bundles, "
                    "1000 wave-vector bins, FP32; faces: contacts isothermal 300 K, plane A specular, outer side and "
                    "top diffuse, bottom GaN/SiC diffuse-mismatch interface" % (args.particles, N),
        "bundles": N, "kernel_ms": r["kernel_ms"], "bundles_per_s": N / (r["kernel_ms"] * 1e-3),
        "segments_per_bundle": r["segments"] / N, "segments_per_s": r["segments"] / (r["kernel_ms"] * 1e-3),
        "scatterings_per_bundle": r["n_scatterings"] / N, "capped": r["capped"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_phonon<float>",
                     "basis": "lane operations of the phonon op model (bench.py OPS_PH_*: per segment, face, "
                              "scattering, bundle and binary-search step) over the kernel's CUDA-event time, "
                              "against 152 SMs x 128 lanes x %.0f MHz" % peaks.get("sm_max_mhz", 2070.0),
                     "ops_per_segment": ops / max(r["segments"], 1),
                     "dram": "tables and tallies stay in L2: ~0.1 MB of DRAM per 10^6 bundles (ncu)"},
        "absorbed_share": (np.asarray(r["absorbed"], float) / N).round(4).tolist(),
        "heat_net_W": net, "heat_abs_W": P,
        "peak_rise_K": {"phonon_mc": peak_mc, "fourier": peak_f, "mc_passes": mc["peak_history"]},
        "R_th_K_per_W_half_wire": {"phonon_mc": peak_mc / net, "fourier": peak_f / net},
        "coupled_fixed_point": {
            "what": "electron MC <-> phonon MC and electron MC <-> Fourier from 300 K (300 + 3000 steps per "
                    "iteration, %d bundles per phonon solve); stop: every subcell within max(0.1 K, the noise)"
                    % args.phonon_loop_bundles,
            "phonon_mc": {"converged": bool(hy["converged"]), "iterations": int(hy["iterations"]),
                          "seconds": round(hy["seconds"], 3), "peak_rise_K": [round(float(x[0]), 2) for x in hy["history"]],
                          "R_th_K_per_W_half_wire": float(hy["R_th_K_per_W"][0])},
            "fourier": {"converged": bool(fo["converged"]), "iterations": int(fo["iterations"]),
                        "seconds": round(fo["seconds"], 3), "peak_rise_K": [round(float(x[0]), 2) for x in fo["history"]],
                        "R_th_K_per_W_half_wire": float(fo["R_th_K_per_W"][0])},
        },
        "rise_along_x_K": {"phonon_mc": (mc["T"].reshape(cfg["nx"], nyz).mean(axis=1) - 300.0)[::10].round(2).tolist(),
                           "fourier": (T_f[0].reshape(cfg["nx"], nyz).mean(axis=1) - 300.0)[::10].round(2).tolist(),
                           "x_um": [round((i + 0.5) / cfg["nx"] * cfg["Lx"] * 1e6, 3) for i in range(0, cfg["nx"], 10)]},
    }
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        from oracle import phonon as PHO
        O.build()
        cores = O.host_cores()
        n_cpu = max(1000, min(N, args.phonon_cpu_bundles))
        # the same geometry, spectrum and faces with a seeded synthetic heat
        # map of the same shape at its default peak (the oracle takes no
        # input from the GPU run; the bundle weight does not change the
        # segments a bundle flies)
        qs = W.heat_map(cfg, seed=1)
        t0 = time.perf_counter()
        ro = PHO.solve(cfg, qs, W.TABLE_II_GAN, emc.emc.WIRE_FACES, n_cpu, seed=77, nb=1000, n_e=cfg["Nd"],
                       elec=W.ELECTRON_PHONON_GAN, substrate=W.TABLE_II_SIC, threads=cores)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ro["segments"] / dt, "unit": "segments/s", "cores": cores, "kind": "oracle",
                               "sample": "%d bundles on the same wire, spectrum and faces with a synthetic heat map "
                                         "of the same shape (FP64 oracle, one pass at 300 K), %.1f s" % (n_cpu, dt),
                               "bundles_per_s": n_cpu / dt}
    return out


def sharded_wire(args, cfgs, shards: int) -> dict:
    """The bias sweep's wires, each wire's particles sharded over `shards`
    contexts on this GPU with the integer charge exchange on the host at the
    end of every Poisson period (the multi-GPU protocol run on one GPU), and
    the same wires unsharded, both timed by the wall clock around the same
    number of steps (the sharded path synchronises at every exchange)."""
    import numpy as np
    import torch
    import paper_1707_09073_gb300 as emc
    from paper_1707_09073_gb300 import shard as SH
    steps = STEPS_PER_POISSON * args.shard_periods
    out = {"shards": shards, "steps": steps, "workload": "the bias sweep (21 wires), particles split over shards"}
    for name, make in (("unsharded", lambda: emc.Context(cfgs)),
                       ("sharded", lambda: SH.LocalWire(cfgs, shards))):
        w = make()
        try:
            w.emc_step(3 * STEPS_PER_POISSON)
            w.emc_tally(emc.TALLY_EVENTS, reset=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            w.emc_step(steps)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ev = int(np.asarray(w.emc_tally(emc.TALLY_EVENTS)).sum())
        finally:
            w.close()
        out[name] = {"events_per_s": ev / dt, "ms_per_step": 1e3 * dt / steps}
    out["sharded_over_unsharded"] = out["sharded"]["events_per_s"] / out["unsharded"]["events_per_s"]
    return out


# --------------------------------------------------------------------- GPU
def run_emc(args, world: int, rank: int, local: int):
    import numpy as np
    import torch

    import __graft_entry__ as G
    G.build()
    import paper_1707_09073_gb300 as emc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    n_part = args.particles
    tune = {k: v for k, v in (("table_smem_kb", args.table_kb), ("block_size", args.block),
                              ("sort_period", args.sort_period)) if v}
    tuned = None
    if not tune and not args.no_tune:
        # block size, staged table size and sort period from the autotuner
        # (timed once per GPU and workload shape, then cached)
        from paper_1707_09073_gb300 import autotune
        tuned = autotune.tune(sweep_configs(rank, n_part))
        tune = dict(tuned)
    cfgs = sweep_configs(rank, n_part, **tune)
    E = len(cfgs)
    ctx = emc.Context(cfgs, stream=stream.cuda_stream)
    n_slots_ctx = ctx.capacity
    steps = STEPS_PER_POISSON
    with torch.cuda.stream(stream):
        # untimed: the electrons first leave the start-up transient (the
        # event rate of the first picoseconds is inflated)
        ctx.emc_step(int(round(args.prewarm_ps * 1000)))
        for _ in range(args.warmup):
            ctx.emc_step(steps)
        ctx.emc_tally(emc.TALLY_OBS, reset=True)
        launches0 = ctx.launch_count()
        # raw clock samples go to $EMC_ARTIFACT_DIR when set (the summary is in the JSON line)
        art = os.environ.get("EMC_ARTIFACT_DIR") or tempfile.gettempdir()
        sampler = ClockSampler(local, os.path.join(art, f"clocks_rank{rank}.csv"))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        ctx.emc_profile(True)
        t_start.record(stream)
        for _ in range(args.steps):
            ctx.emc_step(steps)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop()
        ms = t_start.elapsed_time(t_end)
        flight_ms, flight_launches = ctx.emc_profile_read()
        ctx.emc_profile(False)
        launches = ctx.launch_count() - launches0
        ev = ctx.emc_tally(emc.TALLY_EVENTS)
        obs = ctx.emc_tally(emc.TALLY_OBS, reset=True)
    real = int(ev.sum())
    selfe = int(sum(int(o["self_events"].sum()) for o in obs))
    psteps = int(sum(o["n_samples"] for o in obs))

    # ---- end to end through the public API with host buffers
    bias = torch.zeros((E, 3), dtype=torch.float64).pin_memory()
    for e, c in enumerate(cfgs):
        bias[e, 0], bias[e, 1], bias[e, 2] = c["Vs"], c["Vd"], c["Vg"]
    # results land in page-locked host memory, like the bias that goes in;
    # two buffer sets, so step i + 1 is enqueued before step i's results are
    # waited for (every step's results still reach the host inside the timed
    # region)
    bufs = [(ctx.pinned_tally(emc.TALLY_OBS), ctx.pinned_tally(emc.TALLY_HEAT), ctx.pinned_tally(emc.TALLY_CROSSINGS))
            for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    n_e2e = max(1, min(args.steps, args.e2e_steps))
    with torch.cuda.stream(stream):
        ctx.emc_tally(emc.TALLY_OBS, reset=True)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for i in range(n_e2e):
            ctx.emc_set_bias_all(bias.data_ptr())
            ctx.emc_step(steps)
            ob, ht, cr = bufs[i % 2]
            ctx.emc_tally_async(emc.TALLY_OBS, ob)
            ctx.emc_tally_async(emc.TALLY_HEAT, ht)
            ctx.emc_tally_async(emc.TALLY_CROSSINGS, cr)
            done[i % 2].record(stream)
            if i > 0:
                done[(i - 1) % 2].synchronize()
        done[(n_e2e - 1) % 2].synchronize()
        e2e_s = time.perf_counter() - w0
        ev2 = int(ctx.emc_tally(emc.TALLY_EVENTS, reset=True).sum())
    heat, cross = bufs[0][1], bufs[0][2]
    # drain current of every bias point over the end-to-end window (the
    # crossings accumulate from the reset before the loop): the I-V curve
    last = bufs[(n_e2e - 1) % 2][2]
    window_s = n_e2e * steps * cfgs[0]["dt"]
    iv = []
    for e, c in enumerate(cfgs):
        w = c["Nd"] * c["Lx"] * c["Ly"] * c["Lz"] / c["n_particles"]
        iv.append([c["Vd"], 1e6 * 1.602176634e-19 * w * float(last[e][1] - last[e][3]) / window_s])
    h2d = E * 3 * 8
    d2h = E * 128 + heat.nbytes + cross.nbytes

    # ---- reduce over ranks (max time, summed events)
    (ms, e2e_s), (real, selfe, psteps, ev2) = reduce_over_ranks(world, [ms, e2e_s], [real, selfe, psteps, ev2], dev)
    ctx.close()
    if rank != 0:
        return

    value = real / (ms * 1e-3)
    peaks = load_peaks()
    clk = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    # roofline of the dominant kernel (flight): lane-operation issue rate
    per_launch_ops = (OPS_REAL * real + OPS_SELF * selfe + OPS_STEP * psteps) / max(world, 1) / max(flight_launches, 1)
    avg_s = flight_ms * 1e-3 / max(flight_launches, 1)
    n_slots = n_slots_ctx
    achieved = per_launch_ops / avg_s / 1e12
    peak_max = N_SM * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "Tops/s", "frac": achieved / peak_max,
            "traffic": committed_traffic(), "kernel": "k_flight<float, nanowire>",
            "hbm_view": {"algorithmic_bytes_per_launch": 84 * n_slots,
                         "achieved_gbs": 84 * n_slots / avg_s / 1e9,
                         "peak_gbs": peaks.get("hbm_gbs", 6800.0),
                         "frac": 84 * n_slots / avg_s / 1e9 / peaks.get("hbm_gbs", 6800.0),
                         "basis": "84 B of particle state read and written per slot per launch"},
            "ncu_same_source": {k: v for k, v in (committed_profile() or {}).items()
                                if k in ("issue_active_frac", "lanes_active_per_instruction",
                                         "fp32_pipe_cycles_active_frac", "warps_active_frac")} or None,
            "peak_basis": "152 SMs x 128 lanes x %.0f MHz max SM clock (lane operations/s)" % peaks.get("sm_max_mhz", 2070.0),
            "frac_at_sampled_clock": achieved / (N_SM * LANES_PER_SM * clk * 1e6 / 1e12),
            "flight_share_of_step": flight_ms / ms if ms > 0 else None,
            "op_model": {"per_real_event": OPS_REAL, "per_self_event": OPS_SELF, "per_particle_step": OPS_STEP,
                         "unit": "lane operations of the method's arithmetic (loads/addressing excluded)"}}

    # ---- oracle on the host cores (bounded sample)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        cores = oracle.host_cores()
        s = oracle_sample(args.cpu_particles, steps=2, min_seconds=args.cpu_seconds, threads=cores)
        s1 = oracle_sample(args.cpu_particles, steps=1, min_seconds=args.cpu_seconds / 4, threads=1)
        cpu = {"value": s["events"] / s["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle, particle loop on all %d host cores: 1 of the 21 bias points (V_d = 10 V), "
                         "%d superparticles, %d Poisson periods (%.1f s)" % (cores, s["n_particles"], s["periods"],
                                                                             s["seconds"]),
               "single_thread": {"value": s1["events"] / s1["seconds"], "unit": UNIT, "cores": 1,
                                 "sample": "%d Poisson periods (%.1f s)" % (s1["periods"], s1["seconds"])}}

    phon = None
    if world == 1 and not args.no_phonon:
        torch.cuda.synchronize(dev)
        phon = phonon_comparison(args, stream)

    shw = None
    if world == 1 and args.shards > 1:
        torch.cuda.synchronize(dev)
        shw = sharded_wire(args, cfgs, args.shards)

    mixed = None
    if world == 1 and not args.no_batched:
        torch.cuda.synchronize(dev)
        mixed = batched_mixed(args, stream)

    et = None
    if world == 1 and not args.no_electrothermal:
        torch.cuda.synchronize(dev)
        et = electrothermal_comparison(args, stream)

    cfg = workload_desc(n_part)
    cfg["parallelism"] = "weak: one full sweep per GPU" if world > 1 else "1 GPU"
    props = torch.cuda.get_device_properties(dev)
    cfg["device"] = {"name": props.name, "sms": props.multi_processor_count,
                     "memory_gib": round(props.total_memory / 2**30, 1), "host_cores": len(os.sched_getaffinity(0))}
    cfg["launch"] = dict(tune, source="autotuner" if tuned else ("command line" if tune else "defaults"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "events_incl_self_per_s": (real + selfe) / (ms * 1e-3),
        "particle_steps_per_s": psteps / (ms * 1e-3),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": ev2 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": n_e2e, "path": "emc_set_bias_all (pinned host) + emc_step + emc_tally_async OBS/HEAT/CROSSINGS into pinned host buffers, double-buffered: step i+1 enqueued before step i's results are waited for"},
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"],
                   "samples": clocks["samples"]},
        "gpu_launches": launches,
        "iv_curve": {"unit": "[V_d (V), I_d (uA) of the half wire]", "window_fs": n_e2e * steps,
                     "points": [[v, round(i, 3)] for v, i in iv]} if world == 1 else None,
        "batched_mixed": mixed,
        "sharded_wire": shw,
        "phonon_mc": phon,
        "surrogate_vs_plain_mc": et,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="emc", choices=["emc", "reference"])
    ap.add_argument("--particles", type=int, default=200_000)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--prewarm-ps", type=float, default=8.0,
                    help="untimed simulated time before the warm-up steps (the start-up transient)")
    ap.add_argument("--cpu-particles", type=int, default=200_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--table-kb", type=int, default=0, help="rate-table KiB staged in shared memory (0 = default)")
    ap.add_argument("--block", type=int, default=0, help="flight-kernel block size (0 = default)")
    ap.add_argument("--sort-period", type=int, default=0, help="sort particles every this many launches (0 = never)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--no-electrothermal", action="store_true", help="skip the surrogate vs plain-MC comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-ensemble mixed batch")
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--shards", type=int, default=2,
                    help="also run the sweep with each wire's particles split over this many contexts (0/1: skip)")
    ap.add_argument("--shard-periods", type=int, default=30)
    ap.add_argument("--no-phonon", action="store_true", help="skip the phonon Monte Carlo of the 20 V wire")
    ap.add_argument("--phonon-bundles", type=int, default=10_000_000)
    ap.add_argument("--phonon-cpu-bundles", type=int, default=4_000_000)
    ap.add_argument("--phonon-loop-bundles", type=int, default=2_000_000)
    ap.add_argument("--et-biases", type=int, default=64)
    ap.add_argument("--et-particles", type=int, default=100_000)
    ap.add_argument("--et-referee-steps", type=int, default=5000)
    ap.add_argument("--sur-samples", type=int, default=100_000)
    ap.add_argument("--h-bottom", type=float, default=0.0,
                    help="lumped conductance under the interface, W/m2/K (0: none)")
    ap.add_argument("--interface-area-ratio", type=float, default=10.0,
                    help="GaN/SiC interface area per unit of the wire's bottom face")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_emc(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
