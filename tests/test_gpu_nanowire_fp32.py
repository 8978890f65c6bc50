"""The production build on the benchmarked workload: FP32 flights and
scattering (k_flight<float, nanowire>), one FP64-refined Poisson sweep per
period, on the full half-nanowire geometry (60 x 120 nm x 1 um, 3 x 6 x 100
subcells, 1e18 cm^-3, 200,000 superparticles), against the FP64 oracle.

- Statistics at V_d = 10 V and 20 V: after the same warm-up, the oracle's
  window averages (one run per bias, all host cores) against the GPU's
  (R independent replicas per bias): per-subcell heat maps (net polar optical
  plus intervalley phonon emission) element by element, the heat profile
  along the wire, drain current, mean velocity along the wire, mean energy and
  valley occupancy.  The noise of one run is measured, not assumed: the spread
  of the GPU replicas, with a per-subcell counting model var = phi * (events)
  pooled over all subcells.  Each comparison passes within 1% or within the
  3-sigma criterion taken family-wise (the two-sided 0.27% tail split over
  the comparisons of a family).
- Short horizon: the FP32 build against the FP64 parity build on the same
  Philox streams over 10 steps; the particles whose valley, Philox counter or
  life differ are counted and reported.
- Bit-exact FP64 parity on the full geometry at 20 V (short horizon).
- The production Poisson update's error against the oracle's solve of the
  same subcell charge.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import workloads as W
from tests.emc_harness import oracle_heat

pytestmark = pytest.mark.gpu

Q = 1.602176634e-19
ALPHA3 = 0.0027  # two-sided tail of 3 sigma
R = 16           # GPU replicas per bias point
WARM, AVG = 8000, 2000  # the full wire reaches steady state after ~8 ps
BIASES = (10.0, 20.0)


def artifact(name, obj):
    out = os.environ.get("EMC_ARTIFACT_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, name), "w") as f:
            json.dump(obj, f, indent=1, default=float)
    print(json.dumps(obj, indent=1, default=float))


def window_observables(ev, obs, cross, cfg):
    """Observables of one run over the averaging window: per-subcell net and
    gross phonon events, drain current, mean v_x, mean energy, valley
    fractions."""
    ev = ev.astype(np.int64)
    heat = oracle_heat(ev).sum(1)                       # net POP + intervalley per subcell
    gross = (ev[:, :, 1:3].sum((1, 2)) + ev[:, :, 4:].sum((1, 2)))
    n = obs["n_samples"]
    w = cfg["Nd"] * cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / cfg["n_particles"]
    I = Q * w * float(cross[1] - cross[3]) / (AVG * cfg["dt"])
    return {
        "heat": heat.astype(float), "gross": gross.astype(float),
        "I_drain_A": I,
        "v_x_m_s": obs["sum_v"][0] / n,
        "E_mean_eV": obs["sum_E"] / n / Q,
        "f_Gamma1": obs["valley_steps"][0] / n,
        "f_U": obs["valley_steps"][1] / n,
        "f_Gamma3": obs["valley_steps"][2] / n,
        "heat_total": float(heat.sum()),
    }


@pytest.fixture(scope="module")
def fp32_vs_oracle(emc, oracle_mod):
    cfgs = [W.nanowire(n_particles=200_000, Vd=v, seed=7000 + 100 * b + r)
            for b, v in enumerate(BIASES) for r in range(R)]
    with emc.Context(cfgs) as ctx:
        ctx.emc_step(WARM)
        ctx.emc_tally(emc.TALLY_OBS, reset=True)
        ctx.emc_step(AVG)
        ev = ctx.emc_tally(emc.TALLY_EVENTS_CELL)
        obs = ctx.emc_tally(emc.TALLY_OBS)
        cr = ctx.emc_tally(emc.TALLY_CROSSINGS)
    gpu = [[window_observables(ev[b * R + r], obs[b * R + r], cr[b * R + r], cfgs[b * R + r]) for r in range(R)]
           for b in range(len(BIASES))]
    ref = []
    for b, v in enumerate(BIASES):
        cfg = W.nanowire(n_particles=200_000, Vd=v, seed=7900 + b)
        sim = oracle_mod.Sim(cfg, threads=oracle_mod.host_cores())
        sim.run(WARM)
        t0 = sim.tallies()
        sim.run(AVG)
        t1 = sim.tallies()
        d_ev = t1["events"].astype(np.int64) - t0["events"].astype(np.int64)
        d_obs = {"n_samples": t1["n_samples"] - t0["n_samples"], "sum_v": t1["sum_v"] - t0["sum_v"],
                 "sum_E": t1["sum_E"] - t0["sum_E"], "valley_steps": t1["valley_steps"] - t0["valley_steps"]}
        ref.append(window_observables(d_ev, d_obs, t1["crossings"] - t0["crossings"], cfg))
    return gpu, ref


def test_heat_map_per_subcell(fp32_vs_oracle):
    """Every subcell's net phonon emission over the window: GPU replica mean
    against the oracle run.  sigma^2 of one run = phi * gross events of the
    subcell, phi pooled over all subcells from the replicas' spread.  Subcells
    without phonon events in any run (depleted under the gate) must stay
    without them."""
    gpu, ref = fp32_vs_oracle
    report, checks = {}, []
    for b, v in enumerate(BIASES):
        H = np.array([g["heat"] for g in gpu[b]])       # [R][C]
        nbar = np.array([g["gross"] for g in gpu[b]]).mean(0)
        live = (nbar > 0) | (ref[b]["gross"] > 0)
        phi = ((H - H.mean(0)) ** 2).sum() / ((R - 1) * nbar.sum())
        sig = np.sqrt(phi * np.maximum(nbar, 1.0) * (1.0 / R + 1.0))
        d = H.mean(0) - ref[b]["heat"]
        z = d / sig
        C = int(live.sum())
        zc = stats.norm.isf(ALPHA3 / (2 * C * len(BIASES)))
        rel = np.abs(d) / np.maximum(np.abs(ref[b]["heat"]), 1.0)
        ok = (np.abs(z) <= zc) | (rel <= 0.01)
        # the heat profile along the wire (the cross-section summed per x)
        nx = H.shape[1] // 18
        Hx = H.reshape(R, nx, 18).sum(2)
        nx_bar = nbar.reshape(nx, 18).sum(1)
        hx_ref = ref[b]["heat"].reshape(nx, 18).sum(1)
        phix = ((Hx - Hx.mean(0)) ** 2).sum() / ((R - 1) * nx_bar.sum())
        sx = np.sqrt(phix * np.maximum(nx_bar, 1.0) * (1.0 / R + 1.0))
        dx = Hx.mean(0) - hx_ref
        zx = dx / sx
        zxc = stats.norm.isf(ALPHA3 / (2 * nx * len(BIASES)))
        okx = (np.abs(zx) <= zxc) | (np.abs(dx) <= 0.01 * np.abs(hx_ref))
        chi = float((z[live] ** 2).mean())
        chi_max = stats.chi2.isf(1e-3, C) / C
        report[f"Vd={v:g}"] = {"subcells_with_events": C, "phi": phi, "mean_z2": chi, "mean_z2_limit": chi_max,
                              "max_abs_z": float(np.abs(z[live]).max()), "z_crit": zc,
                              "subcells_outside": int((~ok).sum()), "worst_subcells": np.argsort(-np.abs(z))[:5].tolist(),
                              "profile_phi": phix, "profile_mean_z2": float((zx ** 2).mean()),
                              "profile_max_abs_z": float(np.abs(zx).max()), "profile_z_crit": zxc,
                              "profile_slices_outside": int((~okx).sum()),
                              "total_rel_diff": float(d.sum() / ref[b]["heat"].sum()),
                              "empty_subcells_agree": bool(np.all(H[:, ~live] == 0) and np.all(ref[b]["heat"][~live] == 0))}
        checks.append((ok.all(), okx.all(), chi <= chi_max, report[f"Vd={v:g}"]["empty_subcells_agree"]))
    artifact("nanowire_fp32_heat_map.json", report)
    # per subcell and per slice within the family-wise 3-sigma bound (or 1%);
    # no systematic shift hiding under the per-cell noise (mean z^2 within
    # the 99.9% chi-square band)
    for (a, bb, c, e), v in zip(checks, BIASES):
        assert a and bb and c and e, (v, report)


def test_observables(fp32_vs_oracle):
    gpu, ref = fp32_vs_oracle
    keys = ["I_drain_A", "v_x_m_s", "E_mean_eV", "f_Gamma1", "f_U", "f_Gamma3", "heat_total"]
    n_checks = len(keys) * len(BIASES)
    tcrit = stats.t.isf(ALPHA3 / (2 * n_checks), R - 1)
    report = {}
    for b, v in enumerate(BIASES):
        rep = {}
        for k in keys:
            x = np.array([g[k] for g in gpu[b]])
            s1 = x.std(ddof=1)
            d = x.mean() - ref[b][k]
            sig = s1 * math.sqrt(1.0 / R + 1.0)
            rep[k] = {"gpu_fp32": x.mean(), "oracle_fp64": ref[b][k], "rel_error": d / ref[b][k] if ref[b][k] else 0.0,
                      "sigma_one_run": s1, "z": d / sig if sig > 0 else 0.0}
            if k in ("f_U", "f_Gamma3") and ref[b][k] < 1e-3 and x.mean() < 1e-3:
                assert abs(d) <= tcrit * sig + 1e-5, (v, k, rep[k])
                continue
            assert abs(d) <= max(0.01 * abs(ref[b][k]), tcrit * sig), (v, k, rep[k])
        report[f"Vd={v:g}"] = rep
    report["t_crit"] = tcrit
    artifact("nanowire_fp32_observables.json", report)


def test_fp32_divergence_over_ten_steps(emc):
    """FP32 production against FP64 parity build, same seed and Philox
    streams, full wire at 20 V, 10 steps (one Poisson period with its refill):
    count the particles whose valley, Philox counter or life differ."""
    cfg = W.nanowire(n_particles=200_000, Vd=20.0, seed=31)
    out = {}
    for prec in (emc.FP64, emc.FP32):
        with emc.Context(cfg, precision=prec) as ctx:
            p0 = ctx.debug_particles()
            ctx.emc_step(10)
            out[prec] = (p0, ctx.debug_particles())
    n = cfg["n_particles"]

    def by_id(p):
        order = np.argsort(p["id"], kind="stable")
        return {k: p[k][order] for k in ("valley", "ctr")}

    a0, b0 = by_id(out[emc.FP64][0]), by_id(out[emc.FP32][0])
    init_diff = int(((a0["valley"] != b0["valley"]) | (a0["ctr"] != b0["ctr"])).sum())
    a, b = by_id(out[emc.FP64][1]), by_id(out[emc.FP32][1])
    diverged = (a["valley"] != b["valley"]) | (a["ctr"] != b["ctr"])
    rep = {"particles": n, "diverged_after_10_steps": int(diverged.sum()), "differed_initially": init_diff,
           "fraction": float(diverged.sum()) / n}
    artifact("fp32_divergence_10_steps.json", rep)
    assert init_diff <= n * 1e-4, rep
    assert diverged.sum() <= n * 1e-3, rep


def test_full_wire_fp64_bit_exact(emc, oracle_mod):
    """FP64 parity build against the oracle on the full 1 um geometry at
    20 V, 20,000 electrons, 40 steps (four Poisson periods with refills):
    per-subcell event counts, crossings, subcell charge and the self
    scatterings are equal."""
    cfg = W.nanowire(n_particles=20_000, Vd=20.0, seed=23)
    steps = 40
    ref = oracle_mod.Sim(cfg, threads=oracle_mod.host_cores())
    ref.run(steps)
    rt = ref.tallies()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        ev = ctx.emc_tally(emc.TALLY_EVENTS_CELL)[0]
        cr = ctx.emc_tally(emc.TALLY_CROSSINGS)[0]
        ch = ctx.emc_tally(emc.TALLY_CHARGE)[0]
        ob = ctx.emc_tally(emc.TALLY_OBS)[0]
    assert np.array_equal(ev, rt["events"])
    assert np.array_equal(cr, rt["crossings"])
    assert np.array_equal(ch, rt["charge"])
    assert np.array_equal(ob["self_events"], rt["self_events"].astype(np.int64))
    assert np.array_equal(ob["valley_steps"], rt["valley_steps"])
    assert ob["n_alive"] == rt["n_alive"] and cr[2] + cr[3] > 0


def test_production_poisson_error(emc, oracle_mod):
    """The FP32 build's field update (warm-started, one FP64-refined sweep
    with the FP32 inverse per period) against the oracle's FP64 solve of the
    same subcell charge and bias: the stated error of the production
    potential."""
    cfg = W.nanowire(n_particles=200_000, Vd=20.0, seed=41)
    rep = {}
    with emc.Context(cfg) as ctx:
        for period in range(1, 31):
            ctx.emc_step(10)
            if period in (1, 10, 30):
                ch = ctx.emc_tally(emc.TALLY_CHARGE)[0].astype(float)
                phi = ctx.emc_tally(emc.TALLY_PHI)[0]
                Vcell = cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / ch.size
                w = cfg["Nd"] * cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / cfg["n_particles"]
                rho = Q * (cfg["Nd"] - w * ch / Vcell)
                want = oracle_mod.poisson(cfg, rho, tol=1e-14)
                err = float(np.abs(phi - want).max() / np.abs(want).max())
                rep[f"after {10 * period} fs"] = err
    artifact("production_poisson_error.json", rep)
    assert max(rep.values()) < 1e-5, rep
