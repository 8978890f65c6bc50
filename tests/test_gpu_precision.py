"""Precision variant: the production build (FP32 flights and scattering,
compensated FP32 per-thread sums reduced in FP64, integer tallies) with
10,000,000 electrons simulated for 20 ps against the FP64 oracle with
200,000 electrons, bulk GaN at 100 kV/cm, 1e17 cm^-3, 300 K.  Both are
steady after the first picosecond: the GPU run is averaged over ps 1-20
(blocks of 1 ps), the oracle over ps 1-2 (blocks of 0.1 ps).  The stated
error of each observable is written out and must lie within 1% or 3 combined
standard errors of the block means."""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

Q = 1.602176634e-19


def block_means(step, tally, blocks, per):
    out = []
    prev = tally()
    for _ in range(blocks):
        step(per)
        cur = tally()
        out.append({k: cur[k] - prev[k] for k in cur})
        prev = cur
    return out


def observables(d, hw):
    n = d["n"]
    return {
        "v_drift_m_s": -d["vz"] / n,
        "E_mean_eV": d["E"] / n / Q,
        "f_Gamma1": d["v0"] / n, "f_U": d["v1"] / n, "f_Gamma3": d["v2"] / n,
        "phonon_eV_per_electron_step": (d["pop"] + d["iv"]) * hw / n,
    }


def test_fp32_1e7_20ps_vs_fp64_oracle_2e5(emc, oracle_mod):
    warm, blocks, per = 1000, 10, 100
    g_blocks, g_per = 19, 1000
    big = W.bulk(n_particles=10_000_000, seed=0, steps_per_launch=50)
    small = W.bulk(n_particles=200_000, seed=0)
    hw = small["hw_lo_eV"]

    def gpu_tally(ctx):
        o = ctx.emc_tally(emc.TALLY_OBS)[0]
        ev = ctx.emc_tally(emc.TALLY_EVENTS)[0].astype(np.int64)
        return {"n": o["n_samples"], "vz": o["sum_v"][2], "E": o["sum_E"],
                "v0": o["valley_steps"][0], "v1": o["valley_steps"][1], "v2": o["valley_steps"][2],
                "pop": ev[:, 2].sum() - ev[:, 1].sum(), "iv": ev[:, 5::2].sum() - ev[:, 4::2].sum()}

    def orc_tally(sim):
        t = sim.tallies()
        ev = t["events"].sum(axis=0).astype(np.int64)
        return {"n": t["n_samples"], "vz": t["sum_v"][2], "E": t["sum_E"],
                "v0": t["valley_steps"][0], "v1": t["valley_steps"][1], "v2": t["valley_steps"][2],
                "pop": ev[:, 2].sum() - ev[:, 1].sum(), "iv": ev[:, 5::2].sum() - ev[:, 4::2].sum()}

    with emc.Context(big) as ctx:
        ctx.emc_step(warm)
        g = block_means(ctx.emc_step, lambda: gpu_tally(ctx), g_blocks, g_per)
    sim = oracle_mod.Sim(small)
    sim.run(warm)
    o = block_means(sim.run, lambda: orc_tally(sim), blocks, per)
    G = [observables(b, hw) for b in g]
    O = [observables(b, hw) for b in o]
    report = {}
    for key in G[0]:
        gv = np.array([b[key] for b in G])
        ov = np.array([b[key] for b in O])
        sig = np.sqrt(gv.var(ddof=1) / len(gv) + ov.var(ddof=1) / len(ov))
        rel = (gv.mean() - ov.mean()) / ov.mean() if ov.mean() != 0 else 0.0
        report[key] = {"gpu_fp32_1e7": gv.mean(), "oracle_fp64_2e5": ov.mean(), "rel_error": rel,
                       "sigma_combined": sig}
        if key in ("f_U", "f_Gamma3") and ov.mean() < 1e-4:
            assert gv.mean() < 1e-3
            continue
        assert abs(gv.mean() - ov.mean()) <= max(0.01 * abs(ov.mean()), 3 * sig), (key, report[key])
    # the stated errors, also as a file in $EMC_ARTIFACT_DIR when set
    out = os.environ.get("EMC_ARTIFACT_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "precision_report.json"), "w") as f:
            json.dump(report, f, indent=1, default=float)
    print(json.dumps(report, indent=1, default=float))
