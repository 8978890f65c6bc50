"""The benchmarked workload at its full size, in the launch configuration the
bench times (21 bias points x 200,000 superparticles, 3 x 6 x 100 subcells,
block 256, 16 KiB of the table staged, a sort every 10 launches), checked
where the oracle can follow it and through properties that hold at any
size.

- FP64 parity build of the whole sweep: every ensemble is independent, so
  the oracle's run of one bias point must give exactly the tallies of that
  ensemble inside the 21-ensemble context (sampled: the coolest, a middle
  and the hottest bias point).
- FP32 production build of the whole sweep: particle bookkeeping (live =
  initial + refilled - left), the subcell charge equal to the live count at
  a Poisson update, per-subcell event counts summing to the per-ensemble
  counts, the heat tally equal to the events' net phonons."""
import numpy as np
import pytest

import workloads as W
from emc_harness import oracle_heat

pytestmark = pytest.mark.gpu

LAUNCH = dict(block_size=256, table_smem_kb=16, sort_period=10)


def _sweep():
    return [dict(c, **LAUNCH) for c in W.config_nanowire_sweep()]


def test_full_sweep_fp64_matches_the_oracle_per_ensemble(emc, oracle_mod):
    cfgs = _sweep()
    steps = 30
    with emc.Context(cfgs, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        ev = ctx.emc_tally(emc.TALLY_EVENTS_CELL)
        cross = ctx.emc_tally(emc.TALLY_CROSSINGS)
        charge = ctx.emc_tally(emc.TALLY_CHARGE)
        obs = ctx.emc_tally(emc.TALLY_OBS)
    cores = oracle_mod.host_cores()
    for e in (0, 10, 20):
        ref = oracle_mod.Sim(cfgs[e], threads=cores)
        ref.run(steps)
        rt = ref.tallies()
        assert np.array_equal(ev[e], rt["events"]), e
        assert np.array_equal(cross[e], rt["crossings"]), e
        assert np.array_equal(charge[e], rt["charge"]), e
        assert obs[e]["n_alive"] == rt["n_alive"], e


def test_full_sweep_fp32_bookkeeping(emc):
    cfgs = _sweep()
    K = cfgs[0]["steps_per_poisson"]
    with emc.Context(cfgs) as ctx:
        ctx.emc_step(50 * K)
        obs = ctx.emc_tally(emc.TALLY_OBS)
        cross = ctx.emc_tally(emc.TALLY_CROSSINGS)
        charge = ctx.emc_tally(emc.TALLY_CHARGE)
        ev_cell = ctx.emc_tally(emc.TALLY_EVENTS_CELL)
        ev = ctx.emc_tally(emc.TALLY_EVENTS)
        heat = ctx.emc_tally(emc.TALLY_HEAT)
    for e, c in enumerate(cfgs):
        o = obs[e]
        out, inn = int(cross[e][0] + cross[e][1]), int(cross[e][2] + cross[e][3])
        assert o["n_alive"] == c["n_particles"] + inn - out, e
        assert int(charge[e].sum()) == o["n_alive"], e
        assert np.array_equal(ev_cell[e].sum(axis=0), ev[e]), e
        assert np.array_equal(heat[e], oracle_heat(ev_cell[e])), e
        assert o["n_samples"] > 0 and np.all(np.isfinite(o["sum_v"]))
    # the drain current rises with the bias at first (a sanity check of the sweep)
    net = np.array([int(cross[e][1]) - int(cross[e][3]) for e in range(len(cfgs))])
    assert net[5] > net[0] and net[20] > net[1]
