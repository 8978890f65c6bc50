"""The many-ensemble mixed batch (log-uniform sizes, random field,
temperature and doping, three bulk ensembles per nanowire one), run as one
context per geometry.  FP64 build: every ensemble reproduces its own oracle
run bit for bit.  FP32 build: the batch gives the same integer tallies as the
ensembles run one by one, and at the full 256-ensemble size the particle
bookkeeping closes exactly."""
import numpy as np
import pytest

import workloads as W
from tests.emc_harness import gpu_tallies, oracle_heat

pytestmark = pytest.mark.gpu


def contexts(emc, cfgs, **kw):
    groups = W.by_geometry(cfgs)
    return {g: (idx, emc.Context([cfgs[i] for i in idx], **kw)) for g, idx in groups.items()}


def test_mixed_batch_fp64_bit_exact(emc, oracle_mod):
    # 12 ensembles (9 bulk, 3 nanowire), N from 100 to 10,000; the nanowire
    # ones on a 20-cell-long wire so the oracle finishes in seconds
    cfgs = W.config_batched(n_ens=12, seed=5, scale=0.01)
    for i, c in enumerate(cfgs):
        if c["geometry"] == 1:
            cfgs[i] = W.nanowire(n_particles=c["n_particles"], Vd=c["Vd"] * 0.2, T=c["T"], Nd_cm3=c["Nd"] * 1e-6,
                                 seed=c["seed"], nx=20, Lx=200e-9)
    steps = 30
    ctxs = contexts(emc, cfgs, precision=emc.FP64)
    try:
        for g, (idx, ctx) in ctxs.items():
            ctx.emc_step(steps)
            for k, i in enumerate(idx):
                ref = oracle_mod.Sim(cfgs[i])
                ref.run(steps)
                rt = ref.tallies()
                t = gpu_tallies(emc, ctx, k)
                assert np.array_equal(t["events"], rt["events"].sum(axis=0)), i
                assert np.array_equal(t["obs"]["self_events"], rt["self_events"].astype(np.int64)), i
                assert np.array_equal(t["obs"]["valley_steps"], rt["valley_steps"]), i
                assert t["obs"]["sum_E"] == pytest.approx(rt["sum_E"], rel=1e-10), i
                if g == 1:
                    assert np.array_equal(t["heat"], oracle_heat(rt["events"])), i
                    assert np.array_equal(t["crossings"], rt["crossings"]), i
                    assert np.array_equal(t["charge"], rt["charge"]), i
                    assert t["obs"]["n_alive"] == rt["n_alive"], i
    finally:
        for _, ctx in ctxs.values():
            ctx.close()


def test_mixed_batch_equals_separate_fp32(emc):
    cfgs = W.config_batched(n_ens=8, seed=6, scale=0.05)
    steps = 20
    ctxs = contexts(emc, cfgs)
    try:
        for g, (idx, ctx) in ctxs.items():
            ctx.emc_step(steps)
            ev = ctx.emc_tally(emc.TALLY_EVENTS)
            cr = ctx.emc_tally(emc.TALLY_CROSSINGS)
            for k, i in enumerate(idx):
                with emc.Context(cfgs[i]) as one:
                    one.emc_step(steps)
                    assert np.array_equal(one.emc_tally(emc.TALLY_EVENTS)[0], ev[k]), i
                    assert np.array_equal(one.emc_tally(emc.TALLY_CROSSINGS)[0], cr[k]), i
    finally:
        for _, ctx in ctxs.values():
            ctx.close()


def test_full_mixed_batch_bookkeeping(emc):
    """256 ensembles, 5.5e7 electrons: after 20 fs every nanowire ensemble's
    live count equals initial + injected - absorbed, every bulk ensemble keeps
    all its electrons, and every ensemble samples each live particle-step."""
    cfgs = W.config_batched()
    steps = 20
    ctxs = contexts(emc, cfgs)
    try:
        for g, (idx, ctx) in ctxs.items():
            ctx.emc_step(steps)
            obs = ctx.emc_tally(emc.TALLY_OBS)
            cr = ctx.emc_tally(emc.TALLY_CROSSINGS).astype(np.int64)
            for k, i in enumerate(idx):
                n0 = cfgs[i]["n_particles"]
                if g == 0:
                    assert obs[k]["n_alive"] == n0
                    assert obs[k]["n_samples"] == n0 * steps
                else:
                    # crossings: source out, drain out, source in, drain in
                    assert obs[k]["n_alive"] == n0 - cr[k][0] - cr[k][1] + cr[k][2] + cr[k][3], i
                assert ctx.emc_tally(emc.TALLY_EVENTS)[k].sum() > 0
    finally:
        for _, ctx in ctxs.values():
            ctx.close()


def _batch_for_group():
    cfgs = W.config_batched(n_ens=12, seed=5, scale=0.01)
    for i, c in enumerate(cfgs):
        if c["geometry"] == 1:
            cfgs[i] = W.nanowire(n_particles=c["n_particles"], Vd=c["Vd"] * 0.2, T=c["T"], Nd_cm3=c["Nd"] * 1e-6,
                                 seed=c["seed"], nx=20, Lx=200e-9)
    g = W.by_geometry(cfgs)
    return [cfgs[i] for i in g[0]], [cfgs[i] for i in g[1]]


def _state(emc, ctx):
    d = ctx.debug_particles()
    keep = d["valley"] >= 0
    order = np.lexsort((d["id"][keep], d["ens"][keep]))
    return {k: v[keep][order] for k, v in d.items()}, {
        "events": ctx.emc_tally(emc.TALLY_EVENTS_CELL), "cross": ctx.emc_tally(emc.TALLY_CROSSINGS),
        "charge": ctx.emc_tally(emc.TALLY_CHARGE),
        "alive": [o["n_alive"] for o in ctx.emc_tally(emc.TALLY_OBS)],
        "samples": [o["n_samples"] for o in ctx.emc_tally(emc.TALLY_OBS)]}


@pytest.mark.parametrize("prec_name,kinds", [("FP64", "bulk+wire"), ("FP32", "bulk+wire"), ("FP32", "wire+wire")])
def test_group_step_equals_separate_steps(emc, prec_name, kinds):
    """emc_group_step: the bulk and the nanowire contexts of the mixed batch
    (or two nanowire contexts) in one flight launch per chunk give the same
    particles and integer tallies as each context stepped alone, across
    Poisson periods and a partial one."""
    prec = getattr(emc, prec_name)
    bulk, wire = _batch_for_group()
    pair = (bulk, wire) if kinds == "bulk+wire" else (wire, [dict(c, seed=c["seed"] + 1000) for c in wire])
    steps = 3 * wire[0]["steps_per_poisson"] + 4
    alone = []
    for cf in pair:
        with emc.Context(cf, precision=prec) as ctx:
            ctx.emc_step(steps)
            alone.append(_state(emc, ctx))
    a, b = emc.Context(pair[0], precision=prec), emc.Context(pair[1], precision=prec)
    try:
        emc.emc.group_step([a, b], steps - 4)
        emc.emc.group_step([a, b], 4)
        together = [_state(emc, a), _state(emc, b)]
    finally:
        a.close()
        b.close()
    for (pa, ta), (pb, tb) in zip(alone, together):
        for k in ("k", "r", "tr", "valley", "ens", "id", "ctr"):
            assert np.array_equal(pa[k], pb[k]), k
        for k in ("events", "cross", "charge"):
            assert np.array_equal(ta[k], tb[k]), k
        assert ta["alive"] == tb["alive"] and ta["samples"] == tb["samples"]


def test_group_step_refuses_mismatched_contexts(emc):
    bulk, wire = _batch_for_group()
    with emc.Context(wire) as a, emc.Context([dict(c, seed=c["seed"] + 7) for c in wire]) as b:
        a.emc_step(3)  # out of phase
        with pytest.raises(emc.EmcError):
            emc.emc.group_step([a, b], 10)
    with emc.Context(bulk) as a, emc.Context(wire, precision=emc.FP64) as b:
        with pytest.raises(emc.EmcError):
            emc.emc.group_step([a, b], 10)
