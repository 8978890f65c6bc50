"""One wire's particles sharded over several contexts with the integer
charge exchange before each Poisson update, against the unsharded run of
the same wire and against the oracle.  Every particle keeps its global id
and Philox stream, so the union of the shards must follow the unsharded run
bit for bit: the same particle states (FP64 and FP32), the same per-subcell
event counts, crossings, charge, refill counts and potential.

The shards of a test live in one process on one GPU as separate contexts;
their exchange runs on the host between launches (no kernel of one shard
waits on another's)."""
import numpy as np
import pytest

import workloads as W
from paper_1707_09073_gb300 import shard as SH

pytestmark = pytest.mark.gpu


def _particles_by_gid(emc, ctx, cfgs):
    """Live particles of a context keyed by (ensemble, global id)."""
    d = ctx.debug_particles()
    out = {}
    for s in range(d["id"].size):
        if d["valley"][s] < 0:  # free slot
            continue
        e = int(d["ens"][s])
        c = cfgs[e]
        i = int(d["id"][s])
        n0 = int(c["n_particles"])
        if c.get("shard_n_global", 0):
            g = c["shard_live_base"] + i if i < n0 else c["shard_spare_base"] + i - n0
        else:
            g = i
        out[(e, g)] = (d["k"][s].tobytes(), d["r"][s].tobytes(), d["tr"][s].tobytes(), int(d["valley"][s]),
                       int(d["ctr"][s]))
    return out


def _wire_tallies(emc, t):
    obs = t.emc_tally(emc.TALLY_OBS)
    return {
        "events": np.asarray(t.emc_tally(emc.TALLY_EVENTS_CELL)),
        "cross": np.asarray(t.emc_tally(emc.TALLY_CROSSINGS)),
        "charge": np.asarray(t.emc_tally(emc.TALLY_CHARGE)),
        "phi": np.asarray(t.emc_tally(emc.TALLY_PHI)),
        "alive": [o["n_alive"] for o in obs],
        "starved": [o["inject_starved"] for o in obs],
        "samples": [o["n_samples"] for o in obs],
        "valley_steps": [list(o["valley_steps"]) for o in obs],
        "self": [list(o["self_events"]) for o in obs],
    }


def _assert_same(a, b):
    for k in ("events", "cross", "charge"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("alive", "starved", "samples", "valley_steps", "self"):
        assert a[k] == b[k], (k, a[k], b[k])
    assert np.array_equal(a["phi"], b["phi"])


@pytest.mark.parametrize("prec_name,world", [("FP64", 2), ("FP64", 3), ("FP32", 2), ("FP32", 4)])
def test_sharded_wire_equals_unsharded(emc, prec_name, world):
    """Two ensembles (2 V and 6 V), 12 Poisson periods with contact refills,
    a sort every 4 launches: shards vs one context, bit for bit."""
    prec = getattr(emc, prec_name)
    cfgs = [W.nanowire(n_particles=9000, nx=20, Lx=200e-9, Vd=v, seed=40 + i, sort_period=4)
            for i, v in enumerate((2.0, 6.0))]
    steps = 12 * cfgs[0]["steps_per_poisson"] + 3
    with emc.Context(cfgs, precision=prec) as ctx:
        ctx.emc_step(steps)
        want = _wire_tallies(emc, ctx)
        want_p = _particles_by_gid(emc, ctx, cfgs)
    with SH.LocalWire(cfgs, world, precision=prec) as wire:
        wire.emc_step(steps)
        got = _wire_tallies(emc, wire)
        got_p = {}
        for c in wire.ctxs:
            got_p.update(_particles_by_gid(emc, c, c.cfgs))
    assert sum(want["cross"][0][2:]) > 0  # refills happened
    _assert_same(got, want)
    assert got_p.keys() == want_p.keys()
    assert all(got_p[k] == want_p[k] for k in want_p)


def test_sharded_refill_starved_equals_unsharded(emc):
    """Too few spare slots: the wire's free ids run out, and which ids refill
    which contact subcell follows the global free-id order across shards."""
    # no spare slots and a refill every step: the initial contact-subcell
    # deficits exceed the ids freed by the few electrons that leave in a step
    cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=0.0, seed=5, spare=0, steps_per_poisson=1)
    steps = 30
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        want = _wire_tallies(emc, ctx)
        want_p = _particles_by_gid(emc, ctx, [cfg])
    assert want["starved"][0] > 0
    with SH.LocalWire(cfg, 3, precision=emc.FP64) as wire:
        wire.emc_step(steps)
        got = _wire_tallies(emc, wire)
        got_p = {}
        for c in wire.ctxs:
            got_p.update(_particles_by_gid(emc, c, c.cfgs))
    _assert_same(got, want)
    assert got_p == want_p


def test_sharded_wire_matches_oracle(emc, oracle_mod):
    """FP64 shards against the oracle's unsharded wire: the integer tallies
    bit for bit (the parity test of the unsharded context, through shards)."""
    cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=2.0, seed=7)
    steps = 40
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    with SH.LocalWire(cfg, 2, precision=emc.FP64) as wire:
        wire.emc_step(steps)
        ev = np.asarray(wire.emc_tally(emc.TALLY_EVENTS_CELL))[0]
        cross = np.asarray(wire.emc_tally(emc.TALLY_CROSSINGS))[0]
        charge = np.asarray(wire.emc_tally(emc.TALLY_CHARGE))[0]
        obs = wire.emc_tally(emc.TALLY_OBS)[0]
    assert np.array_equal(ev, rt["events"])
    assert np.array_equal(cross, rt["crossings"])
    assert np.array_equal(charge, rt["charge"])
    assert obs["n_alive"] == rt["n_alive"]


def test_shard_protocol_errors(emc):
    cfg = W.nanowire(n_particles=2000, nx=20, Lx=200e-9, Vd=2.0, seed=1)
    K = cfg["steps_per_poisson"]
    with emc.Context(cfg) as ctx:  # unsharded: no exchange
        with pytest.raises(emc.EmcError):
            ctx.emc_shard_counts()
    c0 = SH.shard_config(cfg, 0, 2)
    with emc.Context(c0) as ctx:
        with pytest.raises(emc.EmcError):  # the initial exchange is pending
            ctx.emc_step(1)
        with pytest.raises(emc.EmcError):
            ctx.emc_get_state()
        q, f = ctx.emc_shard_counts()
        assert q.sum() == c0["n_particles"]
        ctx.emc_shard_tail(q, np.zeros_like(f), f, True)
        with pytest.raises(emc.EmcError):  # nothing pending any more
            ctx.emc_shard_tail(q, np.zeros_like(f), f, True)
        with pytest.raises(emc.EmcError):  # across the end of a period
            ctx.emc_step(K + 1)
        ctx.emc_step(K)
        with pytest.raises(emc.EmcError):
            ctx.emc_set_bias(0, 0.0, 1.0, 0.0)
        q, f = ctx.emc_shard_counts()
        with pytest.raises(emc.EmcError):  # prefix above the total
            ctx.emc_shard_tail(q, f + 1, f, True)


def test_sharded_wire_with_subcell_temperatures_and_resume(emc):
    """Shards under per-subcell lattice temperatures (set between periods,
    as the electrothermal loop does) follow the unsharded run bit for bit,
    and a checkpoint of every shard taken after an exchange resumes into
    fresh shard contexts with the same continuation (FP64)."""
    cfg = W.nanowire(n_particles=8000, nx=20, Lx=200e-9, Vd=5.0, seed=61)
    K = cfg["steps_per_poisson"]
    C = cfg["nx"] * cfg["ny"] * cfg["nz"]
    T = 300.0 + 60.0 * np.linspace(0.0, 1.0, C)
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(3 * K)
        ctx.emc_set_temperature(0, T)
        ctx.emc_step(6 * K)
        want = _wire_tallies(emc, ctx)
        want_p = _particles_by_gid(emc, ctx, [cfg])
    with SH.LocalWire(cfg, 2, precision=emc.FP64) as wire:
        wire.emc_step(3 * K)
        for c in wire.ctxs:
            c.emc_set_temperature(0, T)
        wire.emc_step(3 * K)
        blobs = [c.emc_get_state() for c in wire.ctxs]
        wire.emc_step(3 * K)
        got = _wire_tallies(emc, wire)
        got_p = {}
        for c in wire.ctxs:
            got_p.update(_particles_by_gid(emc, c, c.cfgs))
    _assert_same(got, want)
    assert got_p == want_p
    # resume the checkpoint into fresh shards and finish the same steps
    with SH.LocalWire(cfg, 2, precision=emc.FP64) as wire:
        for c, b in zip(wire.ctxs, blobs):  # the blob carries the temperature tables
            c.emc_set_state(b)
        wire.steps = 6 * K
        wire.emc_step(3 * K)
        res_p = {}
        for c in wire.ctxs:
            res_p.update(_particles_by_gid(emc, c, c.cfgs))
    assert res_p == want_p


NCCL_SCRIPT = r'''
import os, numpy as np, torch, torch.distributed as dist
import workloads as W
import paper_1707_09073_gb300 as emc
from paper_1707_09073_gb300 import shard as SH
torch.cuda.set_device(0)
dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % int(os.environ["PORT"]), rank=0, world_size=1)
cfg = W.nanowire(n_particles=9000, nx=20, Lx=200e-9, Vd=3.0, seed=44)
steps = 5 * cfg["steps_per_poisson"] + 2
with emc.Context(cfg, precision=emc.FP64) as ctx:
    ctx.emc_step(steps)
    want = [ctx.emc_tally(k) for k in (emc.TALLY_EVENTS_CELL, emc.TALLY_CROSSINGS, emc.TALLY_CHARGE, emc.TALLY_PHI)]
    wp = ctx.debug_particles()
wire = SH.DistWire(cfg, precision=emc.FP64)
assert wire.device.type == "cuda"
wire.emc_step(steps)
got = [wire.emc_tally(k) for k in (emc.TALLY_EVENTS_CELL, emc.TALLY_CROSSINGS, emc.TALLY_CHARGE, emc.TALLY_PHI)]
gp = wire.ctx.debug_particles()
for a, b in zip(want, got):
    assert np.array_equal(np.asarray(a), np.asarray(b))
def live(d):
    return {int(d["id"][s]): (d["k"][s].tobytes(), d["r"][s].tobytes(), int(d["valley"][s]), int(d["ctr"][s]))
            for s in range(d["id"].size) if d["valley"][s] >= 0}
assert live(wp) == live(gp)
wire.close()
dist.destroy_process_group()
print("nccl shard ok")
'''


def test_dist_wire_over_nccl_one_rank(emc):
    """The torch.distributed driver on the NCCL backend (one rank on this
    GPU; no kernel waits on another rank): the exchange runs in device
    memory (the library writes and reads the counts there, the collectives
    run on device tensors) and the run equals the unsharded context bit for
    bit (FP64)."""
    import os
    import socket
    import subprocess
    import sys
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PORT=str(port), NCCL_NVLS_ENABLE="0", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", NCCL_SCRIPT], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "nccl shard ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
