"""Host logic of the particle-sharded wire (no GPU): the split of the
wire's ids over shards, the exchange arithmetic, and the torch.distributed
driver on two gloo ranks with stand-in contexts that record what the driver
hands them."""
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_1707_09073_gb300 import shard as SH


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_shards_partition_the_wire_ids(world):
    cfg = W.nanowire(n_particles=1001, nx=20, Lx=200e-9, spare=333)
    N, cap = cfg["n_particles"], cfg["capacity"]
    live, spare = [], []
    prev_l = prev_s = -1
    for r in range(world):
        c = SH.shard_config(cfg, r, world)
        assert c["shard_n_global"] == N
        assert c["shard_live_base"] > prev_l and c["shard_spare_base"] > prev_s  # ordered alike
        prev_l, prev_s = c["shard_live_base"], c["shard_spare_base"]
        live += range(c["shard_live_base"], c["shard_live_base"] + c["n_particles"])
        spare += range(c["shard_spare_base"], c["shard_spare_base"] + c["capacity"] - c["n_particles"])
    assert live == list(range(N))
    assert spare == list(range(N, cap))


def test_exchange_arithmetic():
    rng = np.random.default_rng(0)
    q = rng.integers(0, 50, size=(3, 2, 7))
    f = rng.integers(0, 9, size=(3, 2, 2))
    for r in range(3):
        cg, pre, tot, lead = SH.exchange(list(q), f, r)
        assert cg.dtype == np.int32 and np.array_equal(cg, q.sum(axis=0))
        assert np.array_equal(pre, f[:r].sum(axis=0) if r else np.zeros((2, 2)))
        assert np.array_equal(tot, f.sum(axis=0))
        assert lead == (r == 0)
    # an already summed count is passed through
    cg, *_ = SH.exchange(q.sum(axis=0), f, 1)
    assert np.array_equal(cg, q.sum(axis=0))


class _FakeShard:
    """Stand-in context: counts that depend on the rank, the ensemble, the
    subcell and the number of exchanges so far; records every tail."""

    def __init__(self, cfgs, rank):
        self.cfgs, self.rank = cfgs, rank
        self.E, self.C = len(cfgs), cfgs[0]["nx"] * cfgs[0]["ny"] * cfgs[0]["nz"]
        self.n_ex, self.steps, self.tails = 0, [], []

    def counts(self, rank, n_ex):
        q = (np.arange(self.E * self.C).reshape(self.E, self.C) * (rank + 1) + 7 * n_ex) % 13
        f = np.array([[rank + e + n_ex, 2 * rank + 1] for e in range(self.E)], dtype=np.int64)
        return q.astype(np.int32), f

    def emc_shard_counts(self):
        return self.counts(self.rank, self.n_ex)

    def emc_shard_tail(self, q, pre, tot, lead):
        self.tails.append((np.array(q), np.array(pre), np.array(tot), bool(lead)))
        self.n_ex += 1

    def emc_step(self, k):
        self.steps.append(int(k))

    def emc_tally(self, kind, reset=False):
        from paper_1707_09073_gb300 import emc as E
        if kind == E.TALLY_EVENTS_CELL:
            return np.full((self.E, self.C, 3, 10), 2**62 + self.rank, dtype=np.uint64)
        if kind == E.TALLY_CHARGE:
            return np.full((self.E, self.C), 5, dtype=np.int64)
        raise KeyError(kind)

    def close(self):
        pass


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_1707_09073_gb300 import emc as E
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        cfgs = [W.nanowire(n_particles=100, nx=4, ny=1, nz=2, Lx=40e-9, Vd=v, seed=v) for v in (1.0, 2.0)]
        box = {}

        def make(mine):
            box["s"] = _FakeShard(mine, rank)
            return box["s"]

        wire = SH.DistWire(cfgs, group=None, make_context=make)
        K = cfgs[0]["steps_per_poisson"]
        wire.emc_step(2 * K + 3)
        wire.emc_step(K - 3)
        fake = box["s"]
        ev = wire.emc_tally(E.TALLY_EVENTS_CELL)
        ch = wire.emc_tally(E.TALLY_CHARGE)
        q.put((rank, fake.steps, fake.tails, [c["shard_live_base"] for c in fake.cfgs], ev.ravel()[:3].tolist(),
               int(ch.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_dist_wire_gloo_world_2():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, *rest = q.get(timeout=180)
        got[r] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfgs = [W.nanowire(n_particles=100, nx=4, ny=1, nz=2, Lx=40e-9, Vd=v, seed=v) for v in (1.0, 2.0)]
    K = cfgs[0]["steps_per_poisson"]
    fakes = [_FakeShard(cfgs, r) for r in range(world)]
    for r in range(world):
        steps, tails, bases, ev, charge = got[r]
        # steps never cross the end of a period; one exchange at init and
        # one per completed period
        assert steps == [K, K, 3, K - 3]
        assert len(tails) == 1 + 3
        for n_ex, (qg, pre, tot, lead) in enumerate(tails):
            cs = [fakes[s].counts(s, n_ex) for s in range(world)]
            wq, wpre, wtot, wlead = SH.exchange([c[0] for c in cs], [c[1] for c in cs], r)
            assert np.array_equal(qg, wq) and np.array_equal(pre, wpre) and np.array_equal(tot, wtot)
            assert lead == wlead
        assert bases == [SH.shard_config(c, r, world)["shard_live_base"] for c in cfgs]
        # unsigned event counts summed over ranks (wrapping like uint64); the
        # wire's charge is not summed
        assert ev == [(2 * 2**62 + 1) % 2**64] * 3
        assert charge == 5 * 2 * 8
