"""One nanowire's particles split over several contexts, with the integer
charge exchange of the Poisson update: the field of every period follows
from the electron count of each subcell summed over all particles of the
wire (the Poisson passage next to Table I), so at the end of each period the
shards add their counts, then every shard refills the contacts and solves
the same FP64 Poisson problem.

Every particle keeps its global id and with it its Philox stream, so the
union of the shards reproduces, bit for bit, the run of one unsharded
context: the same particle states and the same integer tallies (summed over
the shards).

- ``shard_config``: the configuration of one shard.
- ``exchange``: the exchange arithmetic (summed counts; free ids of the
  shards below and of the whole wire).
- ``LocalWire``: several shards in one process (the exchange on the host).
- ``DistWire``: one shard per rank of a ``torch.distributed`` group (an
  all-reduce of the counts and an all-gather of the free-id counts per
  period; gloo on CPU tensors, NCCL on device tensors).

Argument marshalling and host bookkeeping only; every step of the path runs
in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import emc as _emc

# tallies that are the wire's on every shard (not summed over shards)
WIRE_TALLIES = (_emc.TALLY_CHARGE, _emc.TALLY_PHI, _emc.TALLY_FIELD)
_OBS_SAME = ("steps_done",)


def _split(n: int, parts: int, r: int):
    """Start and size of part r of n items split as evenly as possible."""
    q, m = divmod(int(n), int(parts))
    return r * q + min(r, m), q + (1 if r < m else 0)


def shard_config(cfg: dict, rank: int, world: int) -> dict:
    """Shard ``rank`` of ``world`` of the wire ``cfg``: a contiguous range of
    the initial-electron ids [0, N) and one of the spare ids [N, capacity)."""
    if not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    N, cap = int(cfg["n_particles"]), max(int(cfg["capacity"]), int(cfg["n_particles"]))
    live0, n_live = _split(N, world, rank)
    spare0, n_spare = _split(cap - N, world, rank)
    c = dict(cfg)
    c["n_particles"] = n_live
    c["capacity"] = n_live + n_spare
    c["shard_n_global"] = N
    c["shard_live_base"] = live0
    c["shard_spare_base"] = N + spare0
    return c


def exchange(charges, frees, rank: int):
    """Inputs of emc_shard_tail for shard ``rank`` from every shard's
    emc_shard_counts: (charge_global int32[E][C], free_prefix int64[E][2],
    free_total int64[E][2], lead).  ``charges``: the counts of all shards,
    or their sum already (an array of shape [E][C]); ``frees``: [R][E][2]."""
    q = np.asarray(charges, dtype=np.int64)
    if q.ndim == 3:
        q = q.sum(axis=0)
    f = np.asarray(frees, dtype=np.int64)
    prefix = f[:rank].sum(axis=0) if rank > 0 else np.zeros_like(f[0])
    return q.astype(np.int32), prefix, f.sum(axis=0), rank == 0


def _sum_tallies(kind, parts):
    if kind in WIRE_TALLIES:
        return parts[0]
    if kind == _emc.TALLY_OBS:
        out = []
        for e in range(len(parts[0])):
            d = {}
            for k, v in parts[0][e].items():
                if k in _OBS_SAME:
                    d[k] = v
                else:
                    d[k] = (np.sum([np.asarray(p[e][k]) for p in parts], axis=0)).tolist() \
                        if np.ndim(v) else type(v)(sum(p[e][k] for p in parts))
            out.append(d)
        return out
    return np.sum(parts, axis=0, dtype=np.asarray(parts[0]).dtype)


class LocalWire:
    """``world`` shards of the wire(s) ``cfgs`` in one process.  Each shard
    is its own context (its own launches); the exchange runs on the host
    between launches, so no kernel of one shard waits for another's."""

    def __init__(self, cfgs, world: int, precision: int = _emc.FP32):
        cfgs = [cfgs] if isinstance(cfgs, dict) else list(cfgs)
        self.world = int(world)
        self.K = int(cfgs[0]["steps_per_poisson"])
        self.steps = 0
        self.ctxs = []
        try:
            for r in range(self.world):
                self.ctxs.append(_emc.Context([shard_config(c, r, self.world) for c in cfgs], precision))
            self._exchange()
        except Exception:
            self.close()
            raise

    def _exchange(self):
        counts = [c.emc_shard_counts() for c in self.ctxs]
        qs, fs = [q for q, _ in counts], [f for _, f in counts]
        for r, c in enumerate(self.ctxs):
            c.emc_shard_tail(*exchange(qs, fs, r))

    def emc_step(self, n: int):
        n = int(n)
        while n > 0:
            into = self.steps % self.K
            k = min(n, self.K - into)
            for c in self.ctxs:
                c.emc_step(k)
            self.steps += k
            n -= k
            if into + k == self.K:
                self._exchange()

    def emc_tally(self, kind: int, reset: bool = False):
        return _sum_tallies(kind, [c.emc_tally(kind, reset=reset) for c in self.ctxs])

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DistWire:
    """This rank's shard of the wire(s) ``cfgs`` in a ``torch.distributed``
    group: per Poisson period one all-reduce of the int64 subcell counts and
    one all-gather of the free-id counts.  ``make_context(cfgs)`` builds the
    shard's context (default: a library context of ``precision``); tensors
    live on ``device`` (CPU for gloo, the rank's GPU for NCCL)."""

    def __init__(self, cfgs, precision: int = _emc.FP32, group=None, device=None, make_context=None):
        import torch
        import torch.distributed as dist
        self._torch, self._dist, self.group = torch, dist, group
        cfgs = [cfgs] if isinstance(cfgs, dict) else list(cfgs)
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if device is None:
            device = torch.device("cpu") if dist.get_backend(group) == "gloo" else \
                torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.K = int(cfgs[0]["steps_per_poisson"])
        self.steps = 0
        mine = [shard_config(c, self.rank, self.world) for c in cfgs]
        self.ctx = make_context(mine) if make_context else _emc.Context(mine, precision)
        self._exchange()

    def _exchange(self):
        torch, dist = self._torch, self._dist
        if self.device.type == "cuda" and isinstance(self.ctx, _emc.Context):
            return self._exchange_device()
        q, f = self.ctx.emc_shard_counts()
        qt = torch.from_numpy(np.ascontiguousarray(q, dtype=np.int64)).to(self.device)
        dist.all_reduce(qt, group=self.group)
        ft = torch.from_numpy(np.ascontiguousarray(f, dtype=np.int64)).to(self.device)
        fall = [torch.empty_like(ft) for _ in range(self.world)]
        dist.all_gather(fall, ft, group=self.group)
        fs = np.stack([t.cpu().numpy() for t in fall])
        self.ctx.emc_shard_tail(*exchange(qt.cpu().numpy(), fs, self.rank))

    def _exchange_device(self):
        """The exchange in device memory (NCCL): the library writes the
        counts straight into device tensors, the collectives run on them, the
        prefix and total of the free-id counts are summed on the device and
        the library reads them back from there."""
        torch, dist = self._torch, self._dist
        E, Cn = self.ctx.n_ens, self.ctx.n_cell
        if not hasattr(self, "_dq"):
            self._dq = torch.empty((E, Cn), dtype=torch.int32, device=self.device)
            self._df = torch.empty((E, 2), dtype=torch.int64, device=self.device)
            self._dall = torch.empty((self.world, E, 2), dtype=torch.int64, device=self.device)
        self.ctx.emc_shard_counts_ptr(self._dq.data_ptr(), self._df.data_ptr())
        dist.all_reduce(self._dq, group=self.group)
        dist.all_gather_into_tensor(self._dall, self._df, group=self.group)
        pre = self._dall[:self.rank].sum(dim=0) if self.rank > 0 else torch.zeros_like(self._df)
        tot = self._dall.sum(dim=0)
        pre, tot = pre.contiguous(), tot.contiguous()
        torch.cuda.current_stream(self.device).synchronize()  # the collectives are done
        self.ctx.emc_shard_tail_ptr(self._dq.data_ptr(), pre.data_ptr(), tot.data_ptr(), self.rank == 0)

    def emc_step(self, n: int):
        n = int(n)
        while n > 0:
            into = self.steps % self.K
            k = min(n, self.K - into)
            self.ctx.emc_step(k)
            self.steps += k
            n -= k
            if into + k == self.K:
                self._exchange()

    def emc_tally(self, kind: int, reset: bool = False):
        """The wire's tally: this shard's summed over the group (the wire's
        charge, potential and field are every shard's already)."""
        torch, dist = self._torch, self._dist
        mine = self.ctx.emc_tally(kind, reset=reset)
        if kind in WIRE_TALLIES:
            return mine
        if kind == _emc.TALLY_OBS:
            parts = [None] * self.world
            dist.all_gather_object(parts, mine, group=self.group)
            return _sum_tallies(kind, parts)
        a = np.ascontiguousarray(mine)
        t = torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).to(self.device)
        dist.all_reduce(t, group=self.group)
        out = t.cpu().numpy()
        return out.view(np.uint64) if a.dtype == np.uint64 else out

    def close(self):
        self.ctx.close()
