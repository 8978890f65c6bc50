"""Asynchronous tallies: every kind read through emc_tally_async (device
packing, one stream-ordered copy into page-locked memory) equals the
synchronous emc_tally read of the same state, for bulk and nanowire
contexts; the reset takes effect in stream order after the copy; and a
pipelined loop (step n + 1 enqueued before step n's tallies are read) gives
the same per-step values as the synchronous loop."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

KINDS = ["TALLY_OBS", "TALLY_EVENTS", "TALLY_HEAT", "TALLY_CHARGE", "TALLY_CROSSINGS", "TALLY_PHI", "TALLY_FIELD",
         "TALLY_HEAT_J", "TALLY_EVENTS_CELL"]


def obs_equal(a, dicts):
    for e, d in enumerate(dicts):
        for k, v in d.items():
            assert np.array_equal(np.asarray(a[k][e]), np.asarray(v)), (e, k)


@pytest.mark.parametrize("geom", ["bulk", "nanowire"])
def test_every_kind_equals_the_synchronous_read(emc, geom):
    if geom == "bulk":
        cfgs = [W.bulk(n_particles=800 + 50 * e, field_V_m=1e7 * (e + 1), seed=80 + e) for e in range(3)]
    else:
        cfgs = [W.nanowire(n_particles=2000, nx=10, Lx=100e-9, Vd=float(v), seed=90 + v) for v in (1, 2)]
    st = torch.cuda.Stream()
    with emc.Context(cfgs, stream=st.cuda_stream) as ctx:
        ctx.emc_step(30)
        bufs = {k: ctx.pinned_tally(getattr(emc, k)) for k in KINDS}
        for k in KINDS:
            ctx.emc_tally_async(getattr(emc, k), bufs[k])
        st.synchronize()
        for k in KINDS:
            want = ctx.emc_tally(getattr(emc, k))
            if k == "TALLY_OBS":
                obs_equal(bufs[k], want)
            else:
                assert np.array_equal(bufs[k], want), k


def test_reset_and_pipelined_loop(emc):
    cfgs = [W.nanowire(n_particles=3000, nx=10, Lx=100e-9, Vd=float(v), seed=95 + v) for v in (1, 3)]
    steps = 6
    # synchronous reference: per step, the heat map and crossings, then reset
    ref = []
    with emc.Context(cfgs) as ctx:
        for _ in range(steps):
            ctx.emc_step(10)
            h = ctx.emc_tally(emc.TALLY_HEAT).copy()
            c = ctx.emc_tally(emc.TALLY_CROSSINGS, reset=True).copy()
            ref.append((h, c))
    # pipelined: two buffer sets; step i + 1 is enqueued before step i is read
    st = torch.cuda.Stream()
    got = []
    with emc.Context(cfgs, stream=st.cuda_stream) as ctx:
        bufs = [(ctx.pinned_tally(emc.TALLY_HEAT), ctx.pinned_tally(emc.TALLY_CROSSINGS)) for _ in range(2)]
        ev = [torch.cuda.Event() for _ in range(2)]
        for i in range(steps):
            ctx.emc_step(10)
            h, c = bufs[i % 2]
            ctx.emc_tally_async(emc.TALLY_HEAT, h)
            ctx.emc_tally_async(emc.TALLY_CROSSINGS, c, reset=True)
            ev[i % 2].record(st)
            if i > 0:
                ev[(i - 1) % 2].synchronize()
                got.append(tuple(x.copy() for x in bufs[(i - 1) % 2]))
        ev[(steps - 1) % 2].synchronize()
        got.append(tuple(x.copy() for x in bufs[(steps - 1) % 2]))
    assert len(got) == steps
    for (h0, c0), (h1, c1) in zip(ref, got):
        assert np.array_equal(h0, h1) and np.array_equal(c0, c1)


def test_device_destination(emc):
    """With a device destination the packed tally lands in device memory
    (here a torch tensor on the context's stream) and equals the host read."""
    cfgs = [W.nanowire(n_particles=2000, nx=10, Lx=100e-9, Vd=float(v), seed=120 + v) for v in (1, 2)]
    st = torch.cuda.Stream()
    with emc.Context(cfgs, stream=st.cuda_stream) as ctx:
        ctx.emc_step(20)
        heat_d = torch.empty((2, ctx.n_cell, 2), dtype=torch.int64, device="cuda")
        hj_d = torch.empty((2, ctx.n_cell), dtype=torch.float64, device="cuda")
        obs_d = torch.empty(2 * emc.emc.OBS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        ctx.emc_tally_async(emc.TALLY_HEAT, heat_d.data_ptr(), device=True)
        ctx.emc_tally_async(emc.TALLY_HEAT_J, hj_d.data_ptr(), device=True)
        ctx.emc_tally_async(emc.TALLY_OBS, obs_d.data_ptr(), device=True)
        st.synchronize()
        assert np.array_equal(heat_d.cpu().numpy(), ctx.emc_tally(emc.TALLY_HEAT))
        assert np.array_equal(hj_d.cpu().numpy(), ctx.emc_tally(emc.TALLY_HEAT_J))
        obs_equal(obs_d.cpu().numpy().view(emc.emc.OBS_DTYPE), ctx.emc_tally(emc.TALLY_OBS))
