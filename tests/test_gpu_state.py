"""Checkpoint/resume through the C ABI (emc_state_size / emc_get_state /
emc_set_state) and the failure paths of invalid inputs.

- 2N steps in one context equal N steps, a state copy into a fresh context of
  the same ensembles, and N more steps: bit for bit in the FP64 build
  (particles and integer tallies; FP64 sums to rounding of the atomic order),
  identical particles and integer tallies in the FP32 production build, with
  particle sorting, the captured refill/Poisson graph and subcell
  temperatures in play.
- A blob of other ensembles, or a short one, is refused with a status.
- Non-finite terminal voltages or charge densities are refused on the host
  (EMC_EINVAL, nothing changes); a non-finite particle energy planted through
  the state blob is caught on the device and reported by the next tally
  (EMC_EOVERFLOW naming it), and restoring a clean state clears it.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def snapshot(emc, ctx):
    # particles by (ensemble, id): sorting may place equal keys in any slot order
    p = ctx.debug_particles()
    order = np.lexsort((p["id"], p["ens"]))
    p = {k: v[order] for k, v in p.items()}
    return {
        "events_cell": ctx.emc_tally(emc.TALLY_EVENTS_CELL),
        "crossings": ctx.emc_tally(emc.TALLY_CROSSINGS),
        "charge": ctx.emc_tally(emc.TALLY_CHARGE),
        "phi": ctx.emc_tally(emc.TALLY_PHI),
        "obs": ctx.emc_tally(emc.TALLY_OBS),
        "particles": p,
    }


def assert_same(a, b, exact_floats: bool, sum_rtol: float):
    for k in ("events_cell", "crossings", "charge"):
        assert np.array_equal(a[k], b[k]), k
    for oa, ob in zip(a["obs"], b["obs"]):
        for k in ("n_samples", "valley_steps", "self_events", "overflow", "steps_done", "n_alive"):
            assert np.array_equal(oa[k], ob[k]), k
        # ensemble sums: the order of the block and warp additions may differ
        np.testing.assert_allclose(oa["sum_E"], ob["sum_E"], rtol=sum_rtol)
        np.testing.assert_allclose(oa["sum_v"], ob["sum_v"], rtol=sum_rtol, atol=sum_rtol * np.abs(oa["sum_v"]).max())
    for k in ("valley", "ens", "id", "ctr"):
        assert np.array_equal(a["particles"][k], b["particles"][k]), k
    for k in ("k", "r", "tr"):
        if exact_floats:
            assert np.array_equal(a["particles"][k], b["particles"][k]), k
        else:
            np.testing.assert_array_equal(a["particles"][k], b["particles"][k])
    if exact_floats:
        np.testing.assert_allclose(a["phi"], b["phi"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_resume_equals_continuous_run(emc, prec):
    torch = pytest.importorskip("torch")
    precision = getattr(emc, prec)
    cfgs = [W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=float(v), seed=300 + v, sort_period=2) for v in (2, 5)]
    C = 20 * 3 * 6
    T = 300.0 + 120.0 * np.exp(-((np.arange(C) // 18 - 14) / 4.0) ** 2)
    st = torch.cuda.Stream()
    N = 30

    def start(ctx):
        ctx.emc_step(10)
        ctx.emc_set_temperature(1, T)
        ctx.emc_step(N - 10)

    with emc.Context(cfgs, precision=precision, stream=st.cuda_stream) as a:
        start(a)
        a.emc_step(N)
        want = snapshot(emc, a)
    with emc.Context(cfgs, precision=precision, stream=st.cuda_stream) as b:
        start(b)
        blob = b.emc_get_state()
    # the resumed context: launch tuning may differ, the ensembles may not
    tuned = [W.copy_config(c, block_size=128) for c in cfgs]
    with emc.Context(tuned, precision=precision, stream=st.cuda_stream) as c:
        c.emc_set_state(blob)
        c.emc_step(N)
        got = snapshot(emc, c)
    # FP64 sums to 1e-12; the FP32 build's compensated float sums to 1e-6
    assert_same(want, got, exact_floats=True, sum_rtol=1e-12 if prec == "FP64" else 1e-6)
    assert got["obs"][0]["steps_done"] == 2 * N


def test_foreign_or_short_blob_is_refused(emc):
    cfg = W.nanowire(n_particles=2000, nx=10, Lx=100e-9, Vd=1.0, seed=5)
    with emc.Context(cfg) as a:
        a.emc_step(10)
        blob = a.emc_get_state()
    with emc.Context(W.copy_config(cfg, seed=6)) as b:
        with pytest.raises(emc.EmcError) as e:
            b.emc_set_state(blob)
        assert e.value.status == 6  # EMC_ESTATE
    with emc.Context(cfg) as c:
        with pytest.raises(emc.EmcError) as e:
            c.emc_set_state(blob[:-8])
        assert e.value.status == 1  # EMC_EINVAL
        with pytest.raises(emc.EmcError):
            c.emc_set_state(np.zeros(100, np.uint8))
        c.emc_step(10)  # still usable


def test_non_finite_inputs_are_refused(emc):
    cfg = W.nanowire(n_particles=2000, nx=10, Lx=100e-9, Vd=1.0, seed=7)
    with emc.Context(cfg) as ctx:
        ctx.emc_step(10)
        phi = ctx.emc_tally(emc.TALLY_PHI).copy()
        for bad in (float("nan"), float("inf")):
            with pytest.raises(emc.EmcError) as e:
                ctx.emc_set_bias(0, 0.0, bad, 0.0)
            assert e.value.status == 1
            with pytest.raises(emc.EmcError):
                ctx.emc_set_bias_all(np.array([[0.0, 1.0, bad]]))
            rho = np.zeros(ctx.n_cell)
            rho[7] = bad
            with pytest.raises(emc.EmcError):
                ctx.poisson_solve(rho, (0.0, 1.0, 0.0))
            with pytest.raises(emc.EmcError):
                ctx.emc_poisson_solve_static(None, (0.0, bad, 0.0))
        assert np.array_equal(ctx.emc_tally(emc.TALLY_PHI), phi)
        ctx.emc_step(10)


def test_non_finite_energy_is_caught_on_the_device(emc):
    """A NaN wave vector planted in one particle (through the state blob) is
    caught by the flight kernel's energy check; the next tally returns
    EMC_EOVERFLOW with the error word, no fault.  Restoring the clean state
    clears the error and the run goes on."""
    cfg = W.nanowire(n_particles=4000, nx=10, Lx=100e-9, Vd=2.0, seed=9)
    with emc.Context(cfg) as ctx:
        ctx.emc_step(10)
        clean = ctx.emc_get_state()
        bad = clean.copy()
        kx = bad[72:72 + 4 * ctx.capacity].view(np.float32)  # FP32 build: k_x of every slot
        kx[0] = np.nan
        ctx.emc_set_state(bad)
        ctx.emc_step(20)
        with pytest.raises(emc.EmcError) as e:
            ctx.emc_tally(emc.TALLY_OBS)
        assert e.value.status == 4 and "non-finite" in str(e.value)
        ctx.emc_set_state(clean)
        ctx.emc_step(20)
        ob = ctx.emc_tally(emc.TALLY_OBS)[0]
        assert ob["steps_done"] == 30 and ob["n_alive"] > 0
