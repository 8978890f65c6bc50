"""Edge and degenerate cases of the method, FP64 parity build against the
oracle bit for bit: more table sets than the kernel stages in shared memory
(physics read from global memory) and more ensembles than it keeps
shared-memory tallies for; energies beyond the rate table (overflow counted,
last bin used); all-specular and all-diffuse walls; mechanism subsets; zero
field."""
import numpy as np
import pytest

import workloads as W
from tests.emc_harness import gpu_tallies, oracle_heat

pytestmark = pytest.mark.gpu


def same_as_oracle(emc, oracle_mod, cfg, steps, ens=0, ctx=None):
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    if ctx is None:
        with emc.Context(cfg, precision=emc.FP64) as c:
            c.emc_step(steps)
            g = gpu_tallies(emc, c)
    else:
        g = gpu_tallies(emc, ctx, ens)
    ob = g["obs"]
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(ob["self_events"], rt["self_events"].astype(np.int64))
    assert np.array_equal(ob["valley_steps"], rt["valley_steps"])
    assert ob["overflow"] == rt["overflow"] and ob["n_samples"] == rt["n_samples"]
    assert ob["sum_E"] == pytest.approx(rt["sum_E"], rel=1e-10)
    if cfg["geometry"] == 1:
        assert np.array_equal(g["heat"], oracle_heat(rt["events"]))
        assert np.array_equal(g["crossings"], rt["crossings"])
        assert np.array_equal(g["charge"], rt["charge"])
        assert ob["n_alive"] == rt["n_alive"]
    return ob


def test_seventy_table_sets_and_ensembles(emc, oracle_mod):
    # 70 bulk ensembles, each its own temperature (70 table sets > 64 staged
    # physics sets; ensembles 32..69 tally straight to global memory)
    cfgs = [W.bulk(n_particles=60 + e, field_V_m=1e6 * (e % 9), T=300.0 + 3.0 * e, seed=900 + e, steps_per_launch=11)
            for e in range(70)]
    steps = 25
    with emc.Context(cfgs, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        for e in (0, 31, 32, 64, 69):
            same_as_oracle(emc, oracle_mod, cfgs[e], steps, ens=e, ctx=ctx)


def test_energies_beyond_the_table(emc, oracle_mod):
    # 100 bins of 2 meV: the hot electrons at 400 kV/cm leave the table
    cfg = W.bulk(n_particles=2000, field_V_m=4e7, n_bins=100, seed=3)
    ob = same_as_oracle(emc, oracle_mod, cfg, 150)
    assert ob["overflow"] > 0


@pytest.mark.parametrize("p", [0.0, 1.0])
def test_walls_all_diffuse_or_all_specular(emc, oracle_mod, p):
    cfg = W.nanowire(n_particles=3000, nx=10, Lx=100e-9, Vd=1.0, p_specular=p, seed=40)
    same_as_oracle(emc, oracle_mod, cfg, 40)


@pytest.mark.parametrize("mask", [0b0000000110, 0b0000001001, 0b1111110000])
def test_mechanism_subsets(emc, oracle_mod, mask):
    # POP only; impurity + acoustic only; intervalley only
    cfg = W.bulk(n_particles=1500, field_V_m=2e7, mech_mask=mask, seed=41, n_bins=2048)
    same_as_oracle(emc, oracle_mod, cfg, 60)


def test_no_mechanism_is_rejected(emc):
    # with every mechanism off a valley has no scattering rate at all (no
    # self-scattering rate Gamma0 to draw flights from): refused with a status
    with pytest.raises(emc.EmcError, match="zero total scattering rate"):
        emc.Context(W.bulk(n_particles=10, mech_mask=0), precision=emc.FP64)


def test_zero_field(emc, oracle_mod):
    same_as_oracle(emc, oracle_mod, W.bulk(n_particles=2000, field_V_m=0.0, seed=42), 100)
