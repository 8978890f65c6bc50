"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  The FP64 parity build must reproduce the oracle's integer
tallies bit for bit over short horizons (same Philox streams, same decisions);
floating sums agree to rounding.  The FP32 production build is compared
statistically."""
import numpy as np
import pytest

import workloads as W
from tests.emc_harness import gpu_tallies, oracle_heat

pytestmark = pytest.mark.gpu


def read_kat():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(x, 16) for x in line.split()]
                rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_device_philox_known_answers(emc):
    rows = read_kat()
    with emc.Context(W.bulk(n_particles=1)) as ctx:
        out = ctx.debug_philox([r[0] for r in rows], [r[1] for r in rows])
    for o, r in zip(out, rows):
        assert list(o) == r[2]


def test_device_philox_matches_oracle_stream(emc, oracle_mod):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(512, 2), dtype=np.uint64).astype(np.uint32)
    with emc.Context(W.bulk(n_particles=1)) as ctx:
        out = ctx.debug_philox(ctr, key)
    for i in range(0, 512, 37):
        assert tuple(int(x) for x in out[i]) == oracle_mod.philox(tuple(int(x) for x in ctr[i]),
                                                                  tuple(int(x) for x in key[i]))


@pytest.mark.parametrize("cfg", [W.bulk(n_particles=1), W.bulk(n_particles=1, T=520.0, Nd_cm3=3e18),
                                 W.nanowire(n_particles=10, nx=4, Lx=40e-9)])
def test_rate_tables_match_oracle(emc, oracle_mod, cfg):
    ref = oracle_mod.Sim(cfg)
    t_ref, g_ref = ref.tables()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        t, g = ctx.debug_tables(0)
    np.testing.assert_allclose(g, g_ref, rtol=1e-12)
    np.testing.assert_allclose(t, t_ref, rtol=1e-11, atol=1e-15)


def test_initial_state_matches_oracle(emc, oracle_mod):
    cfg = W.nanowire(n_particles=3000, nx=10, Lx=100e-9, seed=4)
    ref = oracle_mod.Sim(cfg).particles()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        p = ctx.debug_particles()
    al = ref["alive"].astype(bool)
    assert np.array_equal(p["valley"] >= 0, al)
    np.testing.assert_allclose(p["k"][al], ref["k"][al], rtol=1e-11, atol=1e-3)
    np.testing.assert_allclose(p["r"][al], ref["r"][al], rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(p["tr"][al], ref["tr"][al], rtol=1e-11)
    assert np.array_equal(p["ctr"][al], ref["ctr"][al])


@pytest.mark.parametrize("n,steps,spl", [(10_000, 200, 50), (1537, 60, 7)])
def test_bulk_fp64_bit_exact(emc, oracle_mod, n, steps, spl):
    cfg = W.bulk(n_particles=n, seed=0, steps_per_launch=spl)
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        g = gpu_tallies(emc, ctx)
    ob = g["obs"]
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(ob["self_events"], rt["self_events"].astype(np.int64))
    assert np.array_equal(ob["valley_steps"], rt["valley_steps"])
    assert ob["n_samples"] == rt["n_samples"] and ob["overflow"] == rt["overflow"]
    np.testing.assert_allclose(ob["sum_v"], rt["sum_v"], rtol=1e-9, atol=1e-9 * np.abs(rt["sum_v"]).max())
    assert ob["sum_E"] == pytest.approx(rt["sum_E"], rel=1e-10)
    assert ob["sum_Etot"] == pytest.approx(rt["sum_Etot"], rel=1e-10)


def test_nanowire_fp64_bit_exact(emc, oracle_mod):
    cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=2.0, seed=7)
    steps = 40
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    phi_ref, E_ref = ref.phi()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        g = gpu_tallies(emc, ctx)
        phi = ctx.emc_tally(emc.TALLY_PHI)[0]
        Ef = ctx.emc_tally(emc.TALLY_FIELD)[0]
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(g["heat"], oracle_heat(rt["events"]))
    assert np.array_equal(g["crossings"], rt["crossings"])
    assert np.array_equal(g["charge"], rt["charge"])
    assert g["obs"]["n_alive"] == rt["n_alive"]
    assert np.array_equal(g["obs"]["self_events"], rt["self_events"].astype(np.int64))
    np.testing.assert_allclose(phi, phi_ref, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(Ef, E_ref, rtol=1e-7, atol=1e-3 * np.abs(E_ref).max())


def test_poisson_solve_matches_oracle(emc, oracle_mod):
    cfg = W.nanowire(n_particles=10)
    rng = np.random.default_rng(3)
    from scipy import constants as sc
    rho = sc.e * 1e24 * rng.uniform(-1, 1, 1800)
    want = oracle_mod.poisson(cfg, rho, tol=1e-15, maxit=50000) if False else None
    c2 = dict(cfg); c2.update(Vs=0.0, Vd=7.0, Vg=-1.0)
    want = oracle_mod.poisson(c2, rho, tol=1e-14)
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        got = ctx.poisson_solve(rho, (0.0, 7.0, -1.0))
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_bulk_fp32_statistics(emc, oracle_mod):
    """Production build vs oracle at the 10,000-electron, 100 kV/cm bulk
    workload: drift velocity, mean energy, valley fractions within 1% or 3
    sigma of batch means (the two runs are independent samples)."""
    cfg = W.bulk(n_particles=10_000, seed=0)
    blocks, per = 8, 200
    ref = oracle_mod.Sim(cfg)
    ref.run(400)
    with emc.Context(cfg) as ctx:
        ctx.emc_step(400)
        ctx.emc_tally(emc.TALLY_OBS, reset=True)
        gv, ge, ov, oe = [], [], [], []
        r0 = ref.tallies()
        for b in range(blocks):
            ctx.emc_step(per)
            ob = ctx.emc_tally(emc.TALLY_OBS, reset=True)[0]
            gv.append(-ob["sum_v"][2] / ob["n_samples"])
            ge.append(ob["sum_E"] / ob["n_samples"])
            ref.run(per)
            r1 = ref.tallies()
            ns = r1["n_samples"] - r0["n_samples"]
            ov.append(-(r1["sum_v"][2] - r0["sum_v"][2]) / ns)
            oe.append((r1["sum_E"] - r0["sum_E"]) / ns)
            r0 = r1
    for g, o in ((gv, ov), (ge, oe)):
        g, o = np.array(g), np.array(o)
        sig = np.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
        assert abs(g.mean() - o.mean()) <= max(0.01 * abs(o.mean()), 3 * sig), (g.mean(), o.mean(), sig)


@pytest.mark.parametrize("geom", ["bulk", "nanowire"])
def test_sorted_fp64_bit_exact(emc, oracle_mod, geom):
    """Sorting the particle slots every launch changes nothing: the FP64 build
    still reproduces the oracle's integer tallies exactly."""
    if geom == "bulk":
        cfg = W.bulk(n_particles=5000, seed=5, steps_per_launch=10, sort_period=1)
        steps = 60
    else:
        cfg = W.nanowire(n_particles=5000, nx=20, Lx=200e-9, Vd=3.0, seed=6, sort_period=1)
        steps = 40
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        g = gpu_tallies(emc, ctx)
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(g["obs"]["self_events"], rt["self_events"].astype(np.int64))
    assert np.array_equal(g["obs"]["valley_steps"], rt["valley_steps"])
    if geom == "nanowire":
        assert np.array_equal(g["heat"], oracle_heat(rt["events"]))
        assert np.array_equal(g["crossings"], rt["crossings"])
        assert np.array_equal(g["charge"], rt["charge"])


def test_sorted_fp32_same_integer_tallies(emc):
    """FP32 production build: each particle's arithmetic does not depend on
    its slot, so sorted and unsorted runs give identical integer tallies."""
    base = W.nanowire(n_particles=20_000, nx=30, Lx=300e-9, Vd=4.0, seed=8)
    out = []
    for sp in (0, 2):
        with emc.Context(W.copy_config(base, sort_period=sp)) as ctx:
            ctx.emc_step(50)
            out.append(gpu_tallies(emc, ctx))
    a, b = out
    for k in ("events", "heat", "crossings", "charge"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["obs"]["self_events"], b["obs"]["self_events"])
    assert a["obs"]["n_alive"] == b["obs"]["n_alive"]


def test_batched_equals_separate(emc):
    """Several ensembles in one context give the same integer tallies as each
    ensemble in a context of its own."""
    cfgs = [W.nanowire(n_particles=3000 + 500 * i, nx=10, Lx=100e-9, Vd=float(i), seed=20 + i) for i in range(3)]
    with emc.Context(cfgs) as ctx:
        ctx.emc_step(30)
        ev = ctx.emc_tally(emc.TALLY_EVENTS)
        heat = ctx.emc_tally(emc.TALLY_HEAT)
        cr = ctx.emc_tally(emc.TALLY_CROSSINGS)
    for i, c in enumerate(cfgs):
        with emc.Context(c) as one:
            one.emc_step(30)
            assert np.array_equal(one.emc_tally(emc.TALLY_EVENTS)[0], ev[i])
            assert np.array_equal(one.emc_tally(emc.TALLY_HEAT)[0], heat[i])
            assert np.array_equal(one.emc_tally(emc.TALLY_CROSSINGS)[0], cr[i])


def test_edge_cases(emc):
    # empty ensemble
    with emc.Context(W.bulk(n_particles=0)) as ctx:
        ctx.emc_step(5)
        ob = ctx.emc_tally(emc.TALLY_OBS)[0]
        assert ob["n_samples"] == 0 and ob["n_alive"] == 0
        assert ctx.emc_tally(emc.TALLY_EVENTS).sum() == 0
    # zero steps is a no-op, negative is rejected
    with emc.Context(W.bulk(n_particles=33)) as ctx:
        ctx.emc_step(0)
        with pytest.raises(emc.EmcError):
            ctx.emc_step(-1)
        assert ctx.emc_tally(emc.TALLY_OBS)[0]["n_alive"] == 33
    # invalid configurations
    with pytest.raises(emc.EmcError):
        emc.Context(W.bulk(n_particles=10, T=-1.0))
    with pytest.raises(emc.EmcError):
        emc.Context(W.bulk(n_particles=10, capacity=5))
    with pytest.raises(emc.EmcError):
        emc.Context([W.bulk(n_particles=10), W.nanowire(n_particles=10)])


def test_graph_replay_same_as_direct(emc):
    """On a non-default stream the per-chunk refill + Poisson tail is captured
    once into a CUDA graph and replayed; the results must equal the direct
    launches on the default stream."""
    torch = pytest.importorskip("torch")
    cfgs = [W.nanowire(n_particles=8000, nx=20, Lx=200e-9, Vd=float(v), seed=40 + v) for v in (1, 3)]
    out = []
    for use_stream in (False, True):
        st = torch.cuda.Stream() if use_stream else None
        with emc.Context(cfgs, stream=st.cuda_stream if st else None) as ctx:
            ctx.emc_step(55)
            out.append((ctx.emc_tally(emc.TALLY_EVENTS), ctx.emc_tally(emc.TALLY_HEAT),
                        ctx.emc_tally(emc.TALLY_CHARGE), ctx.emc_tally(emc.TALLY_PHI)))
            launches = ctx.launch_count()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert launches > 0


def test_heterogeneous_batch_fp64_bit_exact(emc, oracle_mod):
    """40 bulk ensembles with different temperature, doping, field and size
    in one context (40 table sets, ensembles beyond the shared-memory tally
    slots): each reproduces its own oracle run exactly."""
    rng = np.random.default_rng(4)
    cfgs = []
    for e in range(40):
        cfgs.append(W.bulk(n_particles=int(10 ** rng.uniform(2, 3.2)), field_V_m=rng.uniform(0, 4e7),
                           T=rng.uniform(300, 600), Nd_cm3=10 ** rng.uniform(16, 19), seed=100 + e,
                           steps_per_launch=9))
    steps = 30
    with emc.Context(cfgs, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        ev = ctx.emc_tally(emc.TALLY_EVENTS)
        obs = ctx.emc_tally(emc.TALLY_OBS)
    for e in (0, 7, 31, 32, 33, 39):
        ref = oracle_mod.Sim(cfgs[e])
        ref.run(steps)
        rt = ref.tallies()
        assert np.array_equal(ev[e], rt["events"].sum(axis=0)), e
        assert np.array_equal(obs[e]["self_events"], rt["self_events"].astype(np.int64)), e
        assert np.array_equal(obs[e]["valley_steps"], rt["valley_steps"]), e
        assert obs[e]["sum_E"] == pytest.approx(rt["sum_E"], rel=1e-10)


def test_subcell_temperature_fp64_bit_exact(emc, oracle_mod):
    """Per-subcell lattice temperature (binned): the parity build reproduces
    the oracle exactly, including the flight rescale at the change of Gamma0
    and thermal refills at hot contacts."""
    cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=2.0, seed=17)
    C = cfg["nx"] * cfg["ny"] * cfg["nz"]
    x = np.repeat(np.arange(cfg["nx"]), cfg["ny"] * cfg["nz"])
    T1 = 300.0 + 250.0 * np.exp(-((x - 14) / 4.0) ** 2)
    T2 = 310.0 + 150.0 * x / cfg["nx"]
    ref = oracle_mod.Sim(cfg)
    ref.run(10)
    ref.set_temperature(T1)
    ref.run(20)
    ref.set_temperature(T2)
    ref.run(20)
    rt = ref.tallies()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(10)
        ctx.emc_set_temperature(0, T1)
        ctx.emc_step(20)
        ctx.emc_set_temperature(0, T2)
        ctx.emc_step(20)
        g = gpu_tallies(emc, ctx)
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(g["heat"], oracle_heat(rt["events"]))
    assert np.array_equal(g["crossings"], rt["crossings"])
    assert np.array_equal(g["charge"], rt["charge"])
    assert C == g["charge"].size


def test_live_contexts_with_different_shared_memory(emc):
    """A context whose flight launch needs more shared memory (one table set,
    staged table) keeps working after a second context that needs less (two
    table sets, nothing staged) was created on the same device."""
    big = emc.Context(W.bulk(n_particles=2000, seed=1))
    try:
        small = emc.Context([W.bulk(n_particles=1000, T=300.0 + 50.0 * i, seed=2 + i) for i in range(2)])
        try:
            small.emc_step(5)
            big.emc_step(5)
            assert big.emc_tally(emc.TALLY_OBS)[0]["n_samples"] == 2000 * 5
        finally:
            small.close()
    finally:
        big.close()


def test_set_bias_resolves_only_on_change(emc):
    """Unchanged terminal voltages leave the field as it is (no solve is
    launched); a changed drain voltage re-solves it."""
    cfgs = [W.nanowire(n_particles=2000, nx=10, Lx=100e-9, Vd=float(v), seed=60 + v) for v in (1, 3)]
    bias = np.array([[c["Vs"], c["Vd"], c["Vg"]] for c in cfgs])
    with emc.Context(cfgs) as ctx:
        ctx.emc_step(10)
        phi0 = ctx.emc_tally(emc.TALLY_PHI).copy()
        n0 = ctx.launch_count()
        ctx.emc_set_bias_all(bias.ctypes.data)
        assert ctx.launch_count() == n0
        assert np.array_equal(ctx.emc_tally(emc.TALLY_PHI), phi0)
        bias[1, 1] = 5.0
        ctx.emc_set_bias_all(bias.ctypes.data)
        assert ctx.launch_count() > n0
        phi1 = ctx.emc_tally(emc.TALLY_PHI)
        assert phi1[1, -1] > phi0[1, -1] + 1.0


def test_small_bulk_workload_in_full(emc, oracle_mod):
    """The small bulk workload as specified (10,000 electrons, 100 kV/cm,
    1e17 cm^-3, 300 K, Philox seed 0, 2 ps = 2000 steps), parity build
    against the oracle.  Every particle takes the same discrete path: the
    same number of random draws (Philox counter) and the same final valley,
    and every event count is equal.  The continuous state does not stay
    bit-equal over 2e7 particle-steps: scattering angles are drawn relative to
    the incoming direction, so the two sides' different floating-point
    operation orders (1e-14 relative after 200 steps) grow chaotically
    (median 1.6e-9, largest ~7% after 2000 steps); drift velocity, mean
    energy and valley occupancy agree to 1e-6."""
    cfg = W.config_bulk_small()
    steps = W.BULK_SMALL_STEPS
    n = cfg["n_particles"]
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    o = ref.particles()
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        g = gpu_tallies(emc, ctx)
        p = ctx.debug_particles()
    assert np.array_equal(p["ctr"][:n], o["ctr"][:n])
    assert np.array_equal(p["valley"][:n], o["valley"][:n])
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    ob = g["obs"]
    assert np.array_equal(ob["self_events"], rt["self_events"].astype(np.int64))
    assert np.array_equal(ob["valley_steps"], rt["valley_steps"])
    assert ob["n_samples"] == rt["n_samples"] == n * steps
    assert ob["sum_v"][2] == pytest.approx(rt["sum_v"][2], rel=1e-6)
    np.testing.assert_allclose(ob["sum_v"][:2], rt["sum_v"][:2], atol=1e-6 * abs(rt["sum_v"][2]))
    assert ob["sum_E"] == pytest.approx(rt["sum_E"], rel=1e-6)


def test_obs_buffer_matches_dicts(emc):
    """The in-place observation read (structured array) carries the same
    values as the list-of-dicts read."""
    cfgs = [W.bulk(n_particles=500 + 100 * e, seed=70 + e) for e in range(3)]
    with emc.Context(cfgs) as ctx:
        ctx.emc_step(20)
        dicts = ctx.emc_tally(emc.TALLY_OBS)
        buf = ctx.emc_tally(emc.TALLY_OBS, out=ctx.obs_buffer())
    for e, d in enumerate(dicts):
        for k, v in d.items():
            assert np.array_equal(np.asarray(buf[k][e]), np.asarray(v)), (e, k)


def test_production_runs_are_reproducible(emc):
    """Two identical production (FP32) runs of nanowires large enough that
    hundreds of electrons are refilled per period give identical integer
    tallies and subcell charge: nothing in the step depends on thread
    timing."""
    cfgs = [W.nanowire(n_particles=50_000, Vd=float(v), seed=110 + v) for v in (5, 20)]
    out = []
    for _ in range(2):
        with emc.Context(cfgs) as ctx:
            ctx.emc_step(100)
            out.append((ctx.emc_tally(emc.TALLY_EVENTS), ctx.emc_tally(emc.TALLY_CROSSINGS),
                        ctx.emc_tally(emc.TALLY_CHARGE), ctx.emc_tally(emc.TALLY_HEAT)))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert out[0][1][:, 2:].sum() > 100  # electrons were refilled
