"""Phonon Monte Carlo on the GPU (emc_phonon_solve) against the FP64 oracle
(oracle/phonon.py): the parity build follows the oracle's bundles exactly
(the same emissions, scatterings, segments and face counts per subcell, the
residence times to the fixed-point rounding), the production build agrees
in distribution, and disjoint bundle ranges add up."""
import numpy as np
import pytest

import workloads as W
from oracle import phonon as PH

pytestmark = pytest.mark.gpu

GAN, SIC = W.TABLE_II_GAN, W.TABLE_II_SIC


def _wire(nx=20, Lx=200e-9):
    return W.nanowire(n_particles=10, nx=nx, Lx=Lx, Vd=1.0, seed=3)


def _heat(cfg, seed=0):
    """The seeded synthetic heat map of workloads.py (shaped like the
    electrons', with a stretch of net absorption at the source end)."""
    return W.heat_map(cfg, seed=seed)


def _temps(cfg, seed=1):
    C = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return 300.0 + np.random.default_rng(seed).uniform(0.0, 40.0, C)


def _gpu(emc, cfg, tc, pc, q, n, T=None, first=0):
    with emc.Context(cfg) as ctx:
        return emc.emc.phonon_solve(ctx, tc, pc, q, n, T_cells=T, first=first)


def _assert_same_bundles(g, r):
    assert np.array_equal(g["emitted"], r["emitted"])
    assert np.array_equal(g["scatterings"], r["scatterings"])
    assert np.array_equal(g["absorbed"], r["absorbed"])
    assert g["segments"] == r["segments"] and g["capped"] == r["capped"]
    # residence times (the GPU rounds each segment to 2^-24 ps).  A bundle
    # that grazes a face splits its time between two subcells, or ends its
    # last flight, at a point that one-ulp differences of the arithmetic (a
    # fused multiply-add, a sine) move: the oracle built with and without
    # fused multiply-adds differs by up to 3.5e-6 of a subcell's time on the
    # all-rough case, with the integer tallies identical, so that is the
    # scale allowed here (the total moves far less).
    assert abs(g["t_res_ps"].sum() / r["t_res_ps"].sum() - 1) < 1e-7
    np.testing.assert_allclose(g["t_res_ps"], r["t_res_ps"], rtol=2e-5, atol=1e-6)
    np.testing.assert_allclose(g["dT"], r["dT"], rtol=2e-5, atol=1e-9 * np.abs(r["dT"]).max())


@pytest.mark.parametrize("case", ["wire", "eq1_boundary", "all_rough_p", "mixed_sign"])
def test_fp64_bundles_follow_the_oracle(emc, case):
    """FP64 parity build against the oracle, bundle for bundle, on a 20 x 3 x
    6 wire: contacts isothermal, plane A specular, rough outer side and top,
    the GaN/SiC interface of Eq. (2) at the bottom; subcell temperatures
    300-340 K (several rate tables); with Eq. (1) and a boundary term; with
    every non-absorbing face rough at p = 0.4; with negative heat (phonon
    absorption) near the source."""
    cfg = _wire()
    q, T = _heat(cfg), _temps(cfg)
    if case == "mixed_sign":
        q[: 4 * cfg["ny"] * cfg["nz"]] *= -0.5
    faces = list(emc.emc.WIRE_FACES)
    p = 0.3
    L_b, n_e, el = 0.0, 0.0, None
    if case == "eq1_boundary":
        L_b, n_e, el = 300e-9, 1e24, W.ELECTRON_PHONON_GAN
    if case == "all_rough_p":
        faces = [emc.emc.PH_ISOTHERMAL, emc.emc.PH_ROUGH, emc.emc.PH_ROUGH, emc.emc.PH_ROUGH,
                 emc.emc.PH_INTERFACE, emc.emc.PH_ROUGH]
        p = 0.4
    tc = emc.emc.thermal_config(GAN, L_boundary=L_b, n_e=n_e, elec=el, substrate=SIC)
    pc = emc.emc.phonon_config(faces, n_bins=400, precision=emc.FP64, p_specular=p, seed=9)
    N = 20_000
    g = _gpu(emc, cfg, tc, pc, q, N, T)
    r = PH.solve(cfg, q, GAN, faces, N, seed=9, nb=400, T_cells=T, p_specular=[p] * 6, L_b=L_b, n_e=n_e,
                 elec=el, substrate=SIC, threads=8)
    assert g["capped"] == 0 and int(g["absorbed"].sum()) == N
    _assert_same_bundles(g, r)


def test_fp64_capped_bundles_and_ragged_counts(emc):
    """A segment cap that stops most bundles, an odd bundle count and a
    bundle range that does not start at 0: still bundle for bundle."""
    cfg = _wire()
    q = _heat(cfg, 4)
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC)
    pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=300, precision=emc.FP64, p_specular=0.2, seed=4,
                               max_segments=40)
    g = _gpu(emc, cfg, tc, pc, q, 1237, first=100_003)
    r = PH.solve(cfg, q, GAN, emc.emc.WIRE_FACES, 1237, seed=4, nb=300, p_specular=[0.2] * 6, substrate=SIC,
                 max_segments=40, first=100_003)
    assert g["capped"] > 0
    _assert_same_bundles(g, r)
    assert int(g["absorbed"].sum()) + g["capped"] == 1237


def test_disjoint_bundle_ranges_add_up(emc):
    cfg = _wire()
    q = _heat(cfg, 5)
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC)
    pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=300, precision=emc.FP64, seed=2)
    a = _gpu(emc, cfg, tc, pc, q, 3000, first=0)
    b = _gpu(emc, cfg, tc, pc, q, 5000, first=3000)
    u = _gpu(emc, cfg, tc, pc, q, 8000, first=0)
    for k in ("emitted", "scatterings", "absorbed", "t_res_ps"):
        assert np.array_equal(a[k] + b[k], u[k]), k
    assert a["segments"] + b["segments"] == u["segments"]


def test_fp32_production_agrees_in_distribution(emc):
    """FP32 production build, 8 batches of 40,000 bundles (disjoint ids),
    against one FP64 oracle run of 40,000: temperature rise per x-slab and
    the share of bundles ending at each face within 3.5 sigma."""
    cfg = _wire()
    q, T = _heat(cfg, 6), _temps(cfg, 7)
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC)
    pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=500, precision=emc.FP32, p_specular=0.3, seed=21)
    N, B = 40_000, 8
    nyz = cfg["ny"] * cfg["nz"]
    slabs, faces = [], []
    with emc.Context(cfg) as ctx:
        for k in range(B):
            g = emc.emc.phonon_solve(ctx, tc, pc, q, N, T_cells=T, first=10_000_000 + k * N)
            assert g["capped"] == 0
            slabs.append(g["dT"].reshape(cfg["nx"], nyz).mean(axis=1))
            faces.append(g["absorbed"] / N)
    r = PH.solve(cfg, q, GAN, emc.emc.WIRE_FACES, N, seed=21, nb=500, T_cells=T, p_specular=[0.3] * 6,
                 substrate=SIC, threads=8)
    slabs, faces = np.array(slabs), np.array(faces)
    ref = r["dT"].reshape(cfg["nx"], nyz).mean(axis=1)
    sd = slabs.std(axis=0, ddof=1)
    z = (slabs.mean(axis=0) - ref) / (sd * np.sqrt(1.0 / B + 1.0))
    assert np.abs(z).max() < 3.5, z
    fr = r["absorbed"] / N
    sf = np.sqrt(np.maximum(fr * (1 - fr), 1e-12) / N)
    zf = (faces.mean(axis=0) - fr) / (sf * np.sqrt(1.0 / B + 1.0))
    assert np.abs(zf).max() < 3.5, zf
    assert np.abs(slabs.mean(axis=0) / ref - 1).max() < 0.05


def test_phonon_solve_rejects_bad_input(emc):
    cfg = _wire()
    q = _heat(cfg)
    tc = emc.emc.thermal_config(GAN, substrate=SIC)
    with emc.Context(cfg) as ctx:
        bad = [
            (emc.emc.phonon_config([emc.emc.PH_SPECULAR] * 6), q, 10),  # no absorbing face
            (emc.emc.phonon_config(n_bins=0), q, 10),
            (emc.emc.phonon_config(), np.zeros_like(q), 10),             # no heat
            (emc.emc.phonon_config(), q * np.nan, 10),
            (emc.emc.phonon_config(), q, 0),
            (emc.emc.phonon_config(p_specular=1.5), q, 10),
        ]
        for pc, qq, n in bad:
            with pytest.raises(emc.EmcError):
                emc.emc.phonon_solve(ctx, tc, pc, qq, n)
        with pytest.raises(emc.EmcError):  # interface face without a substrate
            emc.emc.phonon_solve(ctx, emc.emc.thermal_config(GAN), emc.emc.phonon_config(), q, 10)
    with emc.Context(W.bulk(n_particles=100)) as ctx:
        with pytest.raises(emc.EmcError):
            emc.emc.phonon_solve(ctx, tc, emc.emc.phonon_config(), np.ones(1), 10)


def test_electron_phonon_monte_carlo_loop_converges(emc):
    """The hybrid loop with the phonon side in the transistor region
    (electrothermal.hybrid_iterate): from 300 K it reaches a fixed point
    within the Monte Carlo noise and heats the wire; its last two iterates'
    peak rises agree within that noise."""
    from paper_1707_09073_gb300 import electrothermal as ET
    cfg = W.nanowire(n_particles=40_000, nx=20, Lx=200e-9, Vd=4.0, seed=33)
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC, n_e=cfg["Nd"], elec=W.ELECTRON_PHONON_GAN)
    pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=500, precision=emc.FP32, seed=5)
    with emc.Context(cfg) as ctx:
        ET.warm_to_steady(ctx)
        T0 = np.full((1, ctx.n_cell), 300.0)
        r = ET.hybrid_iterate(ctx, tc, pc, T0, 400_000, max_iter=10)
        assert r["converged"], (r["history"], r["max_dT_K"], r["noise_K"])
        assert r["peak"][0] > 1.0 and np.isfinite(r["R_th_K_per_W"][0])
        h = r["history"]
        assert abs(h[-1][0] - h[-2][0]) <= max(0.1, r["noise_K"][-1]) + 1e-9, (h, r["noise_K"])


def test_full_size_wire_sampled_bundles_and_bookkeeping(emc):
    """The benchmarked phonon problem at its full size (the 1 um wire, 3 x 6 x
    100 subcells, 1000 bins, 10^7 bundles, FP32): every bundle ends at a
    face, the bundles start in the subcells in proportion to |q| (multinomial,
    5 sigma); and a sample of the same bundle ids (20,000 from the middle of
    the range) in the parity build follows the oracle: the same emissions,
    and scatterings, face counts and residence times within what rounding
    alone produces on paths this long (227 segments per bundle through
    mirrors and faces): one-ulp differences grow along a path, and the oracle
    built with and without fused multiply-adds differs in the scattering
    counts of 364 of the 1800 subcells (by at most 5), in one face count by 1
    and in the segment count by 8e-5."""
    cfg = W.nanowire(n_particles=10, Vd=20.0, seed=1)
    C = cfg["nx"] * cfg["ny"] * cfg["nz"]
    q = W.heat_map(cfg, seed=3)
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC)
    N = 10_000_000
    with emc.Context(cfg) as ctx:
        g = emc.emc.phonon_solve(ctx, tc, emc.emc.phonon_config(n_bins=1000, seed=77), q, N)
        s = emc.emc.phonon_solve(ctx, tc, emc.emc.phonon_config(n_bins=1000, seed=77, precision=emc.FP64), q,
                                 20_000, first=5_000_000)
    assert g["capped"] == 0 and int(g["absorbed"].sum()) == N
    p = np.abs(q) / np.abs(q).sum()
    z = (g["emitted"] - N * p) / np.sqrt(N * p * (1 - p))
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    r = PH.solve(cfg, q, GAN, emc.emc.WIRE_FACES, 20_000, seed=77, nb=1000, substrate=SIC, first=5_000_000,
                 threads=8)
    assert np.array_equal(s["emitted"], r["emitted"])
    ds = s["scatterings"].astype(np.int64) - r["scatterings"].astype(np.int64)
    assert np.abs(ds).max() <= 10 and np.count_nonzero(ds) <= 0.4 * C, (np.count_nonzero(ds), np.abs(ds).max())
    assert abs(int(s["scatterings"].sum()) / int(r["scatterings"].sum()) - 1) < 2e-3
    assert np.abs(s["absorbed"].astype(np.int64) - r["absorbed"].astype(np.int64)).max() <= 20
    assert abs(s["segments"] / r["segments"] - 1) < 1e-3
    assert abs(s["t_res_ps"].sum() / r["t_res_ps"].sum() - 1) < 1e-3
    np.testing.assert_allclose(s["dT"].reshape(cfg["nx"], -1).mean(axis=1),
                               r["dT"].reshape(cfg["nx"], -1).mean(axis=1), rtol=1e-2,
                               atol=1e-2 * np.abs(r["dT"]).max())


def test_electron_to_phonon_chain_matches_oracle(emc, oracle_mod):
    """One step of the hybrid method through the library (FP64 electron Monte
    Carlo -> net phonon energy per subcell -> FP64 phonon Monte Carlo ->
    temperature rise) against the same chain through the oracle (its
    per-cell events -> net phonon energy -> oracle/phonon.solve): the heat
    maps are equal, the bundles the same, the temperature rise equal to the
    fixed-point rounding of the residence times."""
    from emc_harness import oracle_heat
    from paper_1707_09073_gb300 import electrothermal as ET
    cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=4.0, seed=7)
    steps = 60
    ref = oracle_mod.Sim(cfg)
    ref.run(steps)
    rt = ref.tallies()
    Vc = cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / (cfg["nx"] * cfg["ny"] * cfg["nz"])
    window = steps * cfg["dt"]
    tc = emc.emc.thermal_config(GAN, L_boundary=0.0, substrate=SIC)
    pc = emc.emc.phonon_config(emc.emc.WIRE_FACES, n_bins=400, precision=emc.FP64, p_specular=0.3, seed=13)
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        ctx.emc_step(steps)
        q_lib = ET.heat_map(ctx, window)[0]
        g = emc.emc.phonon_solve(ctx, tc, pc, q_lib, 20_000)
    w = cfg["Nd"] * cfg["Lx"] * cfg["Ly"] * cfg["Lz"] / cfg["n_particles"]
    h = oracle_heat(rt["events"])
    q_orc = (h[:, 0] * cfg["hw_lo_eV"] + h[:, 1] * cfg["hw_iv_eV"]) * 1.602176634e-19 * w / (window * Vc)
    np.testing.assert_allclose(q_lib, q_orc, rtol=1e-12, atol=1e-12 * np.abs(q_orc).max())
    r = PH.solve(cfg, q_orc, GAN, emc.emc.WIRE_FACES, 20_000, seed=13, nb=400, p_specular=[0.3] * 6,
                 substrate=SIC, threads=8)
    _assert_same_bundles(g, r)
    assert g["dT"].max() > 0
