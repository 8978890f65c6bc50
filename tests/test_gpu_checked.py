"""The checked build (array indices and positions verified in the kernels,
a violation set in the device error word and returned as an error status)
on small cases of every kernel family: the runs must raise no violation and
give the same results as the oracle (the particle-by-particle parity of the
electron and phonon Monte Carlos).  The checks stand in for a memory
checker, which is closed on this machine."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import numpy as np
import workloads as W
import paper_1707_09073_gb300 as emc
from oracle import oracle, phonon as PH
from tests.emc_harness import gpu_tallies, oracle_heat
oracle.build()
# nanowire with refill, sorting and subcell temperatures, FP64 against the oracle
cfg = W.nanowire(n_particles=6000, nx=20, Lx=200e-9, Vd=4.0, seed=7, sort_period=2)
ref = oracle.Sim(cfg)
ref.run(30)
T = 300.0 + 40.0 * np.linspace(0, 1, cfg["nx"] * cfg["ny"] * cfg["nz"])
ref.set_temperature(T)
ref.run(30)
rt = ref.tallies()
with emc.Context(cfg, precision=emc.FP64) as ctx:
    ctx.emc_step(30)
    ctx.emc_set_temperature(0, T)
    ctx.emc_step(30)
    g = gpu_tallies(emc, ctx)
    assert np.array_equal(g["events"], rt["events"].sum(axis=0))
    assert np.array_equal(g["crossings"], rt["crossings"])
    assert np.array_equal(g["charge"], rt["charge"])
# production build of the full wire with sorting
with emc.Context(W.nanowire(n_particles=50_000, Vd=10.0, seed=3, sort_period=3)) as ctx:
    ctx.emc_step(200)
    ctx.emc_tally(emc.TALLY_OBS)
# bulk batch
with emc.Context([W.bulk(n_particles=2000, seed=s) for s in range(3)]) as ctx:
    ctx.emc_step(120)
    ctx.emc_tally(emc.TALLY_OBS)
# phonon Monte Carlo, FP64 against the oracle and FP32
pw = W.nanowire(n_particles=10, nx=8, Lx=80e-9, Vd=1.0, seed=5)
q = np.linspace(1.0, 3.0, 8 * pw["ny"] * pw["nz"]) * 1e17
tc = emc.emc.thermal_config(W.TABLE_II_GAN, L_boundary=0.0, substrate=W.TABLE_II_SIC)
with emc.Context(pw) as ctx:
    g = emc.emc.phonon_solve(ctx, tc, emc.emc.phonon_config(n_bins=200, precision=emc.FP64, p_specular=0.3, seed=3), q, 3000)
    emc.emc.phonon_solve(ctx, tc, emc.emc.phonon_config(n_bins=200, p_specular=0.3, seed=3), q, 30000)
r = PH.solve(pw, q, W.TABLE_II_GAN, emc.emc.WIRE_FACES, 3000, seed=3, nb=200, p_specular=[0.3] * 6, substrate=W.TABLE_II_SIC)
assert np.array_equal(g["scatterings"], r["scatterings"]) and np.array_equal(g["absorbed"], r["absorbed"])
print("checked build ok")
'''


def test_checked_build_runs_clean():
    from paper_1707_09073_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, EMC_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked build ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
