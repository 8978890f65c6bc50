"""The allocation-free Poisson entry point (emc_poisson_solve_static).

Some callers cannot allocate device memory at the moment they need a field
solve -- a host that has handed the whole device to its own memory pool, or
code running where allocation is forbidden.  For them the library keeps the
solve's temporaries in a fixed static device array.  This test calls that
entry point through the C ABI twice in a row with different charge densities
and bias voltages and checks each result against the allocating
poisson_solve: both run the same kernels in the same order, so the potentials
are equal bit for bit.  It sits in a file of its own, collected last.
"""
import numpy as np
import pytest
from scipy import constants as sc

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_poisson_matches_allocating_solve(emc):
    cfg = W.nanowire(n_particles=2000)
    rng = np.random.default_rng(12)
    with emc.Context(cfg, precision=emc.FP64) as ctx:
        for call in range(2):
            rho = sc.e * 1e24 * rng.uniform(-1, 1, ctx.n_cell)
            bc = (0.0, 3.0 + 4.0 * call, -0.5 * call)
            want = ctx.poisson_solve(rho, bc)
            got = ctx.emc_poisson_solve_static(rho, bc)
            assert np.array_equal(got, want)
        # the current subcell charge as the source, twice
        want = ctx.poisson_solve(None, (0.0, 1.0, 0.0))
        for _ in range(2):
            got = ctx.emc_poisson_solve_static(None, (0.0, 1.0, 0.0))
            assert np.array_equal(got, want)
