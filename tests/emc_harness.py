"""Shared helpers of the test-suite: run the oracle and the CUDA library on
the same configuration and collect comparable tallies."""
import numpy as np

NV, NM = 3, 10


def oracle_heat(events: np.ndarray) -> np.ndarray:
    """Net phonon emissions per cell [C][2] from the oracle's per-cell event
    counts: polar optical emission (2) minus absorption (1); intervalley
    emissions (5, 7, 9) minus absorptions (4, 6, 8)."""
    ev = events.astype(np.int64)
    pop = ev[:, :, 2].sum(1) - ev[:, :, 1].sum(1)
    iv = ev[:, :, 5::2].sum((1, 2)) - ev[:, :, 4::2].sum((1, 2))
    return np.stack([pop, iv], axis=1)


def gpu_tallies(emc, ctx, e: int = 0) -> dict:
    ob = ctx.emc_tally(emc.TALLY_OBS)[e]
    return {
        "events": ctx.emc_tally(emc.TALLY_EVENTS)[e],
        "heat": ctx.emc_tally(emc.TALLY_HEAT)[e],
        "charge": ctx.emc_tally(emc.TALLY_CHARGE)[e],
        "crossings": ctx.emc_tally(emc.TALLY_CROSSINGS)[e],
        "obs": ob,
    }
