"""Host-side arithmetic of the electrothermal loop: the Fig. 5 thermal
resistance (peak rise / emitted power) against the closed form of uniform
heating in a wire cooled only at its two ends, using the reference Fourier
solve."""
import numpy as np
import pytest

import workloads as W
from oracle import thermal
from paper_1707_09073_gb300 import electrothermal as ET


def test_thermal_resistance_closed_form():
    # uniform q, adiabatic sides, no bottom loss, tiny rise (kappa constant):
    # with an even number of cells the hottest cell centres sit h/2 from the
    # middle and T_max - T_s = q L^2 / (8 kappa) exactly in the discrete
    # problem, so R_th = (q L^2 / 8 kappa) / (q L A) = L / (8 kappa A)
    c = W.nanowire(n_particles=1, nx=40, Lx=400e-9)
    n = c["nx"] * c["ny"] * c["nz"]
    q = np.full(n, 1e12)
    T = thermal.solve(c, q, W.TABLE_II_GAN, h_bottom=1e-30, L_b=0.0)
    k = thermal.kappa(300.0, W.TABLE_II_GAN)
    A = c["Ly"] * c["Lz"]
    P = np.array([q.sum() * c["Lx"] * A / n])
    R = ET.thermal_resistance(T[None, :], P, 300.0)
    assert R[0] == pytest.approx(c["Lx"] / (8.0 * k * A), rel=1e-4)


def test_thermal_resistance_without_power_is_nan():
    R = ET.thermal_resistance(np.full((2, 3), 300.0), np.array([0.0, 1.0]), 300.0)
    assert np.isnan(R[0]) and R[1] == 0.0
