"""kappa(T) as the library tabulates it (emc_kappa runs on the host: no GPU)
against the reference quadrature, with the boundary term and with the
phonon-electron scattering of Eq. (1) at several electron densities."""
import numpy as np
import pytest

import workloads as W
from oracle import thermal


@pytest.mark.parametrize("n_e", [0.0, 1e22, 1e24, 7e24, 1e26])
def test_library_kappa_matches_reference(emc, n_e):
    el = W.ELECTRON_PHONON_GAN if n_e > 0 else None
    tc = emc.emc.thermal_config(W.TABLE_II_GAN, L_boundary=120e-9, n_e=n_e, elec=el)
    Ts = np.array([150.0, 300.0, 415.0, 600.0, 1500.0])
    got = emc.emc.kappa(tc, Ts)
    want = [thermal.kappa(T, W.TABLE_II_GAN, 120e-9, n_e, el) for T in Ts]
    np.testing.assert_allclose(got, want, rtol=1e-8)


def test_library_rejects_partial_electron_parameters(emc):
    tc = emc.emc.thermal_config(W.TABLE_II_GAN, n_e=1e24, elec=W.ELECTRON_PHONON_GAN)
    tc.rho_kg_m3 = 0.0
    with pytest.raises(emc.EmcError):
        emc.emc.kappa(tc, [300.0])


def test_library_interface_model_matches_reference(emc):
    """Eqs. (2)-(3) as the library tabulates them (host code) against the
    reference quadrature: GaN wire on SiC and SiC on GaN."""
    for m1, m2 in ((W.TABLE_II_GAN, W.TABLE_II_SIC), (W.TABLE_II_SIC, W.TABLE_II_GAN)):
        tc = emc.emc.thermal_config(m1, substrate=m2)
        w = np.linspace(1e10, 0.9999 * m1["omega_max_rad_s"], 41)
        np.testing.assert_allclose(emc.emc.dmm_transmissivity(tc, w), [thermal.tau12(x, m1, m2) for x in w],
                                   rtol=1e-13, atol=1e-15)
        Ts = np.array([150.0, 300.0, 415.0, 800.0, 1500.0])
        np.testing.assert_allclose(emc.emc.interface_conductance(tc, Ts),
                                   [thermal.interface_conductance(T, m1, m2) for T in Ts], rtol=1e-7)
    tc = emc.emc.thermal_config(W.TABLE_II_GAN, substrate=W.TABLE_II_SIC)
    tc.sub_k0_per_m = 0.0
    with pytest.raises(emc.EmcError):
        emc.emc.interface_conductance(tc, [300.0])
