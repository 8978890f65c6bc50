"""FP64 reference of the thermal side (test infrastructure only).

kappa(T): kinetic theory over three identical sine-shaped acoustic branches
omega = omega_max sin(pi q / 2 q0), with 1/tau = A omega^4 + B1 omega^2 T
exp(-B2/T) (the phonon paragraph and Table II) and, optionally, a boundary
term v_g / L_b (the size-modified mean free paths of the paragraph after
Eq. (3)):  kappa = 3 * (1/3) int_0^q0 C(q) v_g(q)^2 tau(q) q^2 / (2 pi^2) dq,
C(q) = hbar omega dn/dT.

Phonon-electron scattering in doped wires (Eq. (1)): an extra rate
tau_E^-1(omega) from the deformation-potential coupling of acoustic phonons
to the free electrons, with the Fermi level of n_e electrons in a parabolic
band of DOS mass m* at the lattice temperature (full ionization).

Fourier problem on the subcell grid: sum over faces g_f (T_c - T_n) +
boundary terms g_b (T_c - T_sink) = q_c, g_f = harmonic-mean kappa / h^2;
contact faces (x = 0, x = L) at T_sink half a cell away; the bottom face
(z = 0) through a conductance h_bottom in series with the half cell; other
faces adiabatic.  kappa(T) by Picard iteration.
"""
import numpy as np
from scipy import constants as sc
from scipy import integrate, optimize, sparse
from scipy.sparse import linalg as spla

HB, KB = sc.hbar, sc.k


def fermi_half(eta):
    """Normalised Fermi-Dirac integral of order 1/2:
    (2/sqrt(pi)) int_0^inf sqrt(x) / (1 + exp(x - eta)) dx."""
    f = lambda x: np.sqrt(x) * np.exp(-np.logaddexp(0.0, x - eta))
    top = max(eta, 0.0) + 80.0
    return 2.0 / np.sqrt(np.pi) * integrate.quad(f, 0.0, top, epsabs=0, epsrel=1e-13, limit=400)[0]


def band_density(T, m_rel):
    """Effective density of states 2 (m* k T / 2 pi hbar^2)^(3/2), m^-3."""
    return 2.0 * (m_rel * sc.m_e * KB * T / (2.0 * np.pi * HB ** 2)) ** 1.5


def fermi_level(n, T, m_rel):
    """E_F (J, from the band edge) with n = N_c F_1/2(E_F / kT)."""
    Nc = band_density(T, m_rel)
    eta = optimize.brentq(lambda e: np.log(fermi_half(e)) - np.log(n / Nc), -200.0, 400.0, xtol=1e-13, rtol=1e-14)
    return eta * KB * T


def tau_e_inv(w, T, n, elec, E_F=None):
    """Phonon-electron scattering rate of Eq. (1) (1/s) for phonons of
    angular frequency w; elec: m_rel (DOS mass), Da_eV, rho_kg_m3, vg_m_s
    (the averaged phonon group velocity)."""
    m = elec["m_rel"] * sc.m_e
    Da = elec["Da_eV"] * sc.e
    v = elec["vg_m_s"]
    kT = KB * T
    if E_F is None:
        E_F = fermi_level(n, T, elec["m_rel"])
    half = 0.5 * m * v * v
    pre = Da ** 2 * m ** 3 * v / (4.0 * np.pi * HB ** 4 * elec["rho_kg_m3"]) * kT / half
    a = (half - E_F) / kT + (HB * w) ** 2 / (8.0 * m * v * v * kT)
    y = HB * w / (2.0 * kT)
    # braces of Eq. (1): hbar w / kT - ln[(1 + e^(a+y)) / (1 + e^(a-y))], with
    # hbar w / kT = 2y.  Written with ln(1 + e^z) = max(z, 0) + ln(1 + e^-|z|)
    # the 2y cancels exactly against the max parts, which keeps the small
    # non-degenerate values (a >> 1) free of cancellation.
    sp = lambda z: np.log1p(np.exp(-abs(z)))
    if a - y >= 0.0:
        br = sp(a - y) - sp(a + y)
    elif a + y <= 0.0:
        br = 2.0 * y - sp(a + y) + sp(a - y)
    else:
        br = (y - a) - sp(a + y) + sp(a - y)
    return pre * br


def kappa(T, mat, L_b=0.0, n_e=0.0, elec=None):
    q0, wm = mat["k0_per_m"], mat["omega_max_rad_s"]
    A, B1, B2 = mat["A_s3"], mat["B1_s_per_K"], mat["B2_K"]
    E_F = fermi_level(n_e, T, elec["m_rel"]) if n_e > 0 else None

    def f(q):
        w = wm * np.sin(np.pi * q / (2 * q0))
        vg = wm * np.pi / (2 * q0) * np.cos(np.pi * q / (2 * q0))
        x = HB * w / (KB * T)
        dndT = x * np.exp(x) / np.expm1(x) ** 2 / T
        rate = A * w ** 4 + B1 * w ** 2 * T * np.exp(-B2 / T)
        if L_b > 0:
            rate = rate + vg / L_b
        if E_F is not None:
            rate = rate + tau_e_inv(w, T, n_e, elec, E_F)
        return HB * w * dndT * vg * vg / rate * q * q / (2 * np.pi ** 2)

    return integrate.quad(f, 0.0, q0, epsabs=0, epsrel=1e-10, limit=400)[0]


def operator(cfg, kap, T_sink, h_bottom, g_if=None):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    hx, hy, hz = cfg["Lx"] / nx, cfg["Ly"] / ny, cfg["Lz"] / nz
    n = nx * ny * nz
    idx = lambda i, j, l: (i * ny + j) * nz + l
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    rhs_b = np.zeros(n)
    for i in range(nx):
        for j in range(ny):
            for l in range(nz):
                c = idx(i, j, l)
                kc = kap[c]
                for (di, dj, dl, h) in ((1, 0, 0, hx), (-1, 0, 0, hx), (0, 1, 0, hy), (0, -1, 0, hy),
                                        (0, 0, 1, hz), (0, 0, -1, hz)):
                    ii, jj, ll = i + di, j + dj, l + dl
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= ll < nz:
                        nb = idx(ii, jj, ll)
                        g = 2 * kc * kap[nb] / (kc + kap[nb]) / h ** 2
                        diag[c] += g
                        rows.append(c); cols.append(nb); vals.append(-g)
                    elif di != 0:  # contact faces: Dirichlet at T_sink
                        g = 2 * kc / h ** 2
                        diag[c] += g
                        rhs_b[c] += g * T_sink
                    elif dl == -1:  # bottom face: conductance to the sink
                        r = h / (2 * kc) + (1.0 / h_bottom if h_bottom > 0 else 0.0)
                        if g_if is not None:  # the interface of Eq. (3) in series
                            r += 1.0 / g_if[c]
                        g = 1.0 / (h * r)
                        diag[c] += g
                        rhs_b[c] += g * T_sink
    A = sparse.csr_matrix((vals + list(diag), (rows + list(range(n)), cols + list(range(n)))), shape=(n, n))
    return A, rhs_b


def solve(cfg, q, mat, T_sink=300.0, h_bottom=1e9, L_b=0.0, tol=1e-8, max_picard=50, T0=None, n_e=0.0, elec=None,
          substrate=None, area_ratio=1.0):
    """Steady temperatures (K) per subcell for heat q (W/m^3).  substrate:
    the Table II column of the material under the bottom face; then the
    interface conductance of Eq. (3) at the adjacent subcell's temperature,
    times area_ratio, is in series with the half cell and h_bottom (h_bottom
    <= 0: no lumped part)."""
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    T = np.full(n, T_sink) if T0 is None else np.array(T0, dtype=float)
    cache, gcache = {}, {}
    def kap_of(t):
        key = round(float(t), 9)
        if key not in cache:
            cache[key] = kappa(t, mat, L_b, n_e, elec)
        return cache[key]
    def gif_of(t):
        key = round(float(t), 9)
        if key not in gcache:
            gcache[key] = area_ratio * interface_conductance(t, mat, substrate)
        return gcache[key]
    for _ in range(max_picard):
        kap = np.array([kap_of(t) for t in T])
        g_if = np.array([gif_of(t) for t in T]) if substrate is not None else None
        A, b = operator(cfg, kap, T_sink, h_bottom, g_if)
        Tn = spla.spsolve(A.tocsc(), q + b)
        done = np.abs(Tn - T).max() < tol
        T = Tn
        if done:
            break
    return T


# ------------------------------------------------------------------ DMM
# Diffuse mismatch model of the interface between material 1 (the wire) and
# material 2 (the substrate), Eqs. (2) and (3), for the paper's phonon model:
# three identical acoustic branches per material with omega = omega_max
# sin(pi q / 2 q0).

def branch(mat, w):
    """Wave vector q(w), group velocity v_g(w) and density of states D(w)
    (per branch and unit volume, q^2 / (2 pi^2 v_g)) of one sine-shaped
    branch; zero states above omega_max."""
    q0, wm = mat["k0_per_m"], mat["omega_max_rad_s"]
    if not (0.0 < w < wm):
        return 0.0, 0.0, 0.0
    q = 2.0 * q0 / np.pi * np.arcsin(w / wm)
    vg = wm * np.pi / (2.0 * q0) * np.cos(np.pi * q / (2.0 * q0))
    return q, vg, q * q / (2.0 * np.pi ** 2 * vg)


def tau12(w, mat1, mat2):
    """Eq. (2): transmissivity from 1 to 2, the sums over the three branches
    of v_g D of each side."""
    _, v1, D1 = branch(mat1, w)
    _, v2, D2 = branch(mat2, w)
    s1, s2 = 3.0 * v1 * D1, 3.0 * v2 * D2
    return s2 / (s1 + s2) if s1 + s2 > 0.0 else 0.0


def interface_conductance(T, mat1, mat2):
    """Eq. (3): 1/R_K = sum over the branches of material 1 of
    int_0^omega_max1 v_g c(w) tau12(w) dw / 4, with c(w) = hbar w D(w) dn/dT
    the spectral heat capacity per unit volume.  W/(m^2 K)."""
    wm = mat1["omega_max_rad_s"]

    def f(w):
        _, v1, D1 = branch(mat1, w)
        x = HB * w / (KB * T)
        if x > 700.0:
            return 0.0
        dndT = x * np.exp(x) / np.expm1(x) ** 2 / T
        return 3.0 * v1 * HB * w * D1 * dndT * tau12(w, mat1, mat2) / 4.0

    pts = sorted({min(mat2["omega_max_rad_s"], wm) * (1 - 1e-12), wm * 0.5})
    return integrate.quad(f, 0.0, wm, epsabs=0, epsrel=1e-11, limit=800, points=pts)[0]
