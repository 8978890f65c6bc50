/*
 * FP64 CPU oracle for the ensemble electron Monte Carlo of wurtzite GaN,
 * Hao et al., arXiv:1707.09073.  TEST INFRASTRUCTURE ONLY (see emc_oracle.h).
 *
 * What the paper fixes: Kane bands E(1+aE) = hbar^2 k^2 / 2m with the energy
 * dependent mass m(1+2aE), three valleys Gamma1/U/Gamma3, four mechanisms
 * (ionized impurity, polar optical, acoustic deformation potential,
 * intervalley optical), all dopants ionized, Table I parameters, the
 * 3 x 6 x 100 subcell grid that counts electrons for the Poisson update and
 * the net electron-to-phonon energy exchange per subcell (the body text next
 * to Table I, and the text after it).  The paper defers the rate expressions
 * to its ref. [7]; the textbook isotropic nonparabolic forms written below
 * (Fermi golden rule with the Froehlich, screened-Coulomb, deformation
 * potential and intervalley matrix elements, overlap factors neglected) are
 * the reading this oracle implements.
 *
 * The steps follow the standard synchronous-ensemble EMC: per time step every
 * particle drifts until its residual flight time runs out, scatters against
 * the tabulated cumulative rates normalised by a constant total rate Gamma0
 * per valley (self-scattering fills the rest), draws a new flight time
 * -ln(u)/Gamma0, and so on until the step ends.
 */
#include "emc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact / recommended values */
#define Q_E   1.602176634e-19
#define HBAR  1.054571817e-34
#define K_B   1.380649e-23
#define M_0   9.1093837015e-31
#define EPS_0 8.8541878128e-12
#define PI_D  3.14159265358979323846

struct orc_sim {
    orc_config c;
    int nb, ncell;
    double m[ORC_NV], a[ORC_NV], Ec[ORC_NV]; /* kg, 1/J, J */
    double hw_lo, hw_iv, kT, beta2, N_lo, N_iv, dE, w, Vcell, dx, dy, dz;
    double *table; /* [NV][NB][NM] cumulative rate / Gamma0 */
    double gamma0[ORC_NV];
    int64_t cap;
    double *kx, *ky, *kz, *x, *y, *z, *tr;
    int32_t *valley;
    uint8_t *alive;
    uint64_t *ctr;
    uint64_t *events; /* [ncell][NV][NM] */
    int64_t *charge;  /* [ncell] */
    double *phi, *Ef; /* [ncell], [ncell][3] */
    orc_tallies t;
    /* per-subcell temperature: bins T_k = 250 + 5 k K, k = 0..150 */
    int tmode;
    double *btab;            /* [NTB][NV][NB][NM] cumulative / Gamma0 of the bin */
    double bg0[151][ORC_NV]; /* Gamma0 of each bin */
    double bbeta2[151], bkT[151];
    double g0e[ORC_NV];      /* Gamma0 of the ensemble (maximum over the bins in use) */
    int *cbin;               /* [ncell] */
    int threads;             /* particle-loop threads (1: the plain serial loop) */
};

/* ---------------------------------------------------------------- Philox */
static uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t* hi)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two
 * round constants, and mixes the high halves with words 1, 3 and the key; the
 * key is bumped by the two Weyl constants between rounds (Salmon et al. 2011). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, hi1;
        uint32_t lo0 = mulhilo32(0xD2511F53u, c0, &hi0);
        uint32_t lo1 = mulhilo32(0xCD9E8D57u, c2, &hi1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): the top 23 bits as an odd multiple of 2^-24.  Exact in
 * float and double, never 0 or 1. */
double orc_u01(uint32_t x)
{
    return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0);
}

/* Four uniforms from particle id's stream; advances its counter. */
static void draw4(orc_sim* s, int64_t id, double u[4])
{
    uint32_t c[4] = {(uint32_t)s->ctr[id], (uint32_t)(s->ctr[id] >> 32), 0u, 0u};
    uint32_t k[2] = {s->c.seed, (uint32_t)id};
    uint32_t o[4];
    orc_philox4x32_10(c, k, o);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(o[i]);
    s->ctr[id] += 1;
}

/* ------------------------------------------------------------ Kane bands */
static double kane_gamma(double E, double a) { return E * (1.0 + a * E); }

/* kinetic energy of wave vector magnitude^2 k2 in valley v:
 * E = 2 g / (1 + sqrt(1 + 4 a g)) with g = hbar^2 k^2 / 2m (root of E(1+aE)=g) */
static double energy_k2(const orc_sim* s, int v, double k2)
{
    double g = HBAR * HBAR * k2 / (2.0 * s->m[v]);
    return 2.0 * g / (1.0 + sqrt(1.0 + 4.0 * s->a[v] * g));
}

static double kmag_E(const orc_sim* s, int v, double E)
{
    return sqrt(2.0 * s->m[v] * kane_gamma(E, s->a[v])) / HBAR;
}

/* --------------------------------------------------------------- rates */
/* Each rate is the golden-rule total out-scattering rate (1/s) at kinetic
 * energy E (J) in valley v. */
double orc_rate(const orc_sim* s, int v, int mech, double E)
{
    const double m = s->m[v], a = s->a[v];
    const double g = kane_gamma(E, a);
    if (E < 0.0 || mech < 0 || mech >= ORC_NM) return 0.0;
    if (!((s->c.mech_mask >> mech) & 1u)) return 0.0;
    if (mech == 3 && s->c.const_rate > 0.0) return s->c.const_rate;
    if (mech == 0) { /* ionized impurity, Brooks-Herring, N_I = N_d */
        if (E <= 0.0) return 0.0;
        double k = sqrt(2.0 * m * g) / HBAR;
        double es = s->c.eps_s * EPS_0;
        double num = s->c.Nd * pow(Q_E, 4) * m * k * (1.0 + 2.0 * a * E);
        double den = PI_D * pow(HBAR, 3) * es * es * s->beta2 * (4.0 * k * k + s->beta2);
        return num / den;
    }
    if (mech == 1 || mech == 2) { /* polar optical (Froehlich) */
        double Ep = (mech == 1) ? E + s->hw_lo : E - s->hw_lo;
        if (Ep <= 0.0) return 0.0;
        double gp = kane_gamma(Ep, a);
        double w0 = s->hw_lo / HBAR;
        double C0 = Q_E * Q_E * w0 * sqrt(m) * (1.0 / s->c.eps_inf - 1.0 / s->c.eps_s) /
                    (4.0 * sqrt(2.0) * PI_D * EPS_0 * HBAR);
        double occ = (mech == 1) ? s->N_lo : s->N_lo + 1.0;
        double sg = sqrt(g), sgp = sqrt(gp);
        double F; /* ln|(sg+sgp)/(sg-sgp)| / sg, with its E -> 0 limit 2/sgp */
        if (g == 0.0)
            F = 2.0 / sgp;
        else
            F = log(fabs((sg + sgp) / (sg - sgp))) / sg;
        return C0 * (1.0 + 2.0 * a * Ep) * F * occ;
    }
    if (mech == 3) { /* acoustic deformation potential, elastic equipartition */
        double Da = s->c.Da_eV * Q_E;
        return sqrt(2.0) * Da * Da * s->kT * pow(m, 1.5) * sqrt(g) * (1.0 + 2.0 * a * E) /
               (PI_D * pow(HBAR, 4) * s->c.rho * s->c.vs * s->c.vs);
    }
    if (mech >= 4 && mech < ORC_NM) { /* intervalley optical phonon */
        int j = (mech - 4) / 2;
        int absorb = ((mech - 4) % 2) == 0;
        int Zf = (j == v) ? s->c.Z[j] - 1 : s->c.Z[j];
        if (Zf <= 0) return 0.0;
        double Ep = E + (absorb ? s->hw_iv : -s->hw_iv) - (s->Ec[j] - s->Ec[v]);
        if (Ep <= 0.0) return 0.0;
        double mj = s->m[j], aj = s->a[j];
        double gp = kane_gamma(Ep, aj);
        double D = s->c.Dij_eV_per_m * Q_E;
        double wiv = s->hw_iv / HBAR;
        double occ = absorb ? s->N_iv : s->N_iv + 1.0;
        return D * D * (double)Zf * pow(mj, 1.5) * sqrt(gp) * (1.0 + 2.0 * aj * Ep) * occ /
               (sqrt(2.0) * PI_D * s->c.rho * pow(HBAR, 3) * wiv);
    }
    return 0.0;
}

/* temperature-dependent constants of the rates */
static void set_temperature_consts(orc_sim* s, double T)
{
    s->kT = K_B * T;
    s->beta2 = Q_E * Q_E * s->c.Nd / (s->c.eps_s * EPS_0 * s->kT);
    s->N_lo = 1.0 / (exp(s->hw_lo / s->kT) - 1.0);
    s->N_iv = 1.0 / (exp(s->hw_iv / s->kT) - 1.0);
}

/* Tables at the lower edge of each bin; Gamma0 per valley is the maximum
 * total over the table; entries are cumulative sums over the mechanism index
 * divided by Gamma0. */
static void build_tables(orc_sim* s)
{
    const int nb = s->nb;
    for (int v = 0; v < ORC_NV; ++v) {
        double gmax = 0.0;
        for (int b = 0; b < nb; ++b) {
            double E = b * s->dE, acc = 0.0;
            for (int mch = 0; mch < ORC_NM; ++mch) {
                acc += orc_rate(s, v, mch, E);
                s->table[((size_t)v * nb + b) * ORC_NM + mch] = acc;
            }
            if (acc > gmax) gmax = acc;
        }
        if (s->c.exact_rates) {
            /* exact mode: Gamma0 must bound the rates between the bin edges
             * too; take the maximum on an 8x finer grid with a 2% margin */
            for (int b = 0; b < 8 * nb; ++b) {
                double E = b * s->dE / 8.0, acc = 0.0;
                for (int mch = 0; mch < ORC_NM; ++mch) acc += orc_rate(s, v, mch, E);
                if (acc > gmax) gmax = acc;
            }
            gmax *= 1.02;
        }
        s->gamma0[v] = gmax;
        for (int b = 0; b < nb; ++b)
            for (int mch = 0; mch < ORC_NM; ++mch)
                s->table[((size_t)v * nb + b) * ORC_NM + mch] /= gmax;
    }
}

void orc_get_tables(const orc_sim* s, double* table, double* gamma0)
{
    memcpy(table, s->table, sizeof(double) * ORC_NV * (size_t)s->nb * ORC_NM);
    memcpy(gamma0, s->gamma0, sizeof(double) * ORC_NV);
}

/* ------------------------------------------------------- angle samplers */
/* POP: P(cos t) ~ 1/(k^2 + k'^2 - 2 k k' cos t) inverted exactly:
 * cos t = ((1 + xi) - (1 + 2 xi)^u) / xi, xi = 2 k k' / (k - k')^2. */
double orc_cos_pop(double k, double kp, double u)
{
    double d = k - kp;
    double xi = 2.0 * k * kp / (d * d);
    if (!(xi >= 1e-6)) return 1.0 - 2.0 * u;
    return ((1.0 + xi) - pow(1.0 + 2.0 * xi, u)) / xi;
}

/* Brooks-Herring: P(cos t) ~ 1/(2k^2(1 - cos t) + beta^2)^2 inverted exactly. */
double orc_cos_imp(double k, double beta2, double u)
{
    return 1.0 - 2.0 * u / (1.0 + 4.0 * k * k * (1.0 - u) / beta2);
}

/* Rotate (cos t, phi) about unit vector n into an absolute direction using the
 * branchless orthonormal basis of Duff et al. (JCGT 2017). */
void orc_rotate(const double n[3], double ct, double ph, double out[3])
{
    double sgn = copysign(1.0, n[2]);
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    double e1[3] = {1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]};
    double e2[3] = {b, sgn + n[1] * n[1] * a, -n[1]};
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double cp = cos(ph), sp = sin(ph);
    for (int i = 0; i < 3; ++i) out[i] = st * cp * e1[i] + st * sp * e2[i] + ct * n[i];
}

/* ------------------------------------------------------------- geometry */
static int cell_of(const orc_sim* s, int64_t p)
{
    if (s->c.geometry == 0) return 0;
    int ix = (int)floor(s->x[p] / s->dx), iy = (int)floor(s->y[p] / s->dy),
        iz = (int)floor(s->z[p] / s->dz);
    if (ix < 0) ix = 0;
    if (ix > s->c.nx - 1) ix = s->c.nx - 1;
    if (iy < 0) iy = 0;
    if (iy > s->c.ny - 1) iy = s->c.ny - 1;
    if (iz < 0) iz = 0;
    if (iz > s->c.nz - 1) iz = s->c.nz - 1;
    return (ix * s->c.ny + iy) * s->c.nz + iz;
}

/* ------------------------------------------------------------ particles */
static double valley_E(const orc_sim* s, int64_t p)
{
    double k2 = s->kx[p] * s->kx[p] + s->ky[p] * s->ky[p] + s->kz[p] * s->kz[p];
    return energy_k2(s, s->valley[p], k2);
}

/* Kane-Maxwellian g(E) exp(-E/kT) by rejection from Gamma(3/2, kT): the
 * proposal is -kT (ln u0 + ln u1 cos^2(pi u2 / 2)), accepted when
 * u3 h(Emax) <= h(E), h(E) = sqrt(1 + aE)(1 + 2aE), E <= Emax. */
static double draw_maxwell_E(orc_sim* s, int64_t id, int v)
{
    double a = s->a[v], Emax = s->c.emax_init_kT * s->kT;
    double hmax = sqrt(1.0 + a * Emax) * (1.0 + 2.0 * a * Emax);
    double E = 0.0, u[4];
    for (int trial = 0; trial < 1000; ++trial) {
        draw4(s, id, u);
        double c = cos(0.5 * PI_D * u[2]);
        E = -s->kT * (log(u[0]) + log(u[1]) * c * c);
        if (E <= Emax && u[3] * hmax <= sqrt(1.0 + a * E) * (1.0 + 2.0 * a * E)) return E;
    }
    return fmin(E, Emax);
}

/* A fresh thermal electron in valley 0: energy, isotropic direction, position
 * (uniform in the box [lo, lo+len] for the nanowire), then a flight time. */
static void new_electron(orc_sim* s, int64_t id, const double lo[3], const double len[3])
{
    double u[4];
    s->valley[id] = 0;
    double E = draw_maxwell_E(s, id, 0);
    double km = kmag_E(s, 0, E);
    draw4(s, id, u);
    double ct = 1.0 - 2.0 * u[0], st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * PI_D * u[1];
    s->kx[id] = km * st * cos(ph);
    s->ky[id] = km * st * sin(ph);
    s->kz[id] = km * ct;
    if (s->c.geometry == 1) {
        draw4(s, id, u);
        s->x[id] = lo[0] + u[0] * len[0];
        s->y[id] = lo[1] + u[1] * len[1];
        s->z[id] = lo[2] + u[2] * len[2];
    } else {
        s->x[id] = s->y[id] = s->z[id] = 0.0;
    }
    draw4(s, id, u);
    s->tr[id] = -log(u[0]) / (s->tmode ? s->g0e[0] : s->gamma0[0]);
    s->alive[id] = 1;
}

void orc_sample_initial_energy(const orc_sim* s0, int64_t n, double* E)
{
    orc_sim* s = (orc_sim*)s0;
    for (int64_t i = 0; i < n && i < s->cap; ++i) {
        uint64_t save = s->ctr[i];
        s->ctr[i] = 0;
        E[i] = draw_maxwell_E(s, i, 0);
        s->ctr[i] = save;
    }
}

/* --------------------------------------------------------- free flight */
/* Drift particle p for time t under field F (V/m): hbar dk/dt = -q F.  Along
 * F the displacement follows from energy conservation (dE = -q F . dr); across
 * F it is the mean of the start and end group velocities times t. */
static void drift(orc_sim* s, int64_t p, const double F[3], double t)
{
    int v = s->valley[p];
    double k0[3] = {s->kx[p], s->ky[p], s->kz[p]};
    double k1[3];
    for (int i = 0; i < 3; ++i) k1[i] = k0[i] - Q_E * F[i] * t / HBAR;
    s->kx[p] = k1[0];
    s->ky[p] = k1[1];
    s->kz[p] = k1[2];
    if (s->c.geometry == 0) return;
    double E0 = energy_k2(s, v, k0[0] * k0[0] + k0[1] * k0[1] + k0[2] * k0[2]);
    double E1 = energy_k2(s, v, k1[0] * k1[0] + k1[1] * k1[1] + k1[2] * k1[2]);
    double f0 = HBAR / (s->m[v] * (1.0 + 2.0 * s->a[v] * E0));
    double f1 = HBAR / (s->m[v] * (1.0 + 2.0 * s->a[v] * E1));
    double dr[3];
    for (int i = 0; i < 3; ++i) dr[i] = 0.5 * (f0 * k0[i] + f1 * k1[i]) * t;
    double Fm = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    if (Fm > 0.0) {
        double fh[3] = {F[0] / Fm, F[1] / Fm, F[2] / Fm};
        double par_trap = dr[0] * fh[0] + dr[1] * fh[1] + dr[2] * fh[2];
        double par = -(E1 - E0) / (Q_E * Fm);
        for (int i = 0; i < 3; ++i) dr[i] += (par - par_trap) * fh[i];
    }
    s->x[p] += dr[0];
    s->y[p] += dr[1];
    s->z[p] += dr[2];
}

/* ----------------------------------------------------------- boundaries */
/* cosine-weighted direction about inward normal axis (sign sn on axis ax)
 * with tangents t1, t2; |k| kept. */
static void diffuse_k(orc_sim* s, int64_t p, int ax, double sn, const double u[4])
{
    double km = sqrt(s->kx[p] * s->kx[p] + s->ky[p] * s->ky[p] + s->kz[p] * s->kz[p]);
    double ca = sqrt(u[1]), sa = sqrt(1.0 - u[1]), ph = 2.0 * PI_D * u[2];
    double d[3];
    if (ax == 1) { /* y wall: tangents x, z */
        d[0] = sa * cos(ph);
        d[1] = sn * ca;
        d[2] = sa * sin(ph);
    } else { /* z wall: tangents x, y */
        d[0] = sa * cos(ph);
        d[1] = sa * sin(ph);
        d[2] = sn * ca;
    }
    s->kx[p] = km * d[0];
    s->ky[p] = km * d[1];
    s->kz[p] = km * d[2];
}

/* Contacts (absorb at x < 0 / x > Lx), plane A (y = 0, always specular), and
 * the outer side / bottom / top walls (specular with probability p, else
 * diffuse).  Returns 1 if the particle left through a contact. */
static int walls(orc_sim* s, int64_t p, orc_tallies* t)
{
    if (s->x[p] < 0.0) {
        s->alive[p] = 0;
        t->crossings[0]++;
        return 1;
    }
    if (s->x[p] > s->c.Lx) {
        s->alive[p] = 0;
        t->crossings[1]++;
        return 1;
    }
    double u[4];
    if (s->y[p] < 0.0) {
        s->y[p] = -s->y[p];
        s->ky[p] = -s->ky[p];
    } else if (s->y[p] > s->c.Ly) {
        s->y[p] = 2.0 * s->c.Ly - s->y[p];
        draw4(s, p, u);
        if (u[0] < s->c.p_spec) s->ky[p] = -s->ky[p];
        else diffuse_k(s, p, 1, -1.0, u);
    }
    if (s->y[p] < 0.0) s->y[p] = 0.0;
    if (s->y[p] > s->c.Ly) s->y[p] = s->c.Ly;
    if (s->z[p] < 0.0) {
        s->z[p] = -s->z[p];
        draw4(s, p, u);
        if (u[0] < s->c.p_spec) s->kz[p] = -s->kz[p];
        else diffuse_k(s, p, 2, 1.0, u);
    } else if (s->z[p] > s->c.Lz) {
        s->z[p] = 2.0 * s->c.Lz - s->z[p];
        draw4(s, p, u);
        if (u[0] < s->c.p_spec) s->kz[p] = -s->kz[p];
        else diffuse_k(s, p, 2, -1.0, u);
    }
    if (s->z[p] < 0.0) s->z[p] = 0.0;
    if (s->z[p] > s->c.Lz) s->z[p] = s->c.Lz;
    return 0;
}

/* -------------------------------------------------------------- scatter */
static void scatter(orc_sim* s, int64_t p, orc_tallies* t, uint64_t* events)
{
    double u[4];
    draw4(s, p, u);
    int v = s->valley[p];
    double k2 = s->kx[p] * s->kx[p] + s->ky[p] * s->ky[p] + s->kz[p] * s->kz[p];
    double E = energy_k2(s, v, k2);
    double fb = floor(E / s->dE);
    int b;
    if (fb >= (double)s->nb) {
        b = s->nb - 1;
        t->overflow++;
    } else {
        b = (int)fb;
    }
    const double* C = s->table + ((size_t)v * s->nb + b) * ORC_NM;
    double beta2 = s->beta2;
    int mech = -1;
    if (s->tmode) {
        /* the table of the particle's subcell temperature, tried against the
         * ensemble's Gamma0 */
        int k = s->cbin[cell_of(s, p)];
        C = s->btab + (((size_t)k * ORC_NV + v) * s->nb + b) * ORC_NM;
        u[0] = u[0] * (s->g0e[v] / s->bg0[k][v]);
        beta2 = s->bbeta2[k];
    }
    if (s->c.exact_rates && !s->tmode) {
        double acc = 0.0;
        for (int m = 0; m < ORC_NM; ++m) {
            acc += orc_rate(s, v, m, E) / s->gamma0[v];
            if (mech < 0 && u[0] < acc) mech = m;
        }
        if (acc > 1.0) t->overflow++;
    } else {
        for (int m = 0; m < ORC_NM; ++m)
            if (u[0] < C[m]) {
                mech = m;
                break;
            }
    }
    int vn = v;
    if (mech >= 0) {
        double Ep;
        int j = v;
        if (mech == 0 || mech == 3) Ep = E;
        else if (mech == 1) Ep = E + s->hw_lo;
        else if (mech == 2) Ep = E - s->hw_lo;
        else {
            j = (mech - 4) / 2;
            Ep = E + (((mech - 4) % 2) == 0 ? s->hw_iv : -s->hw_iv) - (s->Ec[j] - s->Ec[v]);
        }
        if (!(Ep > 0.0)) {
            t->rejected++;
            mech = -1;
        } else {
            double k = sqrt(k2);
            double kp = kmag_E(s, j, Ep);
            double ph = 2.0 * PI_D * u[3];
            double dir[3];
            if (mech == 0 || mech == 1 || mech == 2) {
                double n[3] = {0.0, 0.0, 1.0};
                if (k > 0.0) {
                    n[0] = s->kx[p] / k;
                    n[1] = s->ky[p] / k;
                    n[2] = s->kz[p] / k;
                }
                double ct = (mech == 0) ? orc_cos_imp(k, beta2, u[2]) : orc_cos_pop(k, kp, u[2]);
                orc_rotate(n, ct, ph, dir);
            } else {
                double ct = 1.0 - 2.0 * u[2], st = sqrt(fmax(0.0, 1.0 - ct * ct));
                dir[0] = st * cos(ph);
                dir[1] = st * sin(ph);
                dir[2] = ct;
            }
            s->kx[p] = kp * dir[0];
            s->ky[p] = kp * dir[1];
            s->kz[p] = kp * dir[2];
            s->valley[p] = j;
            vn = j;
            events[((size_t)cell_of(s, p) * ORC_NV + v) * ORC_NM + mech]++;
        }
    }
    if (mech < 0) t->self_events[v]++;
    s->tr[p] = -log(u[1]) / (s->tmode ? s->g0e[vn] : s->gamma0[vn]);
}

/* ------------------------------------------------------------- Poisson */
/* Cell-centred 7-point finite differences of div(eps_s eps0 grad phi) = -rho on
 * the subcell grid.  Dirichlet faces (source x = 0: Vs, drain x = Lx: Vd, and
 * the gate on the top and outer side faces where the cell centre lies in
 * [gate_x0, gate_x1]: Vg) sit half a cell from the centre; every other face is
 * Neumann (plane A, bottom, ungated top/side). */
static int is_gate(const orc_config* c, int ix)
{
    if (!c->gate_on) return 0;
    double xc = (ix + 0.5) * c->Lx / c->nx;
    return xc >= c->gate_x0 && xc <= c->gate_x1;
}

/* out = L phi, L = -(discrete Laplacian) with homogeneous Dirichlet faces. */
void orc_poisson_apply(const orc_config* c, const double* phi, double* out)
{
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    double ax = 1.0 / pow(c->Lx / nx, 2), ay = 1.0 / pow(c->Ly / ny, 2), az = 1.0 / pow(c->Lz / nz, 2);
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int l = 0; l < nz; ++l) {
                int id = (i * ny + j) * nz + l;
                double pc = phi[id], acc = 0.0;
                if (i > 0) acc += ax * (pc - phi[id - ny * nz]);
                else acc += 2.0 * ax * pc;
                if (i < nx - 1) acc += ax * (pc - phi[id + ny * nz]);
                else acc += 2.0 * ax * pc;
                if (j > 0) acc += ay * (pc - phi[id - nz]);
                if (j < ny - 1) acc += ay * (pc - phi[id + nz]);
                else if (is_gate(c, i)) acc += 2.0 * ay * pc;
                if (l > 0) acc += az * (pc - phi[id - 1]);
                if (l < nz - 1) acc += az * (pc - phi[id + 1]);
                else if (is_gate(c, i)) acc += 2.0 * az * pc;
                out[id] = acc;
            }
}

static void poisson_rhs(const orc_config* c, const double* rho, double* b)
{
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    double ax = 1.0 / pow(c->Lx / nx, 2), ay = 1.0 / pow(c->Ly / ny, 2), az = 1.0 / pow(c->Lz / nz, 2);
    double es = c->eps_s * EPS_0;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int l = 0; l < nz; ++l) {
                int id = (i * ny + j) * nz + l;
                double r = rho ? rho[id] / es : 0.0;
                if (i == 0) r += 2.0 * ax * c->Vs;
                if (i == nx - 1) r += 2.0 * ax * c->Vd;
                if (j == ny - 1 && is_gate(c, i)) r += 2.0 * ay * c->Vg;
                if (l == nz - 1 && is_gate(c, i)) r += 2.0 * az * c->Vg;
                b[id] = r;
            }
}

/* Conjugate gradients on L phi = b, starting from the phi passed in; stops
 * when ||r|| <= tol ||b||.  Returns the iteration count, or -1. */
int orc_poisson(const orc_config* c, const double* rho, double* phi, double tol, int maxit)
{
    int n = c->nx * c->ny * c->nz;
    double *b = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n),
           *d = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    poisson_rhs(c, rho, b);
    orc_poisson_apply(c, phi, q);
    double bb = 0.0, rr = 0.0;
    for (int i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        d[i] = r[i];
        bb += b[i] * b[i];
        rr += r[i] * r[i];
    }
    int it = 0, ok = -1;
    double stop = tol * tol * (bb > 0.0 ? bb : 1.0);
    for (; it <= maxit; ++it) {
        if (rr <= stop) {
            ok = it;
            break;
        }
        orc_poisson_apply(c, d, q);
        double dq = 0.0;
        for (int i = 0; i < n; ++i) dq += d[i] * q[i];
        double al = rr / dq, rn = 0.0;
        for (int i = 0; i < n; ++i) {
            phi[i] += al * d[i];
            r[i] -= al * q[i];
            rn += r[i] * r[i];
        }
        double be = rn / rr;
        rr = rn;
        for (int i = 0; i < n; ++i) d[i] = r[i] + be * d[i];
    }
    free(b);
    free(r);
    free(d);
    free(q);
    return ok;
}

/* E = -grad phi per cell: central differences inside, one-sided differences
 * with the interior neighbour in the boundary cells, zero along an axis of
 * one cell. */
void orc_field(const orc_config* c, const double* phi, double* Ef)
{
    const int n[3] = {c->nx, c->ny, c->nz};
    const double h[3] = {c->Lx / c->nx, c->Ly / c->ny, c->Lz / c->nz};
    const int st[3] = {c->ny * c->nz, c->nz, 1};
    for (int i = 0; i < c->nx; ++i)
        for (int j = 0; j < c->ny; ++j)
            for (int l = 0; l < c->nz; ++l) {
                int id = (i * c->ny + j) * c->nz + l;
                int idx[3] = {i, j, l};
                for (int a = 0; a < 3; ++a) {
                    double g;
                    if (n[a] == 1) g = 0.0;
                    else if (idx[a] == 0) g = (phi[id + st[a]] - phi[id]) / h[a];
                    else if (idx[a] == n[a] - 1) g = (phi[id] - phi[id - st[a]]) / h[a];
                    else g = (phi[id + st[a]] - phi[id - st[a]]) / (2.0 * h[a]);
                    Ef[id * 3 + a] = -g;
                }
            }
}

/* ------------------------------------------------------ nanowire chunk */
static void count_charge(orc_sim* s)
{
    memset(s->charge, 0, sizeof(int64_t) * s->ncell);
    for (int64_t p = 0; p < s->cap; ++p)
        if (s->alive[p]) s->charge[cell_of(s, p)]++;
}

/* Refill each contact cell (the x = 0 and x = Lx layers, source first, cells
 * in (y, z) order) up to N_d V_cell / w electrons, taking dead particle ids in
 * increasing order. */
static void inject(orc_sim* s)
{
    int64_t target = llround(s->c.Nd * s->Vcell / s->w);
    int64_t next = 0;
    for (int side = 0; side < 2; ++side) {
        int ix = side == 0 ? 0 : s->c.nx - 1;
        for (int j = 0; j < s->c.ny; ++j)
            for (int l = 0; l < s->c.nz; ++l) {
                int cid = (ix * s->c.ny + j) * s->c.nz + l;
                int64_t need = target - s->charge[cid];
                for (int64_t q = 0; q < need; ++q) {
                    while (next < s->cap && s->alive[next]) ++next;
                    if (next >= s->cap) {
                        s->t.inject_starved += need - q;
                        break;
                    }
                    double lo[3] = {ix * s->dx, j * s->dy, l * s->dz};
                    double len[3] = {s->dx, s->dy, s->dz};
                    if (s->tmode) set_temperature_consts(s, 250.0 + 5.0 * s->cbin[cid]);
                    new_electron(s, next, lo, len);
                    if (s->tmode) set_temperature_consts(s, s->c.T);
                    s->t.crossings[2 + side]++;
                    ++next;
                }
            }
    }
}

static void solve_field(orc_sim* s)
{
    double* rho = malloc(sizeof(double) * s->ncell);
    for (int c = 0; c < s->ncell; ++c)
        rho[c] = Q_E * (s->c.Nd - s->w * (double)s->charge[c] / s->Vcell);
    orc_poisson(&s->c, rho, s->phi, 1e-13, 100000);
    orc_field(&s->c, s->phi, s->Ef);
    free(rho);
}

/* ---------------------------------------------------------------- setup */
orc_sim* orc_create(const orc_config* cfg)
{
    orc_sim* s = calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    s->threads = 1;
    s->nb = cfg->n_bins;
    s->ncell = cfg->geometry == 1 ? cfg->nx * cfg->ny * cfg->nz : 1;
    for (int v = 0; v < ORC_NV; ++v) {
        s->m[v] = cfg->m_rel[v] * M_0;
        s->a[v] = cfg->alpha_per_eV[v] / Q_E;
        s->Ec[v] = cfg->Ec_eV[v] * Q_E;
    }
    s->hw_lo = cfg->hw_lo_eV * Q_E;
    s->hw_iv = cfg->hw_iv_eV * Q_E;
    s->kT = K_B * cfg->T;
    s->beta2 = Q_E * Q_E * cfg->Nd / (cfg->eps_s * EPS_0 * s->kT);
    s->N_lo = 1.0 / (exp(s->hw_lo / s->kT) - 1.0);
    s->N_iv = 1.0 / (exp(s->hw_iv / s->kT) - 1.0);
    s->dE = cfg->dE_eV * Q_E;
    s->table = malloc(sizeof(double) * ORC_NV * (size_t)s->nb * ORC_NM);
    build_tables(s);
    s->cap = cfg->capacity > cfg->n_particles ? cfg->capacity : cfg->n_particles;
    int64_t n = s->cap > 0 ? s->cap : 1;
    s->kx = calloc(n, sizeof(double));
    s->ky = calloc(n, sizeof(double));
    s->kz = calloc(n, sizeof(double));
    s->x = calloc(n, sizeof(double));
    s->y = calloc(n, sizeof(double));
    s->z = calloc(n, sizeof(double));
    s->tr = calloc(n, sizeof(double));
    s->valley = calloc(n, sizeof(int32_t));
    s->alive = calloc(n, 1);
    s->ctr = calloc(n, sizeof(uint64_t));
    s->events = calloc((size_t)s->ncell * ORC_NV * ORC_NM, sizeof(uint64_t));
    s->charge = calloc(s->ncell, sizeof(int64_t));
    s->phi = calloc(s->ncell, sizeof(double));
    s->Ef = calloc((size_t)s->ncell * 3, sizeof(double));
    if (cfg->geometry == 1) {
        s->dx = cfg->Lx / cfg->nx;
        s->dy = cfg->Ly / cfg->ny;
        s->dz = cfg->Lz / cfg->nz;
        s->Vcell = s->dx * s->dy * s->dz;
        s->w = cfg->n_particles > 0 ? cfg->Nd * cfg->Lx * cfg->Ly * cfg->Lz / (double)cfg->n_particles : 1.0;
    } else {
        s->Vcell = 1.0;
        s->w = 1.0;
    }
    double lo[3] = {0.0, 0.0, 0.0}, len[3] = {cfg->Lx, cfg->Ly, cfg->Lz};
    for (int64_t p = 0; p < cfg->n_particles; ++p) new_electron(s, p, lo, len);
    if (cfg->geometry == 1) {
        count_charge(s);
        solve_field(s);
    }
    s->t.n_alive = cfg->n_particles;
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->table);
    free(s->kx); free(s->ky); free(s->kz);
    free(s->x); free(s->y); free(s->z);
    free(s->tr); free(s->valley); free(s->alive); free(s->ctr);
    free(s->events); free(s->charge); free(s->phi); free(s->Ef);
    free(s->btab); free(s->cbin);
    free(s);
}

int orc_ncell(const orc_sim* s) { return s->ncell; }

/* Lattice temperature per subcell (n = subcell count, or 1): bins of 5 K
 * from 250 K, nearest bin per subcell; the ensemble's Gamma0 is the largest
 * total rate over the bins in use and residual flights are rescaled by
 * Gamma0_old / Gamma0_new. */
void orc_set_temperature(orc_sim* s, const double* T, int n)
{
    const int NTB = 151;
    if (!s->tmode) {
        s->btab = malloc(sizeof(double) * NTB * ORC_NV * (size_t)s->nb * ORC_NM);
        double* keep = s->table;
        double keepg[ORC_NV];
        memcpy(keepg, s->gamma0, sizeof keepg);
        for (int k = 0; k < NTB; ++k) {
            set_temperature_consts(s, 250.0 + 5.0 * k);
            s->table = s->btab + (size_t)k * ORC_NV * s->nb * ORC_NM;
            build_tables(s);
            memcpy(s->bg0[k], s->gamma0, sizeof s->bg0[k]);
            s->bbeta2[k] = s->beta2;
            s->bkT[k] = s->kT;
        }
        s->table = keep;
        memcpy(s->gamma0, keepg, sizeof keepg);
        set_temperature_consts(s, s->c.T);
        s->cbin = malloc(sizeof(int) * s->ncell);
        memcpy(s->g0e, s->gamma0, sizeof s->g0e);
        s->tmode = 1;
    }
    for (int c = 0; c < s->ncell; ++c) {
        double t = (n == 1) ? T[0] : T[c];
        long k = lround((t - 250.0) / 5.0);
        if (k < 0) k = 0;
        if (k > NTB - 1) k = NTB - 1;
        s->cbin[c] = (int)k;
    }
    double gnew[ORC_NV] = {0.0, 0.0, 0.0};
    for (int c = 0; c < s->ncell; ++c)
        for (int v = 0; v < ORC_NV; ++v)
            if (s->bg0[s->cbin[c]][v] > gnew[v]) gnew[v] = s->bg0[s->cbin[c]][v];
    for (int64_t p = 0; p < s->cap; ++p)
        if (s->alive[p]) s->tr[p] *= s->g0e[s->valley[p]] / gnew[s->valley[p]];
    memcpy(s->g0e, gnew, sizeof gnew);
}

void orc_set_bias(orc_sim* s, double Vs, double Vd, double Vg)
{
    s->c.Vs = Vs;
    s->c.Vd = Vd;
    s->c.Vg = Vg;
    if (s->c.geometry == 1) solve_field(s);
}

/* ------------------------------------------------------------------ run */
/* One time step of particle p: flights and scatterings until the step ends,
 * then the particle-step sample.  Tallies go to t / events. */
static void step_particle(orc_sim* s, int64_t p, orc_tallies* t, uint64_t* events)
{
    const int nw = s->c.geometry == 1;
    const double* F = nw ? s->Ef + 3 * (size_t)cell_of(s, p) : s->c.field;
    double tleft = s->c.dt;
    for (;;) {
        if (s->tr[p] >= tleft) {
            drift(s, p, F, tleft);
            s->tr[p] -= tleft;
            if (nw) walls(s, p, t);
            break;
        }
        drift(s, p, F, s->tr[p]);
        tleft -= s->tr[p];
        if (nw && walls(s, p, t)) break;
        scatter(s, p, t, events);
    }
    if (!s->alive[p]) return;
    int v = s->valley[p];
    double k[3] = {s->kx[p], s->ky[p], s->kz[p]};
    double E = energy_k2(s, v, k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    double f = HBAR / (s->m[v] * (1.0 + 2.0 * s->a[v] * E));
    for (int i = 0; i < 3; ++i) t->sum_v[i] += f * k[i];
    t->sum_E += E;
    t->sum_Etot += E + s->Ec[v];
    t->valley_steps[v]++;
    t->n_samples++;
}

/* add the per-step tallies of b into a */
static void add_tallies(orc_tallies* a, const orc_tallies* b)
{
    for (int i = 0; i < ORC_NV; ++i) {
        a->self_events[i] += b->self_events[i];
        a->valley_steps[i] += b->valley_steps[i];
    }
    a->overflow += b->overflow;
    a->rejected += b->rejected;
    for (int i = 0; i < 4; ++i) a->crossings[i] += b->crossings[i];
    a->n_samples += b->n_samples;
    for (int i = 0; i < 3; ++i) a->sum_v[i] += b->sum_v[i];
    a->sum_E += b->sum_E;
    a->sum_Etot += b->sum_Etot;
}

/* Particles are independent within a step (each has its own random stream
 * and the field changes only between steps), so the particle loop may run on
 * several threads.  Thread 0 accumulates into the simulation's own tallies,
 * which makes one thread exactly the plain serial loop; every other thread
 * keeps its own partial tallies, added in thread order after each step
 * (integer tallies are then identical for any thread count; floating sums
 * differ only by the order of additions). */
void orc_run(orc_sim* s, int64_t n_steps)
{
    const int nw = s->c.geometry == 1;
    const int nt = s->threads > 1 ? s->threads : 1;
    const size_t nev = (size_t)s->ncell * ORC_NV * ORC_NM;
    orc_tallies* pt = calloc((size_t)nt, sizeof(orc_tallies));
    uint64_t** pev = calloc((size_t)nt, sizeof(uint64_t*));
    pev[0] = s->events;
    for (int i = 1; i < nt; ++i) pev[i] = calloc(nev, sizeof(uint64_t));
    for (int64_t st = 0; st < n_steps; ++st) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
        for (int64_t p = 0; p < s->cap; ++p) {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            if (s->alive[p]) step_particle(s, p, tid == 0 ? &s->t : &pt[tid], pev[tid]);
        }
        for (int i = 1; i < nt; ++i) {
            add_tallies(&s->t, &pt[i]);
            memset(&pt[i], 0, sizeof(orc_tallies));
        }
        s->t.steps_done++;
        if (nw && (s->t.steps_done % s->c.steps_per_poisson) == 0) {
            count_charge(s);
            inject(s);
            count_charge(s);
            solve_field(s);
        }
    }
    for (int i = 1; i < nt; ++i) {
        for (size_t j = 0; j < nev; ++j) s->events[j] += pev[i][j];
        free(pev[i]);
    }
    free(pev);
    free(pt);
    int64_t alive = 0;
    for (int64_t p = 0; p < s->cap; ++p) alive += s->alive[p];
    s->t.n_alive = alive;
    if (!nw) s->charge[0] = alive;
}

void orc_set_threads(orc_sim* s, int n) { s->threads = n > 1 ? n : 1; }

/* ------------------------------------------------------------ test hooks */
/* One free flight of a lone electron in valley v from wave vector k0 and
 * position r0 under the field F (V/m) for time t: the nanowire's position
 * update (particle slot 0 of s serves as scratch). */
void orc_test_drift(orc_sim* s, int v, const double k0[3], const double r0[3], const double F[3], double t,
                    double k1[3], double r1[3])
{
    s->valley[0] = v;
    s->kx[0] = k0[0]; s->ky[0] = k0[1]; s->kz[0] = k0[2];
    s->x[0] = r0[0]; s->y[0] = r0[1]; s->z[0] = r0[2];
    drift(s, 0, F, t);
    k1[0] = s->kx[0]; k1[1] = s->ky[0]; k1[2] = s->kz[0];
    r1[0] = s->x[0]; r1[1] = s->y[0]; r1[2] = s->z[0];
}

/* The wall and contact treatment of a lone electron at position r0 with wave
 * vector k0 whose random stream (key: the ensemble seed and particle id 0)
 * stands at counter ctr.  Returns 1 if it left through a contact; r1, k1 and
 * *ctr_out receive the state after the walls (slot 0 of s is scratch). */
int orc_test_walls(orc_sim* s, const double r0[3], const double k0[3], uint64_t ctr, double r1[3], double k1[3],
                   uint64_t* ctr_out)
{
    orc_tallies t;
    memset(&t, 0, sizeof t);
    s->alive[0] = 1;
    s->kx[0] = k0[0]; s->ky[0] = k0[1]; s->kz[0] = k0[2];
    s->x[0] = r0[0]; s->y[0] = r0[1]; s->z[0] = r0[2];
    s->ctr[0] = ctr;
    int out = walls(s, 0, &t);
    k1[0] = s->kx[0]; k1[1] = s->ky[0]; k1[2] = s->kz[0];
    r1[0] = s->x[0]; r1[1] = s->y[0]; r1[2] = s->z[0];
    *ctr_out = s->ctr[0];
    return out;
}

void orc_get_tallies(const orc_sim* s, orc_tallies* out) { *out = s->t; }

void orc_get_events(const orc_sim* s, uint64_t* ev)
{
    memcpy(ev, s->events, sizeof(uint64_t) * (size_t)s->ncell * ORC_NV * ORC_NM);
}

void orc_get_charge(const orc_sim* s, int64_t* ch)
{
    orc_sim* m = (orc_sim*)s;
    if (s->c.geometry == 1) count_charge(m);
    memcpy(ch, s->charge, sizeof(int64_t) * s->ncell);
}

void orc_get_phi(const orc_sim* s, double* phi, double* Ef)
{
    memcpy(phi, s->phi, sizeof(double) * s->ncell);
    memcpy(Ef, s->Ef, sizeof(double) * 3 * (size_t)s->ncell);
}

void orc_get_particles(const orc_sim* s, double* k, double* r, double* tr, int32_t* valley,
                       uint8_t* alive, uint64_t* ctr)
{
    for (int64_t p = 0; p < s->cap; ++p) {
        k[3 * p] = s->kx[p];
        k[3 * p + 1] = s->ky[p];
        k[3 * p + 2] = s->kz[p];
        r[3 * p] = s->x[p];
        r[3 * p + 1] = s->y[p];
        r[3 * p + 2] = s->z[p];
        tr[p] = s->tr[p];
        valley[p] = s->valley[p];
        alive[p] = s->alive[p];
        ctr[p] = s->ctr[p];
    }
}
