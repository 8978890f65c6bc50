/* FP64 CPU oracle of the phonon Monte Carlo of the transistor region
 * (TEST INFRASTRUCTURE ONLY: called by tests/ and bench.py's cpu_baseline
 * leg through oracle/phonon.py; never by the product library).
 *
 * What it computes.  Phonons of three identical sine-shaped acoustic
 * branches (the phonon-model paragraph and Table II) carry the heat that the
 * electrons emit in each subcell through the wire.  The steady temperature
 * rise follows from the energy-based deviational Monte Carlo of Peraud and
 * Hadjiconstantinou (2011): every simulated phonon bundle carries the same
 * share P / N of the power P = sum |q| V; a bundle is emitted in a subcell
 * with probability proportional to the magnitude of that subcell's heat,
 * and carries the heat's sign (negative where the electrons absorb more
 * phonon energy than they emit: a deficit of phonons); it flies at the group
 * velocity of its frequency, scatters at the rate 1/tau(omega, T) of the
 * paragraph's relaxation-time model (plus, optionally, the boundary term and
 * Eq. (1), folded into the rate tables the caller passes), is re-emitted
 * after a scattering with a frequency drawn from C(omega)/tau(omega) and an
 * isotropic direction (energy conserved bundle by bundle), and ends where it
 * leaves the domain through an isothermal face or is transmitted into the
 * substrate (Eq. (2)).  The deviational energy of subcell c is P times the
 * mean signed time a bundle spends there; divided by C V it is the
 * temperature rise.
 *
 * Frequencies are binned (the caller's bins; a bundle uses its bin's group
 * velocity and rates).  Lengths in nm, times in ps.
 *
 * Random numbers: Philox4x32-10 keyed by (seed, bundle id) with counter
 * words (n, 0, 0, 1), n = 0, 1, ... per bundle; four uniforms per call as
 * odd multiples of 2^-24.  Uses of each call:
 *   emission   call 0: subcell, position in the subcell (x, y, z);
 *              call 1: frequency bin, cos(theta) = 2u - 1, phi = 2 pi u,
 *                      optical depth -ln u;
 *   scattering one call: frequency bin, cos(theta), phi, optical depth;
 *   rough / interface face: one call: specular (u < p) or transmitted
 *              (u < tau12), then a cosine-law direction about the inward
 *              normal (cos(theta) = sqrt(u), phi = 2 pi u).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "phonon_oracle.h"

#define PI_D 3.14159265358979323846

static uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t* hi)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds; each
 * multiplies words 0 and 2 by the round constants and mixes the high halves
 * with words 1, 3 and the key; the key advances by the Weyl constants. */
static void philox(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
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

static double u01(uint32_t x) { return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0); }

typedef struct {
    uint32_t seed, id;
    uint64_t n;
} stream;

static void draw4(stream* s, double u[4])
{
    uint32_t c[4] = {(uint32_t)s->n, (uint32_t)(s->n >> 32), 0u, 1u};
    uint32_t o[4];
    philox(c, s->seed, s->id, o);
    for (int i = 0; i < 4; ++i) u[i] = u01(o[i]);
    s->n += 1;
}

/* smallest i in [0, n) with cdf[i] > u (cdf ascending, cdf[n-1] = 1) */
static int inverse_cdf(const double* cdf, int n, double u)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

static void isotropic(double cth, double phi, double d[3])
{
    double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    d[0] = sth * cos(phi);
    d[1] = sth * sin(phi);
    d[2] = cth;
}

/* cosine-law direction into the domain through face f (axis f/2; f even:
 * the low face, inward normal +axis; f odd: the high face, -axis); the two
 * tangent axes in the order (axis+1) % 3, (axis+2) % 3 */
static void lambert(int f, double u1, double u2, double d[3])
{
    int a = f / 2;
    double ct = sqrt(u1), st = sqrt(1.0 - u1), ph = 2.0 * PI_D * u2;
    d[a] = (f % 2 == 0) ? ct : -ct;
    d[(a + 1) % 3] = st * cos(ph);
    d[(a + 2) % 3] = st * sin(ph);
}

void ph_run(const ph_problem* P, int64_t first, int64_t n, ph_tally* T)
{
    const int nc[3] = {P->nx, P->ny, P->nz};
    const double L[3] = {P->Lx, P->Ly, P->Lz};
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = L[a] / nc[a];
    const int nb = P->nb;
    for (int64_t t = first; t < first + n; ++t) {
        stream s = {P->seed, (uint32_t)t, 0};
        double u[4];
        /* emission */
        draw4(&s, u);
        int c = inverse_cdf(P->cell_cdf, P->nx * P->ny * P->nz, u[0]);
        int ix[3];
        ix[0] = c / (P->ny * P->nz);
        ix[1] = (c / P->nz) % P->ny;
        ix[2] = c % P->nz;
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = (ix[a] + u[1 + a]) * h[a];
        T->emitted[c] += 1;
        const double sg = P->cell_sign[c];
        draw4(&s, u);
        int b = inverse_cdf(P->cdf + (size_t)P->tix[c] * nb, nb, u[0]);
        double d[3];
        isotropic(2.0 * u[1] - 1.0, 2.0 * PI_D * u[2], d);
        double depth = -log(u[3]);
        int64_t seg = 0;
        for (;;) {
            if (seg >= P->max_segments) {
                T->capped += 1;
                break;
            }
            seg += 1;
            T->segments += 1;
            const double v = P->vg[b];
            const double r = P->rate[(size_t)P->tix[c] * nb + b];
            /* time to the faces of the subcell, the earliest axis first */
            int ax = -1;
            double t_exit = INFINITY;
            for (int a = 0; a < 3; ++a) {
                double ta = INFINITY;
                if (d[a] > 0.0) ta = ((ix[a] + 1) * h[a] - p[a]) / (v * d[a]);
                else if (d[a] < 0.0) ta = (ix[a] * h[a] - p[a]) / (v * d[a]);
                if (ta < 0.0) ta = 0.0;
                if (ta < t_exit) {
                    t_exit = ta;
                    ax = a;
                }
            }
            const double t_scat = r > 0.0 ? depth / r : INFINITY;
            if (t_scat < t_exit) {
                for (int a = 0; a < 3; ++a) p[a] += v * d[a] * t_scat;
                T->t_res[c] += sg * t_scat;
                T->scatterings[c] += 1;
                draw4(&s, u);
                b = inverse_cdf(P->cdf + (size_t)P->tix[c] * nb, nb, u[0]);
                isotropic(2.0 * u[1] - 1.0, 2.0 * PI_D * u[2], d);
                depth = -log(u[3]);
                continue;
            }
            for (int a = 0; a < 3; ++a) p[a] += v * d[a] * t_exit;
            T->t_res[c] += sg * t_exit;
            depth -= r * t_exit;
            if (depth < 0.0) depth = 0.0;
            const int up = d[ax] > 0.0;
            p[ax] = (ix[ax] + up) * h[ax]; /* on the face */
            const int nxt = ix[ax] + (up ? 1 : -1);
            if (nxt >= 0 && nxt < nc[ax]) {
                ix[ax] = nxt;
                c = (ix[0] * P->ny + ix[1]) * P->nz + ix[2];
                continue;
            }
            /* a face of the domain */
            const int f = 2 * ax + up;
            const int kind = P->face[f];
            if (kind == PH_ISOTHERMAL) {
                T->absorbed[f] += 1;
                break;
            }
            if (kind == PH_SPECULAR) {
                d[ax] = -d[ax];
                continue;
            }
            draw4(&s, u);
            if (kind == PH_INTERFACE) {
                if (u[0] < P->tau12[b]) {
                    T->absorbed[f] += 1;
                    break;
                }
                lambert(f, u[1], u[2], d);
            } else { /* PH_ROUGH */
                if (u[0] < P->p_specular[f]) d[ax] = -d[ax];
                else lambert(f, u[1], u[2], d);
            }
        }
    }
}

void ph_test_lambert(int f, double u1, double u2, double d[3]) { lambert(f, u1, u2, d); }

void ph_test_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox(ctr, key[0], key[1], out); }

void ph_test_draw(uint32_t seed, uint32_t id, uint64_t n0, int count, double* u)
{
    stream s = {seed, id, n0};
    for (int i = 0; i < count; ++i) draw4(&s, u + 4 * i);
}
