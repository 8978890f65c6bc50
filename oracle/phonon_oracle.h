/* FP64 CPU oracle of the phonon Monte Carlo (test infrastructure only). */
#ifndef PHONON_ORACLE_H
#define PHONON_ORACLE_H
#include <stdint.h>

enum { PH_SPECULAR = 0, PH_ROUGH = 1, PH_ISOTHERMAL = 2, PH_INTERFACE = 3 };

typedef struct {
    int32_t nx, ny, nz, nb, nt, pad_;
    double Lx, Ly, Lz;          /* nm */
    const double* vg;           /* [nb] group velocity of each frequency bin, nm/ps */
    const double* rate;         /* [nt][nb] scattering rate 1/tau, 1/ps */
    const double* cdf;          /* [nt][nb] cumulative of C / tau (last = 1) */
    const int32_t* tix;         /* [C] rate table of each subcell */
    const double* cell_cdf;     /* [C] cumulative of the subcells' |heat| (last = 1) */
    const double* cell_sign;    /* [C] +1, or -1 where the heat is negative */
    const double* tau12;        /* [nb] interface transmissivity (PH_INTERFACE faces) */
    int32_t face[6];            /* faces x=0, x=Lx, y=0, y=Ly, z=0, z=Lz */
    double p_specular[6];       /* PH_ROUGH faces */
    uint32_t seed, pad2_;
    int64_t max_segments;       /* per bundle */
} ph_problem;

typedef struct {
    double* t_res;              /* [C] time spent per subcell, ps (accumulating) */
    uint64_t* scatterings;      /* [C] */
    uint64_t* emitted;          /* [C] */
    uint64_t absorbed[6];       /* per face: absorbed (isothermal) or transmitted (interface) */
    uint64_t segments, capped;
} ph_tally;

void ph_run(const ph_problem* P, int64_t first, int64_t n, ph_tally* T);
void ph_test_lambert(int f, double u1, double u2, double d[3]);
void ph_test_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ph_test_draw(uint32_t seed, uint32_t id, uint64_t n0, int count, double* u);
#endif
