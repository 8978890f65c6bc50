/*
 * FP64 CPU oracle for the ensemble electron Monte Carlo of wurtzite GaN
 * (Hao et al., "Hybrid Electrothermal Simulation of a 3D FinFET Based on GaN
 * Nanowires", arXiv:1707.09073).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * library shares no code, header, table or constant with it.
 *
 * Everything is SI and double precision.  Valleys: 0 = Gamma1, 1 = U,
 * 2 = Gamma3.  Mechanism index per valley (ORC_NM = 10):
 *   0 ionized impurity (Brooks-Herring, elastic)
 *   1 polar optical absorption, 2 polar optical emission
 *   3 acoustic deformation potential (elastic, equipartition)
 *   4 + 2j intervalley absorption into valley j, 5 + 2j emission into j
 * Anything above the cumulative total of these is self-scattering.
 */
#ifndef EMC_ORACLE_H
#define EMC_ORACLE_H
#include <stdint.h>

#define ORC_NV 3
#define ORC_NM 10

typedef struct orc_config {
    double m_rel[3], Ec_eV[3], alpha_per_eV[3];
    double eps_s, eps_inf, rho, Da_eV, Dij_eV_per_m, hw_lo_eV, hw_iv_eV, vs;
    double T, Nd;          /* K, m^-3 */
    double field[3];       /* V/m, bulk only */
    double dt;             /* s */
    double dE_eV;          /* table bin width */
    double emax_init_kT;
    double Lx, Ly, Lz, gate_x0, gate_x1, Vs, Vd, Vg, p_spec;
    double const_rate;     /* test hook: >0 replaces the acoustic rate by this constant (1/s) */
    int64_t n_particles, capacity;
    int32_t Z[3];
    int32_t geometry;      /* 0 bulk, 1 half nanowire */
    int32_t n_bins, steps_per_poisson;
    int32_t nx, ny, nz, gate_on;
    uint32_t seed;
    uint32_t mech_mask;    /* bit m set = mechanism m enabled */
    int32_t exact_rates;   /* 1: rates at the exact energy instead of the table bin */
    int32_t pad_;
} orc_config;

typedef struct orc_sim orc_sim;

/* Tally snapshot (integer tallies are exact; sums are FP64). */
typedef struct orc_tallies {
    uint64_t self_events[ORC_NV];
    uint64_t overflow;            /* lookups above the table range */
    uint64_t rejected;            /* chosen channels with E' <= 0 (never expected) */
    int64_t crossings[4];         /* source out, drain out, source in, drain in */
    int64_t valley_steps[ORC_NV]; /* sum over steps of the valley population */
    int64_t n_samples;            /* particle-steps sampled */
    int64_t steps_done;
    int64_t n_alive;
    int64_t inject_starved;
    double sum_v[3];              /* sum over particle-steps of group velocity, m/s */
    double sum_E;                 /* kinetic energy, J */
    double sum_Etot;              /* kinetic + valley minimum, J */
} orc_tallies;

/* Philox4x32-10 (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);

orc_sim* orc_create(const orc_config* cfg);
void orc_destroy(orc_sim* s);
int orc_ncell(const orc_sim* s);
double orc_rate(const orc_sim* s, int valley, int mech, double E_J);
void orc_get_tables(const orc_sim* s, double* table /* [NV][NB][NM] */, double* gamma0 /* [NV] */);
void orc_run(orc_sim* s, int64_t n_steps);
/* threads of the particle loop in orc_run (default 1; integer tallies do not
 * depend on it) */
void orc_set_threads(orc_sim* s, int n);
void orc_get_tallies(const orc_sim* s, orc_tallies* out);
void orc_get_events(const orc_sim* s, uint64_t* ev /* [ncell][NV][NM] */);
void orc_get_charge(const orc_sim* s, int64_t* ch /* [ncell] */);
void orc_get_phi(const orc_sim* s, double* phi, double* Ef /* [ncell][3] */);
void orc_get_particles(const orc_sim* s, double* k /* [cap][3] */, double* r /* [cap][3] */,
                       double* tr, int32_t* valley, uint8_t* alive, uint64_t* ctr);
void orc_set_bias(orc_sim* s, double Vs, double Vd, double Vg);
void orc_set_temperature(orc_sim* s, const double* T, int n);
/* Kane-Maxwellian initial energy draw, exposed for distribution tests:
 * fills E[n] (J) from stream key (seed, id) starting at counter 0. */
void orc_sample_initial_energy(const orc_sim* s, int64_t n, double* E);
/* angle samplers (cos theta) for distribution tests */
double orc_cos_pop(double k, double kp, double u);
double orc_cos_imp(double k, double beta2, double u);
void orc_rotate(const double n[3], double ct, double ph, double out[3]);

/* test hooks (slot 0 of s is overwritten): one free flight, one pass
 * through the walls and contacts */
void orc_test_drift(orc_sim* s, int v, const double k0[3], const double r0[3], const double F[3], double t,
                    double k1[3], double r1[3]);
int orc_test_walls(orc_sim* s, const double r0[3], const double k0[3], uint64_t ctr, double r1[3], double k1[3],
                   uint64_t* ctr_out);

/* Poisson on the subcell grid: charge density rho (C/m^3) -> phi (V). */
int orc_poisson(const orc_config* cfg, const double* rho, double* phi, double tol, int maxit);
void orc_poisson_apply(const orc_config* cfg, const double* phi, double* out);
void orc_field(const orc_config* cfg, const double* phi, double* Ef);

#endif
