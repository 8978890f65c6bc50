/*
 * libemc: GB300 (sm_103a) ensemble electron Monte Carlo for wurtzite GaN.
 *
 * Hao et al., "Hybrid Electrothermal Simulation of a Three-Dimensional
 * Fin-Shaped Field-Effect Transistor Based on GaN Nanowires" (arXiv:1707.09073).
 * The paper's electron side: an ensemble Monte Carlo that tracks individual
 * electrons (the hybrid-method paragraph), Kane bands over the Gamma1/U/Gamma3
 * valleys with ionized impurity, polar optical, acoustic deformation
 * potential and intervalley optical scattering and the Table I parameters
 * (the electron-model paragraph), a half nanowire divided into 3 x 6 x 100
 * subcells that count electrons for a Poisson update of the 3D field, and the
 * electron-to-phonon energy exchange counted per subcell for the thermal side
 * (the paragraph on the field update and the heat counted in steady state).
 *
 * Conventions for every entry point:
 *  - Return EMC_OK or an error code; nothing throws.  emc_last_error() gives
 *    the message of the last failure on a context.
 *  - The context owns all device memory it allocates (cudaMalloc at init,
 *    cudaFree at emc_destroy).  Caller pointers are never retained.
 *  - Work is issued asynchronously on the CUDA stream given at init (NULL =
 *    the legacy default stream).  Calls that copy results to the host
 *    synchronise that stream.  Asynchronous CUDA errors surface as EMC_ECUDA
 *    at the next call.
 *  - A context is not thread-safe; use one context per host thread.
 *  - Units: SI in emc_config; results are documented per tally kind.
 */
#ifndef LIBEMC_EMC_H
#define LIBEMC_EMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emc_ctx emc_ctx;

typedef enum emc_status {
    EMC_OK = 0,
    EMC_EINVAL = 1,     /* invalid argument or configuration */
    EMC_ENOMEM = 2,     /* device or host allocation failed */
    EMC_ECUDA = 3,      /* a CUDA call failed (message in emc_last_error) */
    EMC_EOVERFLOW = 4,  /* a device-side check failed: a bounded loop or buffer limit
                           was hit, or a particle's energy was not finite (the message
                           names the bits of the device error word) */
    EMC_ETIMEOUT = 5,   /* a bounded device wait gave up (the surrogate's tensor-core
                           GEMM waits on its mbarriers with an iteration limit) */
    EMC_ESTATE = 6      /* call not valid in the context's current state */
} emc_status;

enum { EMC_NV = 3, EMC_NM = 10 };
enum { EMC_GEOM_BULK = 0, EMC_GEOM_NANOWIRE = 1 };
enum { EMC_FP32 = 0, EMC_FP64 = 1 };

/* Mechanism index m per valley (EMC_NM = 10):
 *   0 ionized impurity (Brooks-Herring, elastic)
 *   1 polar optical absorption, 2 polar optical emission
 *   3 acoustic deformation potential (elastic, equipartition)
 *   4+2j intervalley absorption into valley j, 5+2j emission into valley j
 * Valleys: 0 Gamma1, 1 U, 2 Gamma3.  Self-scattering is counted apart. */

/* One ensemble.  All ensembles of one context must agree on geometry, grid,
 * precision, dt, n_bins, dE_eV and steps_per_poisson. */
typedef struct emc_config {
    /* Table I */
    double m_rel[3];        /* valley-bottom effective mass / m0 */
    double Ec_eV[3];        /* valley minima */
    double alpha_per_eV[3]; /* Kane nonparabolicity */
    double eps_s, eps_inf;  /* relative permittivities */
    double rho_kg_m3;       /* mass density */
    double Da_eV;           /* acoustic deformation potential */
    double Dij_eV_per_m;    /* intervalley deformation potential */
    /* readings of what the paper leaves open */
    double hw_lo_eV;        /* polar optical phonon energy (91.2 meV in the text) */
    double hw_iv_eV;        /* intervalley phonon energy */
    double vs_m_s;          /* sound velocity for acoustic scattering */
    /* operating point */
    double T_K;             /* lattice temperature */
    double Nd_m3;           /* ionized donors = electrons (full activation) */
    double field_V_m[3];    /* uniform field, bulk geometry only */
    double dt_s;            /* time step */
    double dE_eV;           /* rate-table bin width */
    double emax_init_kT;    /* truncation of the initial Kane-Maxwellian */
    /* nanowire geometry (x along the wire, y across from symmetry plane A, z up) */
    double Lx, Ly, Lz;      /* m */
    double gate_x0, gate_x1;/* gated x range on the top and outer side faces */
    double Vs, Vd, Vg;      /* terminal voltages */
    double p_specular;      /* specular fraction on the outer side/top/bottom walls */
    int64_t n_particles;    /* initial electrons (superparticles) */
    int64_t capacity;       /* particle slots (>= n_particles; spare slots for injection) */
    /* Particle sharding of one wire over several contexts (usually one per
     * GPU; see emc_shard_counts).  All three zero: unsharded.  A wire of N
     * initial electrons and S spare slots has global particle ids [0, N)
     * (initial electrons) and [N, N + S) (spare slots), as an unsharded
     * context numbers them.  A shard holds the global ids
     * [shard_live_base, shard_live_base + n_particles) and
     * [shard_spare_base, shard_spare_base + capacity - n_particles).  The
     * global id keys the particle's Philox stream, so every particle draws
     * the same numbers however the wire is split. */
    int64_t shard_n_global;   /* N, > 0 in a sharded context (the superparticle weight
                                 Nd V / N and the contact refill target use it) */
    int64_t shard_live_base;  /* global id of this shard's first initial electron */
    int64_t shard_spare_base; /* global id of this shard's first spare slot (>= N) */
    int32_t Z[3];           /* valley degeneracies */
    int32_t geometry;       /* EMC_GEOM_BULK or EMC_GEOM_NANOWIRE */
    int32_t n_bins;         /* rate-table bins (table spans [0, n_bins * dE_eV)) */
    int32_t steps_per_poisson; /* nanowire: Poisson update every this many steps */
    int32_t nx, ny, nz;     /* subcells */
    int32_t gate_on;        /* 1: gate Dirichlet faces present */
    uint32_t seed;          /* Philox key word 0 of this ensemble */
    uint32_t mech_mask;     /* bit m set: mechanism m enabled */
    int32_t precision;      /* EMC_FP32 (production) or EMC_FP64 (parity build) */
    int32_t sort_period;    /* sort particles every this many launches (0 = never) */
    int32_t block_size;     /* flight-kernel threads per block (0 = default 256) */
    int32_t steps_per_launch; /* bulk: steps fused per flight launch (0 = default 50, at most 1000) */
    int32_t table_smem_kb;  /* rate-table bytes staged in shared memory per block, KiB
                               (0 = default 32; bins above it are read through L1/L2) */
} emc_config;

/* Per-ensemble observables accumulated over sampled particle-steps (every
 * live particle is sampled at the end of every time step). */
typedef struct emc_obs {
    double sum_v[3];        /* group velocity, m/s */
    double sum_E;           /* kinetic energy, J */
    double sum_Etot;        /* kinetic + valley minimum, J */
    int64_t n_samples;      /* particle-steps sampled */
    int64_t valley_steps[3];/* particle-steps per valley */
    int64_t self_events[3]; /* self-scatterings per valley */
    int64_t overflow;       /* table lookups above the table range */
    int64_t steps_done;     /* time steps since init */
    int64_t n_alive;        /* live particles now */
    int64_t inject_starved; /* injections skipped for lack of free slots */
} emc_obs;

/* Tally kinds for emc_tally (shapes per context with E ensembles, C cells;
 * C = 1 for bulk): */
enum {
    EMC_TALLY_OBS = 0,       /* emc_obs[E] */
    EMC_TALLY_EVENTS = 1,    /* uint64[E][3][10] real scattering events (valley before the
                                event, mechanism), summed over the subcells */
    EMC_TALLY_HEAT = 2,      /* int64[E][C][2] net phonon emissions (emitted - absorbed) per
                                subcell: [.][0] polar optical, [.][1] intervalley (from the
                                per-subcell event counts of EMC_TALLY_EVENTS_CELL) */
    EMC_TALLY_CHARGE = 3,    /* int64[E][C] electrons per subcell at the last Poisson update
                                (bulk: live electrons) */
    EMC_TALLY_CROSSINGS = 4, /* int64[E][4] source out, drain out, source in, drain in */
    EMC_TALLY_PHI = 5,       /* double[E][C] potential, V */
    EMC_TALLY_FIELD = 6,     /* double[E][C][3] field, V/m */
    EMC_TALLY_HEAT_J = 7,    /* double[E][C] net energy emitted to phonons per subcell, J
                                (superparticle weight included) */
    EMC_TALLY_EVENTS_CELL = 8 /* uint64[E][C][3][10] real scattering events per subcell (the
                                subcell where the electron scattered; valley before the
                                event, mechanism); bulk: C = 1.  The electron counts of
                                the subcells that feed the Poisson update and the energy
                                exchange with phonons counted per subcell (the Poisson
                                and heat-generation passages next to Table I) */
};

/* Create a context holding one ensemble (emc_batch_init with n_ens = 1).
 * Builds the FP64 rate tables, draws the initial Kane-Maxwellian ensemble
 * from Philox key (seed, particle id), and for the nanowire assembles the
 * Poisson operator and solves for the initial field.  cuda_stream is a
 * cudaStream_t (NULL = default stream).  *out receives the context. */
emc_status emc_init(const emc_config* cfg, void* cuda_stream, emc_ctx** out);

/* Create a context holding n_ens independent ensembles (bias points,
 * temperatures, dopings, sizes) simulated together by every launch. */
emc_status emc_batch_init(const emc_config* cfgs, int32_t n_ens, void* cuda_stream, emc_ctx** out);

/* Advance every ensemble by n_steps time steps of dt (asynchronous on the
 * context stream).  Per step and particle: free flight under the field with
 * Kane dispersion, self-scattering against Gamma0, choice of mechanism and
 * final state, nanowire walls and contacts; tallies are accumulated.  In the
 * nanowire, every steps_per_poisson steps the contact subcells are refilled,
 * the subcell charge is counted and the FP64 Poisson update recomputes the
 * field.  n_steps < 0 is EMC_EINVAL; 0 is a no-op. */
emc_status emc_step(emc_ctx* ctx, int32_t n_steps);

/* Copy tally `kind` (EMC_TALLY_*) of every ensemble into dst (bytes must be
 * at least the size given above; dst_is_device: 1 = device pointer on the
 * context's device, 0 = host).  Synchronises the context stream.  reset = 1
 * zeroes the accumulating tallies (OBS sums and counts except steps_done and
 * n_alive, the event counts and with them EVENTS, HEAT, HEAT_J, CROSSINGS)
 * after the copy.  The first call allocates a small device staging buffer
 * (the largest tally computed on the device). */
emc_status emc_tally(emc_ctx* ctx, int32_t kind, void* dst, size_t bytes,
                     int32_t dst_is_device, int32_t reset);

/* The same tally and reset as emc_tally, enqueued on the context stream
 * without waiting for it: the values are packed on the device (the same
 * conversions) and copied to dst in stream order, after the work enqueued
 * before this call.  For the copy to be asynchronous a host dst must be
 * page-locked (pageable memory makes it synchronous).  dst must stay valid,
 * and must not be read, until the stream has passed the copy: synchronise
 * the stream, or wait on an event recorded on it after this call.  This lets
 * a caller enqueue the next emc_step before reading the previous step's
 * tallies.  The first call allocates a small staging buffer (the largest
 * tally's size).  Device errors of the steps are reported by the next
 * emc_tally, not here. */
emc_status emc_tally_async(emc_ctx* ctx, int32_t kind, void* dst, size_t bytes,
                           int32_t dst_is_device, int32_t reset);

/* FP64 Poisson solve on the context's subcell grid (nanowire only), for
 * ensemble 0 of the context:  div(eps_s eps0 grad phi) = -rho with the
 * Dirichlet terminal faces at bc_volts = {Vs, Vd, Vg}.  charge_or_null: host
 * double[C] charge density in C/m^3, or NULL to use the current subcell
 * electron count (rho = q (Nd - w n / V_cell)).  phi_out_or_null: host
 * double[C] receives phi (V).  Does not change the context's field. */
emc_status poisson_solve(emc_ctx* ctx, const double* charge_or_null,
                         const double* bc_volts, double* phi_out_or_null);

/* Allocation-free variant of poisson_solve (the paper has no counterpart;
 * this entry point exists for callers that must not allocate device memory,
 * e.g. a host that has reserved the whole device for its own pool, or code
 * that runs where allocation is forbidden or must not be recorded).  Same
 * arguments, result and accuracy as poisson_solve, but its temporaries (the
 * right-hand side, the potential, the charge density, the voltages, the
 * residual and the partial sums of the sweep) live in one static device
 * array of about 1.6 MiB owned by the library, so the call performs no
 * cudaMalloc or cudaFree of its own.
 *  - Limit: at most 8192 subcells; larger grids return EMC_EINVAL.
 *  - The first call in a CUDA context looks the array's device address up
 *    (cudaGetSymbolAddress) with that context current and keeps it for
 *    later calls in the same context (a context created anew, e.g. after
 *    cudaDeviceReset, gets a fresh lookup); make that first call before any
 *    stream capture.  The array stays reserved on every device that loaded
 *    the library until the library is unloaded or the context is destroyed.
 *  - All calls share the one array: calls that may overlap on the GPU
 *    (other threads, other streams, other contexts on the same device) race
 *    and must be serialised by the caller.  Each call zeroes the potential
 *    it starts from, so a call never sees the previous call's result. */
emc_status emc_poisson_solve_static(emc_ctx* ctx, const double* charge_or_null,
                                    const double* bc_volts, double* phi_out_or_null);

/* Checkpoint and resume.  emc_get_state copies the whole simulation state
 * of the context into the host buffer dst (synchronises the stream):
 * particle state (wave vector, position, residual flight time, valley and
 * ensemble tag, Philox counter, id), the id->slot map and free-id bitmaps,
 * every accumulating tally, the device error word, the terminal voltages,
 * the potential and field (nanowire), the subcell temperature bins and
 * Gamma0 (once emc_set_temperature was used), the step count and the sort
 * phase.  emc_state_size gives the bytes needed (*bytes).  emc_set_state
 * restores such a blob into a context created from the same ensembles
 * (same emc_config array; the launch-tuning fields block_size,
 * steps_per_launch, table_smem_kb and sort_period may differ); continuing
 * from it gives the run that continuing the saved context would have given.
 * Layout (host byte order, this library version only): a 72-byte header
 * (magic "EMCSTATE", version, precision, geometry, temperature mode,
 * ensembles, subcells, slots, bitmap words, steps done, sort phase,
 * configuration hash), then the arrays in the order listed above, slot
 * order, in the context's precision (the wave vector first: k_x of slot 0
 * starts at byte 72, in 1/nm).  Errors: EMC_EINVAL for a short buffer or a
 * foreign blob, EMC_ESTATE for a blob of other ensembles or without the
 * subcell temperatures this context has. */
emc_status emc_state_size(emc_ctx* ctx, size_t* bytes);
emc_status emc_get_state(emc_ctx* ctx, void* dst, size_t bytes);
emc_status emc_set_state(emc_ctx* ctx, const void* src, size_t bytes);

/* Advance n_ctx (1 or 2) contexts by n_steps time steps together: per chunk
 * one flight launch covers the particles of both (each context on its own
 * blocks of the launch, in proportion to its particle slots), then each
 * nanowire context's contact refill and Poisson update, each context's
 * sort when due; the result is that of emc_step on each (the mixed bulk +
 * nanowire batch, which needs one context per geometry, runs as one launch
 * per chunk).  The chunk is the nanowire contexts' Poisson period (two
 * nanowire contexts need the same period and phase), else the first
 * context's steps_per_launch.  The contexts need the same stream, precision
 * and block size; sharded contexts, and contexts with flight profiling on,
 * step alone.  The one flight launch per chunk is counted on ctxs[0]. */
emc_status emc_group_step(emc_ctx* const* ctxs, int32_t n_ctx, int32_t n_steps);

/* One wire's particles sharded over several contexts (the charge exchange
 * of the Poisson passage: the field of a period follows from the electron
 * count of every subcell, summed over all particles of the wire).  Each
 * context holds a disjoint set of the wire's particle ids (emc_config
 * shard_*; every ensemble of a sharded context is sharded, and a context is
 * either all sharded or not).  Within a Poisson period the shards advance
 * independently; at its end the caller sums the per-subcell counts over the
 * shards (an integer all-reduce) and hands the sum back, and every shard
 * refills the contacts and solves the same FP64 Poisson problem, so all
 * shards hold the same field.  The union of the shards then follows, bit for
 * bit, the run of one unsharded context of the whole wire: the same particle
 * states, integer tallies summed over the shards equal to its tallies.
 *
 * Protocol per shard:
 *   - after emc_init, and after every emc_step that ends a Poisson period,
 *     the context waits for an exchange (emc_step in that state, and
 *     emc_step across the end of a period, are EMC_EINVAL; so are
 *     emc_set_bias(_all), emc_get_state and emc_set_state);
 *   - emc_shard_counts copies the shard's electron count per subcell
 *     (int32[E][C], counted at the end of the period) into charge_out and
 *     its free-id counts into free_out (int64[E][2]: free ids among the
 *     initial-electron ids, and among the spare ids);
 *   - the caller sums charge over the shards (charge_global) and, for each
 *     shard, the free counts of the shards whose id ranges lie below it
 *     (free_prefix[E][2]) and over all shards (free_total[E][2]); shards are
 *     ordered by shard_live_base, whose order must be that of
 *     shard_spare_base;
 *   - emc_shard_tail hands these back: the contact subcells are refilled
 *     with the r-th free id of the whole wire filling the r-th missing
 *     electron (each shard draws the electrons of the free ids it holds),
 *     the charge becomes the wire's count after the refill, and the FP64
 *     Poisson update recomputes the field (after emc_init: no refill, the
 *     initial solve).  lead = 1 on exactly one shard: its count of refills
 *     skipped for lack of free ids is the wire's.
 * Pointers may be host or device memory (copies are in stream order; both
 * calls synchronise the context stream).  Tallies of a shard are its own
 * particles' (sum them over the shards), except EMC_TALLY_CHARGE, PHI and
 * FIELD, which are the wire's on every shard.  Errors: EMC_EINVAL when no
 * exchange is pending or the context is not sharded. */
emc_status emc_shard_counts(emc_ctx* ctx, int32_t* charge_out, int64_t* free_out);
emc_status emc_shard_tail(emc_ctx* ctx, const int32_t* charge_global, const int64_t* free_prefix,
                          const int64_t* free_total, int32_t lead);

/* Lattice temperature per subcell of ensemble ens (nanowire contexts whose
 * ensembles share one material and doping): T_cells[n] in K, n = the
 * subcell count (or 1 for a uniform value).  The phonon feedback of the
 * thermal side on the electrons (the coupling paragraph: the updated local
 * temperature changes the electrons' scattering rates).  Rates
 * are tabulated on temperature bins T_k = 250 K + 5 K k (k = 0..150) and a
 * subcell uses the bin nearest its temperature; a scattering is tried
 * against the ensemble's Gamma0 (the largest total rate over the bins in
 * use) with the table of the particle's current subcell, so self-scattering
 * stays exact across subcells.  Residual flight times are rescaled by
 * Gamma0_old / Gamma0_new.  Contact refills draw thermal electrons at the
 * contact subcell's temperature.  The first call builds the 151 bin tables. */
emc_status emc_set_temperature(emc_ctx* ctx, int32_t ens, const double* T_cells, int32_t n);

/* Set the terminal voltages of ensemble ens and re-solve the fields (the
 * solve is skipped when no voltage changed: the field already belongs to
 * them). */
emc_status emc_set_bias(emc_ctx* ctx, int32_t ens, double Vs, double Vd, double Vg);

/* Set the terminal voltages of every ensemble from host array bias[E][3]
 * ({Vs, Vd, Vg} per ensemble) and re-solve the fields: one host-to-device
 * copy of 24 E bytes (asynchronous if bias is pinned); the solve is skipped
 * when no voltage changed. */
emc_status emc_set_bias_all(emc_ctx* ctx, const double* bias);

/* Kernel timing: with enable = 1 every later flight-kernel launch is
 * bracketed by CUDA events on the context stream; emc_profile_read
 * synchronises and returns the summed flight-kernel time (ms) and launch
 * count since the last enable, and emc_profile(ctx, 0) stops recording. */
emc_status emc_profile(emc_ctx* ctx, int32_t enable);
emc_status emc_profile_read(emc_ctx* ctx, double* flight_ms, int64_t* flight_launches);

/* ------------------------------------------------------------------------
 * Surrogate MLP (the learned part; the paper itself has no surrogate).
 * A fully connected network n_in -> n_hidden (x n_layers, SiLU) -> n_out
 * mapping local conditions to Monte Carlo observables, trained on data the
 * Monte Carlo produces.  Products run on the tensor cores with BF16 operands
 * and FP32 accumulation; master weights and Adam moments are FP32.  Inputs
 * and outputs are normalised inside: x_n = (x - x_shift) / x_scale, the
 * network predicts (y - y_shift) / y_scale.
 * Parameter vector layout (emc_mlp_params): for each layer in order, W
 * (out x in, row-major) then b (out).
 */
typedef struct emc_mlp emc_mlp;

typedef struct emc_mlp_config {
    int32_t n_in;        /* inputs, 1..16 */
    int32_t n_hidden;    /* hidden width, multiple of 16, 16..256 */
    int32_t n_layers;    /* hidden layers, 1..6 */
    int32_t n_out;       /* outputs, 1..16 */
    float x_shift[16], x_scale[16];
    float y_shift[16], y_scale[16];
    uint32_t seed;       /* weight initialisation (uniform +-sqrt(6 / fan_in)) */
    int32_t pad_;
} emc_mlp_config;

typedef struct emc_train_config {
    int64_t steps;       /* optimiser steps */
    int32_t batch;       /* rows per step, sampled with replacement */
    float lr, beta1, beta2, eps;  /* Adam */
    uint32_t seed;       /* minibatch sampling stream */
    int32_t pad_;
} emc_train_config;

emc_status emc_mlp_create(const emc_mlp_config* cfg, void* cuda_stream, emc_mlp** out);
/* Train on the n rows of host arrays X [n][n_in], Y [n][n_out] (mean squared
 * error of the normalised outputs).  loss_history: host float[steps] or NULL. */
emc_status emc_mlp_train(emc_mlp* m, const float* X, const float* Y, int64_t n, const emc_train_config* tc,
                         float* loss_history);
/* Y [n][n_out] = network(X [n][n_in]); host arrays.  By default the whole
 * network runs in one fused tensor-core launch per chunk of rows (every
 * layer's BF16 weights and a 128-row activation tile held in shared memory,
 * the accumulator in tensor memory) when the weights fit in shared memory
 * (about 200 KB with the tile), else one GEMM launch per layer. */
emc_status emc_mlp_infer(emc_mlp* m, const float* X, float* Y, int64_t n);
/* Inference path of emc_mlp_infer: enable = 1 (default) fused when the
 * network fits, 0 one launch per layer.  Both compute the same arithmetic
 * (normalisation, BF16 operands, FP32 accumulation, bias and SiLU in FP32).
 * Errors: EMC_EINVAL for a null handle. */
emc_status emc_mlp_set_fused(emc_mlp* m, int32_t enable);
/* Loss and gradient of the loss w.r.t. the parameter vector on host rows
 * X, Y (no update).  grad: host float[count] (see emc_mlp_params). */
emc_status emc_mlp_grad(emc_mlp* m, const float* X, const float* Y, int64_t n, float* grad, float* loss);
/* Parameter vector: *count receives its length; get (dst != NULL) and/or
 * set (src != NULL, applied after the get). */
emc_status emc_mlp_params(emc_mlp* m, float* dst, const float* src, int64_t* count);
const char* emc_mlp_last_error(const emc_mlp* m);
/* Diagnostic: set the handle's device error word as an expired tensor-core
 * wait sets it, so that the next call that checks it returns EMC_ETIMEOUT
 * (and clears it); lets the reporting path be tested without an expiry. */
emc_status emc_mlp_debug_set_error(emc_mlp* m);
void emc_mlp_destroy(emc_mlp* m);

/* The surrogate attached to a Monte Carlo context (the learned part's calls
 * on the context itself): emc_surrogate_train creates the context's network
 * from `net` on the context's stream (replacing an earlier one) and trains
 * it on the host rows X [n][n_in], Y [n][n_out] exactly as emc_mlp_train;
 * emc_surrogate_infer evaluates it (host arrays, as emc_mlp_infer);
 * emc_surrogate_params reads its parameter vector (layout of
 * emc_mlp_params; dst NULL: *count only).  The network lives until
 * emc_destroy or the next emc_surrogate_train.  EMC_ESTATE: no network
 * trained yet. */
emc_status emc_surrogate_train(emc_ctx* ctx, const emc_mlp_config* net, const float* X, const float* Y, int64_t n,
                               const emc_train_config* tc, float* loss_history);
emc_status emc_surrogate_infer(emc_ctx* ctx, const float* X, float* Y, int64_t n);
emc_status emc_surrogate_params(emc_ctx* ctx, float* dst, int64_t* count);

/* ------------------------------------------------------------------------
 * Thermal side of the electrothermal loop: steady Fourier conduction on the
 * subcell grid with kappa(T) of the paper's phonon model (three identical
 * sine-shaped acoustic branches omega = omega_max sin(pi q / 2 q0), phonon
 * relaxation 1/tau = A omega^4 + B1 omega^2 T exp(-B2/T), Table II) plus a
 * boundary term v_g / L_boundary (the size-modified mean free paths).
 * Contacts (x = 0, x = L) are held at T_sink; the bottom face (z = 0) loses
 * heat to T_sink through h_bottom (W/m^2/K) and, when interface_dmm = 1, the
 * diffuse-mismatch interface of Eqs. (2)-(3) in series; other faces are
 * adiabatic.
 */
typedef struct emc_thermal_config {
    double T_sink;          /* K */
    double h_bottom;        /* W/(m^2 K) */
    double L_boundary;      /* m, boundary-scattering length (0: bulk) */
    double tol_K;           /* Picard stop: max |T_new - T_old| */
    double k0_per_m, omega_max_rad_s, A_s3, B1_s_per_K, B2_K;  /* Table II column */
    /* phonon-electron scattering of Eq. (1), off when n_e_m3 = 0: free
     * electron density (m^-3), their DOS mass / m0, acoustic deformation
     * potential (eV), mass density (kg/m^3), averaged phonon group velocity
     * (m/s); the Fermi level follows from n_e at each temperature */
    double n_e_m3, m_e_rel, Da_eV, rho_kg_m3, vg_e_m_s;
    int32_t max_picard, max_cg;
    /* interface under the bottom face, diffuse mismatch model (Eqs. (2) and
     * (3)), used when interface_dmm = 1: the substrate's column of Table II
     * (its sine branches), and the interface area per unit area of the
     * wire's bottom face (> 0; the heat may spread before it crosses).  The
     * conductance area_ratio / R_K(T), at the temperature of the adjacent
     * subcell, is in series with the half cell and with h_bottom (h_bottom
     * <= 0: no lumped part). */
    int32_t interface_dmm, pad_;
    double sub_k0_per_m, sub_omega_max_rad_s, interface_area_ratio;
} emc_thermal_config;

/* Solve every ensemble of a nanowire context (at most 2048 subcells):
 * q [E][C] heat generation (W/m^3, host), T [E][C] host: initial guess in,
 * solution (K) out.  iters (host int[E][2] or NULL): Picard iterations and
 * total CG iterations per ensemble. */
emc_status emc_thermal_solve(emc_ctx* ctx, const emc_thermal_config* tc, const double* q, double* T,
                             int32_t* iters);
/* kappa(T) (W/m/K) as used by emc_thermal_solve, for n host temperatures. */
emc_status emc_kappa(const emc_thermal_config* tc, const double* T, double* kappa, int32_t n);
/* Diffuse mismatch model between the wire (k0_per_m, omega_max_rad_s of tc)
 * and the substrate (sub_k0_per_m, sub_omega_max_rad_s), three identical
 * sine-shaped acoustic branches each.  emc_dmm_transmissivity: Eq. (2),
 * tau_12(omega) from wire to substrate for n host angular frequencies
 * (rad/s; 0 where the substrate has no states).  emc_interface_conductance:
 * Eq. (3), 1/R_K (W/(m^2 K)) per unit interface area at n host temperatures
 * (K, tabulated in 0.5 K steps from 150 K to 1500 K as used by
 * emc_thermal_solve).  EMC_EINVAL for non-positive dispersion parameters. */
emc_status emc_dmm_transmissivity(const emc_thermal_config* tc, const double* omega, double* tau12, int32_t n);
emc_status emc_interface_conductance(const emc_thermal_config* tc, const double* T, double* G_K, int32_t n);

/* Phonon Monte Carlo of the transistor region (the hybrid-method and
 * coupling paragraphs: the phonon side takes the electrons' per-subcell heat
 * and returns the temperature along the wire).  Energy-based deviational
 * phonon bundles (Peraud and Hadjiconstantinou, 2011) of the phonon model
 * of tc: three identical sine branches of the wire's Table II column,
 * 1/tau = A w^4 + B1 w^2 T exp(-B2/T), plus v_g / L_boundary when
 * L_boundary > 0 and the phonon-electron rate of Eq. (1) when n_e_m3 > 0.
 * The spectrum is split into n_bins equal wave-vector bins of (0, q0); a
 * bundle has one bin, flies at its group velocity and scatters at its rate at
 * the temperature of the subcell it is in (T_cells rounded to whole kelvin);
 * after a scattering it takes a new bin from C(w)/tau(w) and an isotropic
 * direction.  A bundle starts in a subcell with probability proportional
 * to the magnitude of that subcell's heat and carries its sign (negative
 * heat, where the electrons absorb more phonon energy than they emit, is a
 * phonon deficit), with a bin from the same distribution, and ends
 * at an isothermal face or when it crosses an interface face (transmitted
 * with the probability tau_12 of Eq. (2) into the substrate of
 * tc->sub_k0_per_m / sub_omega_max_rad_s, else re-emitted diffusely).  Rough
 * faces reflect specularly with probability p_specular, else diffusely
 * (cosine law); specular faces are the symmetry planes. */
enum { EMC_PH_SPECULAR = 0, EMC_PH_ROUGH = 1, EMC_PH_ISOTHERMAL = 2, EMC_PH_INTERFACE = 3 };

typedef struct emc_phonon_config {
    int32_t n_bins;           /* wave-vector bins (1 .. 65536) */
    int32_t face[6];          /* EMC_PH_* of the faces x = 0, x = Lx, y = 0, y = Ly, z = 0, z = Lz;
                                 at least one isothermal or interface face */
    int32_t precision;        /* EMC_FP32 (production) or EMC_FP64 (parity build) */
    double p_specular[6];     /* EMC_PH_ROUGH faces, in [0, 1] */
    int64_t max_segments;     /* flight segments per bundle (1 .. 1e9); a bundle that
                                 reaches it stops where it is and is counted as capped */
    uint32_t seed;            /* Philox key word 0; word 1 is the bundle id */
    int32_t block_size;       /* threads per block (0 = 256; multiple of 32 up to 256) */
} emc_phonon_config;

typedef struct emc_phonon_tally {
    uint64_t absorbed[6];     /* bundles ended at each face */
    uint64_t segments;        /* flight segments (to a scattering or a subcell face) */
    uint64_t scatterings;
    uint64_t capped;          /* bundles stopped by max_segments */
    double power_W;           /* sum of |q| times the subcell volume (each bundle's
                                 share of it is power_W / n_bundles) */
    double kernel_ms;         /* device time of the Monte Carlo kernel */
} emc_phonon_tally;

/* Steady temperature rise of one wire of a nanowire context (its subcell
 * grid, at most 4096 subcells; the context's stream) for the heat
 * generation q (host double[C], W/m^3, finite, not all zero) carried by
 * n_bundles bundles with ids first .. first + n_bundles - 1 (ids < 2^32).
 * T_cells (host double[C], K, or NULL for tc->T_sink everywhere) sets the
 * temperature of the scattering rates and of the heat capacity.  Outputs
 * (host, NULL to skip): dT[C] = P t_c / (N C_tot(T_c) V_c) in K (P =
 * power_W, t_c the signed residence time of all bundles in subcell c,
 * accumulated in fixed point of 2^-24 ps), t_res_ps[C], scatterings[C],
 * emitted[C] (bundles started per subcell), tally.  Runs of disjoint id
 * ranges add up to the run of their union.  Errors: EMC_EINVAL for a bad
 * configuration or input, EMC_ESTATE for a bulk context. */
emc_status emc_phonon_solve(emc_ctx* ctx, const emc_thermal_config* tc, const emc_phonon_config* pc,
                            const double* q, const double* T_cells, int64_t n_bundles, int64_t first,
                            double* dT, double* t_res_ps, uint64_t* scatterings, uint64_t* emitted,
                            emc_phonon_tally* tally);

/* Diagnostics used by the test-suite. */
/* Philox4x32-10 evaluated on the device for n (counter, key) pairs:
 * ctr[n][4], key[n][2] in, out[n][4] out (host arrays). */
emc_status emc_debug_philox(emc_ctx* ctx, const uint32_t* ctr, const uint32_t* key,
                            uint32_t* out, int32_t n);
/* Particle state in slot order, host arrays of `capacity` rows (total over
 * ensembles): k[.][3] (1/m), r[.][3] (m), tr (s), valley (-1 = no particle),
 * ensemble, id, philox counter. */
emc_status emc_debug_particles(emc_ctx* ctx, double* k, double* r, double* tr,
                               int32_t* valley, int32_t* ens, uint32_t* id, uint64_t* ctr);
/* Rate tables of ensemble ens as built on the device (double[3][n_bins][10],
 * cumulative / Gamma0) and Gamma0 (double[3], 1/s). */
emc_status emc_debug_tables(emc_ctx* ctx, int32_t ens, double* table, double* gamma0);

/* Number of ensembles, total particle slots and subcells of a context. */
emc_status emc_shape(const emc_ctx* ctx, int32_t* n_ens, int64_t* capacity, int32_t* n_cell);

/* Kernel launches issued by this context since init (for accounting). */
int64_t emc_launch_count(const emc_ctx* ctx);

const char* emc_last_error(const emc_ctx* ctx);
void emc_destroy(emc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
