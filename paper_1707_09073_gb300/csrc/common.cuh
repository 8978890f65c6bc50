// Device-side definitions shared by the libemc translation units.
//
// Internal units on the device: length nm, time fs, energy eV, wave vector
// 1/nm.  Rates are 1/fs.  The config arrives in SI and is converted once on
// the host.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace emc {

constexpr int NV = 3;   // Gamma1, U, Gamma3
constexpr int NM = 10;  // mechanisms per valley (see include/emc.h)
constexpr int WE = 32;  // ensembles with shared-memory block tallies (by index)
constexpr uint32_t DEAD = 0xFFu;
constexpr int MAX_FLIGHTS_PER_STEP = 1 << 16;
#ifndef EMC_CHUNK_RUN
#define EMC_CHUNK_RUN 2
#endif
constexpr int kChunkRun = EMC_CHUNK_RUN;  // consecutive 32-slot chunks a warp of the flight kernel takes
// per-subcell lattice temperature: rates tabulated on bins T_k = 250 K + 5 K k
constexpr double TBIN_LO = 250.0, TBIN_DT = 5.0;
constexpr int NTBIN = 151;
constexpr int MAX_INIT_TRIALS = 1000;

// CODATA 2018 (SI)
constexpr double kQ = 1.602176634e-19;
constexpr double kHbar = 1.054571817e-34;
constexpr double kKB = 1.380649e-23;
constexpr double kM0 = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;
// derived, in nm / fs / eV
constexpr double kHbarEVfs = kHbar / kQ * 1e15;               // hbar, eV fs
constexpr double kCk0 = kHbar * kHbar / (2.0 * kM0) / kQ * 1e18; // hbar^2/2m0, eV nm^2
constexpr double kVk0 = kHbar / kM0 * 1e3;                    // hbar/m0, nm^2/fs
constexpr double kE2Eps0 = kQ / kEps0 * 1e9;                  // e^2/eps0, eV nm (= q/eps0 in V nm)

// error word bits (device -> host)
enum : int { ERR_FLIGHTS = 1, ERR_NAN = 2, ERR_INIT = 4, ERR_BOUNDS = 8 };

// The checked build (compiled with EMC_CHECKED) verifies array indices and
// positions in the kernels and sets ERR_BOUNDS in the device error word
// when one is out of range; the production build compiles the checks away.
#ifdef EMC_CHECKED
#define EMC_CHECK(err, cond)                            \
    do {                                                \
        if (!(cond)) atomicOr((err), (int)ERR_BOUNDS);  \
    } while (0)
#else
#define EMC_CHECK(err, cond) \
    do {                     \
    } while (0)
#endif

// Final-state physics of one table set, in device units.
template <typename Real>
struct Phys {
    Real ck[NV];      // hbar^2 / 2m_v  (gamma = ck k^2), eV nm^2
    Real vk[NV];      // hbar / m_v, nm^2/fs
    Real alpha[NV];   // 1/eV
    Real Ec[NV];      // eV
    Real inv_g0[NV];  // 1 / Gamma0, fs
    Real hw_lo, hw_iv;
    Real beta2;       // Debye screening wave vector^2, 1/nm^2
    Real kT, emax_init, hmax0;  // initial Kane-Maxwellian of valley 0
};

// Everything a kernel needs, passed by value.  Real-typed arrays are void*
// and cast by the templated kernels.
struct DevParams {
    // particle SoA (slot order)
    void *kx, *ky, *kz, *x, *y, *z, *tr;
    uint32_t* tag;  // (ensemble << 8) | valley, valley DEAD = no particle
    uint64_t* ctr;  // Philox counter of the particle's stream
    uint32_t* id;   // particle id within its ensemble's slots (local id)
    int64_t n_slots;
    // per ensemble
    int32_t n_ens;
    const int64_t* ens_off;   // first slot (and first id-indexed row) of ensemble e
    const int64_t* ens_cap;   // slots of ensemble e
    const int64_t* ens_n0;    // initial particles of ensemble e
    const uint32_t* seed;
    const int32_t* tabset;
    const void* acc_bulk;     // Real[E][4]: dk/dt under the uniform field, 1/(nm fs); 4th unused
    const void* acc_cell;     // Real[E][C][4]: dk/dt per subcell and 1/(hbar |dk/dt|)
    const int32_t* n_target;  // contact-cell refill target per ensemble
    // global particle ids (the Philox key word 1): local id i < n0 is global
    // id gid[e][0] + i, a spare local id i >= n0 is gid[e][1] + i - n0
    // (unsharded: {0, n0}, the global id is the local id)
    const uint32_t* ens_gid;  // [E][2]
    // sharded contexts: per ensemble {free ids of the lower shards among the
    // initial-electron ids, among the spare ids, the wire's free initial-
    // electron ids, the wire's free spare ids, lead shard}; null: unsharded
    const long long* shard;   // [E][5]
    uint32_t* slot_of_id;     // [total slots] global slot of (ensemble, id)
    uint32_t* dead_bits;      // per-ensemble bitmaps of free ids
    const int64_t* bits_off;  // word offset of ensemble e's bitmap
    // tables
    const void* table;        // Real[TS][NV][NB][NM] cumulative rate / Gamma0
    const void* phys;         // Phys<Real>[TS]
    int32_t n_tab, nb, nb_smem;
    double inv_dE;            // 1/eV
    // geometry (nm)
    int32_t nx, ny, nz, ncell;
    double Lx, Ly, Lz, dx, dy, dz, p_spec;
    double dt;                // fs
    // tallies (accumulating)
    unsigned long long* events;   // [E][C][NV][NM] real events per subcell (bulk: C = 1)
    unsigned long long* cnt;      // [E][NCNT]
    double* sums;                 // [E][NSUM]
    int* charge;                  // [E][C]
    long long* alive;             // [E] live particles (never reset)
    // per-subcell temperature (null cell_bin: one temperature per ensemble)
    const int32_t* cell_bin;      // [E][C] temperature bin of each subcell
    const void* bin_table;        // Real[NTBIN][NV][NB][NM], cumulative / Gamma0 of the bin
    const void* bin_phys;         // Phys<Real>[NTBIN]
    const void* ens_g0;           // Real[E][NV]: Gamma0 of the ensemble (1/fs)
    const void* ens_ig0;          // Real[E][NV]: its inverse (fs)
    int* err;
};

enum { CNT_SAMPLES = 0, CNT_V0 = 1, CNT_SELF0 = 4, CNT_OVERFLOW = 7, CNT_REJECT = 8,
       CNT_SRC_OUT = 9, CNT_DRN_OUT = 10, CNT_SRC_IN = 11, CNT_DRN_IN = 12, CNT_STARVED = 13,
       NCNT = 16 };
enum { SUM_VX = 0, SUM_VY, SUM_VZ, SUM_E, SUM_ETOT, NSUM = 8 };

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64 bit multiplies by fixed odd constants; the high halves are xored with
// the other two words and the key, the low halves move to the odd slots; the
// two key words advance by the golden-ratio and sqrt(3)-1 Weyl constants
// between rounds.
struct U4 {
    uint32_t a, b, c, d;
};

__host__ __device__ __forceinline__ U4 philox10(U4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = 0xD2511F53ull * x.a;
        const uint64_t p1 = 0xCD9E8D57ull * x.c;
        U4 y;
        y.a = uint32_t(p1 >> 32) ^ x.b ^ k0;
        y.b = uint32_t(p1);
        y.c = uint32_t(p0 >> 32) ^ x.d ^ k1;
        y.d = uint32_t(p0);
        x = y;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

// (2 (x >> 9) + 1) / 2^24: an exact odd multiple of 2^-24 in (0, 1).
template <typename Real>
__host__ __device__ __forceinline__ Real u01(uint32_t x)
{
    return Real(2u * (x >> 9) + 1u) * Real(5.9604644775390625e-08);
}
// The same number without an integer-to-float conversion: the top 23 bits
// as the mantissa of a float in [1, 2), minus 1 (exact), plus 2^-24 (exact:
// the sum has 24 significant bits).
template <>
__host__ __device__ __forceinline__ float u01<float>(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return (__uint_as_float(0x3F800000u | (x >> 9)) - 1.0f) + 5.9604644775390625e-08f;
#else
    return float(2u * (x >> 9) + 1u) * 5.9604644775390625e-08f;
#endif
}

}  // namespace emc
