// Templated particle kernels of libemc: the fused flight/scatter step, the
// initial ensemble, and the contact re-injection.  Real = float is the
// production path, Real = double the parity build.
//
// Method (Hao et al., arXiv:1707.09073; the hybrid-method and electron-model
// paragraphs, Table I): every electron is tracked
// through free flights under the local field with the Kane dispersion
// E(1 + aE) = hbar^2 k^2 / 2m, interrupted by scatterings chosen against a
// constant total rate Gamma0 per valley (self-scattering fills the gap to the
// real rates); the subcells count electrons for the Poisson update and the
// net energy handed to phonons.
#pragma once
#include <map>
#include <type_traits>
#include <mutex>

#include "common.cuh"

namespace emc {

// ------------------------------------------------------------- math
// The float build compiles with approximate division and square root
// (-prec-div=false -prec-sqrt=false); logarithm and sine/cosine go to the
// special-function unit with the argument kept in its accurate range.
template <typename Real>
struct Mth;
template <>
struct Mth<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    // -ln(u) of a uniform in (0,1) for a flight time: never negative
    static __device__ __forceinline__ float neglog_u(float u) { return fmaxf(0.f, -__logf(u)); }
    // hardware log2 approximation: the FP32 build's angles need no more
    static __device__ __forceinline__ float pow_(float b, float e) { return exp2f(e * __log2f(b)); }
    static __device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
    // sin and cos of 2 pi u, u in (0,1): evaluated at 2 pi (u - 1/2) in (-pi, pi)
    // where the hardware approximation is accurate, then negated
    static __device__ __forceinline__ void sincos2pi_u(float u, float* s, float* c)
    {
        float ss, cc;
        __sincosf(6.283185307179586f * (u - 0.5f), &ss, &cc);
        *s = -ss;
        *c = -cc;
    }
    static __device__ __forceinline__ float cospi_(float x) { return cospif(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    // floor straight to an integer (one conversion; saturates, NaN -> 0)
    static __device__ __forceinline__ int floor_i(float x) { return __float2int_rd(x); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float copysign_(float a, float b) { return copysignf(a, b); }
};
template <>
struct Mth<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double neglog_u(double u) { return -log(u); }
    static __device__ __forceinline__ double pow_(double b, double e) { return pow(b, e); }
    static __device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }
    static __device__ __forceinline__ void sincos2pi_u(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
    static __device__ __forceinline__ double cospi_(double x) { return cospi(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ int floor_i(double x) { return __double2int_rd(x); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double copysign_(double a, double b) { return copysign(a, b); }
};

// Fused multiply-add, written out so that every kernel that inlines the
// particle arithmetic rounds it the same way (the compiler may otherwise fuse
// a*b + c*d either way round, differently in different kernels).
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Kinetic energy whose Kane gamma is g: the positive root of E(1 + aE) = g,
// written as 2g / (1 + sqrt(1 + 4ag)) (exact for a = 0, no cancellation).
template <typename Real>
__device__ __forceinline__ Real kane_E(Real g, Real a)
{
    return Real(2) * g / (Real(1) + Mth<Real>::sqrt_(fma_(Real(4) * a, g, Real(1))));
}

// The same energy and s = sqrt(1 + 4ag), which equals 1 + 2aE (the group
// velocity's denominator): the float build takes it from here instead of
// forming 1 + 2aE again.
template <typename Real>
__device__ __forceinline__ Real kane_E_s(Real g, Real a, Real& s)
{
    s = Mth<Real>::sqrt_(fma_(Real(4) * a, g, Real(1)));
    return Real(2) * g / (Real(1) + s);
}

// |k|^2
template <typename Real>
__device__ __forceinline__ Real norm2(Real x, Real y, Real z)
{
    return fma_(z, z, fma_(y, y, x * x));
}

// Compensated (Kahan) accumulator for the float build; plain sum for double.
template <typename Real>
struct Acc {
    Real s = 0, c = 0;
    __device__ __forceinline__ void add(Real x)
    {
        Real y = x - c;
        Real t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
    __device__ __forceinline__ Real comp() const { return c; }
    __device__ __forceinline__ void clear() { s = c = 0; }
};
template <>
struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ double comp() const { return 0.0; }
    __device__ __forceinline__ void clear() { s = 0; }
};

// Launch constants in the kernel's own precision (no conversions in the loop).
template <typename Real>
struct KConst {
    Real Lx, Ly, Lz, inv_dx, inv_dy, inv_dz, p_spec, dt, inv_dE;
    int nx, ny, nz, ncell, nb, nbs, n_tab, n_tab_s;
    int64_t per_block;
    int* err;  // device error word (checked build)
};

// Shared-memory tallies of the ensembles [e_base, e_base + WE) of a block.
struct BlockTally {
    unsigned int ev[WE][NV * NM];
    unsigned int cnt[WE][NCNT];
    double sums[WE][NSUM];
};

__device__ __forceinline__ void tally_cnt(BlockTally* bt, const DevParams& P, int e, int e_base,
                                          int idx, unsigned int n)
{
    const int w = e - e_base;
    if (w >= 0 && w < WE) {
        atomicAdd(&bt->cnt[w][idx], n);
    } else {
        atomicAdd(&P.cnt[(size_t)e * NCNT + idx], (unsigned long long)n);
        if (idx == CNT_SRC_OUT || idx == CNT_DRN_OUT)
            atomicAdd(reinterpret_cast<unsigned long long*>(&P.alive[e]), (unsigned long long)(-(long long)n));
    }
}

// Increment of base[idx] by the lanes currently executing together: lanes
// with the same counter (particles of one subcell after sorting, scattering
// by the same mechanism) are counted together and one of them issues the
// atomic.
__device__ __forceinline__ void agg_inc_u64(unsigned long long* base, unsigned long long idx)
{
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(base + idx, (unsigned long long)__popc(peers));
}

__device__ __forceinline__ void agg_add_i(int* base, int key)
{
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(base + key, __popc(peers));
}

// ------------------------------------------------------------ particle
template <typename Real>
struct Part {
    Real kx, ky, kz, x, y, z, tr, E;  // E: kinetic energy of k, carried along
    Real f;                           // hbar/(m(1 + 2 alpha E)): v = f k, carried with E
    uint64_t ctr;
    uint32_t id, seed;
    int v, e;

    __device__ __forceinline__ U4 draw()
    {
        U4 c{uint32_t(ctr), uint32_t(ctr >> 32), 0u, 0u};
        ++ctr;
        return philox10(c, seed, id);
    }
};

// global id (Philox key word 1) of local id i of ensemble e
__device__ __forceinline__ uint32_t gid_of(const DevParams& P, int e, uint32_t i)
{
    const uint32_t n0 = uint32_t(P.ens_n0[e]);
    return i < n0 ? P.ens_gid[2 * e] + i : P.ens_gid[2 * e + 1] + (i - n0);
}

template <typename Real>
__device__ __forceinline__ int cell_of(const KConst<Real>& K, Real x, Real y, Real z)
{
    // floor of the scaled coordinate, converted straight to an integer (a
    // NaN converts to 0 and lands in subcell 0, an overflow saturates)
    const int fx = Mth<Real>::floor_i(x * K.inv_dx);
    const int fy = Mth<Real>::floor_i(y * K.inv_dy);
    const int fz = Mth<Real>::floor_i(z * K.inv_dz);
    // a position on a far face belongs to the last subcell; anything further
    // out, or not a number, is a bug (checked build)
    EMC_CHECK(K.err, fx >= 0 && fx <= K.nx && fy >= 0 && fy <= K.ny && fz >= 0 && fz <= K.nz && x == x && y == y &&
                         z == z);
    const int ix = min(max(fx, 0), K.nx - 1);
    const int iy = min(max(fy, 0), K.ny - 1);
    const int iz = min(max(fz, 0), K.nz - 1);
    return (ix * K.ny + iy) * K.nz + iz;
}

template <typename Real>
__device__ __forceinline__ void load4(const Real* p, Real o[4]);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float o[4])
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double o[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// u3 h(Emax) <= h(E), h(E) = sqrt(1 + aE)(1 + 2aE), E <= Emax.
template <typename Real>
__device__ Real draw_maxwell(Part<Real>& q, const Phys<Real>* ph, int* err)
{
    const Real a = ph->alpha[0], kT = ph->kT, Emax = ph->emax_init, hmax = ph->hmax0;
    Real E = 0;
    for (int t = 0; t < MAX_INIT_TRIALS; ++t) {
        U4 r = q.draw();
        Real c = Mth<Real>::cospi_(Real(0.5) * u01<Real>(r.c));
        E = -kT * (Mth<Real>::log_(u01<Real>(r.a)) + Mth<Real>::log_(u01<Real>(r.b)) * c * c);
        if (E <= Emax &&
            u01<Real>(r.d) * hmax <= Mth<Real>::sqrt_(Real(1) + a * E) * (Real(1) + Real(2) * a * E))
            return E;
    }
    atomicOr(err, ERR_INIT);
    return E < Emax ? E : Emax;
}

// A thermal electron in valley 0: energy, isotropic direction, a uniform
// position in the box lo + [0, len) (nanowire), then the first flight time.
template <typename Real, bool NW>
__device__ void new_electron(Part<Real>& q, const Phys<Real>* ph, const Real lo[3], const Real len[3], int* err)
{
    q.v = 0;
    Real E = draw_maxwell(q, ph, err);
    Real km = Mth<Real>::sqrt_(E * (Real(1) + ph->alpha[0] * E) / ph->ck[0]);
    U4 r = q.draw();
    Real ct = Real(1) - Real(2) * u01<Real>(r.a);
    Real st = Mth<Real>::sqrt_(Mth<Real>::max_(Real(0), fma_(-ct, ct, Real(1))));
    Real sp, cp;
    Mth<Real>::sincospi_(Real(2) * u01<Real>(r.b), &sp, &cp);
    q.kx = km * st * cp;
    q.ky = km * st * sp;
    q.kz = km * ct;
    if (NW) {
        r = q.draw();
        q.x = lo[0] + u01<Real>(r.a) * len[0];
        q.y = lo[1] + u01<Real>(r.b) * len[1];
        q.z = lo[2] + u01<Real>(r.c) * len[2];
    } else {
        q.x = q.y = q.z = Real(0);
    }
    r = q.draw();
    q.tr = -Mth<Real>::log_(u01<Real>(r.a)) * ph->inv_g0[0];
}

template <typename Real>
__device__ __forceinline__ void store(const DevParams& P, int64_t s, const Part<Real>& q, bool NW)
{
    static_cast<Real*>(P.kx)[s] = q.kx;
    static_cast<Real*>(P.ky)[s] = q.ky;
    static_cast<Real*>(P.kz)[s] = q.kz;
    if (NW) {
        static_cast<Real*>(P.x)[s] = q.x;
        static_cast<Real*>(P.y)[s] = q.y;
        static_cast<Real*>(P.z)[s] = q.z;
    }
    static_cast<Real*>(P.tr)[s] = q.tr;
    P.ctr[s] = q.ctr;
}
// --------------------------------------------------------- free flight
// k advances linearly (hbar dk/dt = force = hbar a); the carried energy is
// updated.  In the nanowire the position moves along the force by the energy
// gained over the force (exact for any band) and across it by the mean of the
// start and end group velocities times t.  f4 = (a_x, a_y, a_z, 1/(hbar |a|)).
template <typename Real, bool NW>
__device__ __forceinline__ void drift(Part<Real>& q, const Phys<Real>& ph, const Real f4[4], Real t)
{
    const Real k0x = q.kx, k0y = q.ky, k0z = q.kz;
    q.kx = fma_(f4[0], t, k0x);
    q.ky = fma_(f4[1], t, k0y);
    q.kz = fma_(f4[2], t, k0z);
    const int v = q.v;
    const Real al = ph.alpha[v];
    const Real E0 = q.E;
    Real s1;
    const Real E1 = kane_E_s(ph.ck[v] * norm2(q.kx, q.ky, q.kz), al, s1);
    q.E = E1;
    // the parity build forms 1 + 2 alpha E as the oracle does
    const Real f1 = ph.vk[v] / (std::is_same<Real, float>::value ? s1 : fma_(Real(2) * al, E1, Real(1)));
    if (NW) {
        const Real f0 = q.f;
        const Real h = Real(0.5) * t;
        Real dx = h * fma_(f0, k0x, f1 * q.kx);
        Real dy = h * fma_(f0, k0y, f1 * q.ky);
        Real dz = h * fma_(f0, k0z, f1 * q.kz);
        const Real ihF = f4[3];
        if (ihF > Real(0)) {
            const Real s = Real(kHbarEVfs) * ihF;  // 1/|a|
            const Real ax = f4[0] * s, ay = f4[1] * s, az = f4[2] * s;
            const Real d = fma_(E1 - E0, ihF, -fma_(dz, az, fma_(dy, ay, dx * ax)));
            dx = fma_(d, ax, dx);
            dy = fma_(d, ay, dy);
            dz = fma_(d, az, dz);
        }
        q.x += dx;
        q.y += dy;
        q.z += dz;
    }
    q.f = f1;
}

// ------------------------------------------------------------- walls
// Contacts absorb at x < 0 (source) and x > Lx (drain).  Plane A (y = 0) is a
// symmetry plane: always specular.  The outer side (y = Ly), bottom and top
// walls reflect specularly with probability p, else diffusely with a
// cosine-weighted inward direction and |k| kept.  Returns true if absorbed.
template <typename Real>
__device__ __forceinline__ void diffuse(Part<Real>& q, int axis, Real sn, U4 r)
{
    const Real km = Mth<Real>::sqrt_(norm2(q.kx, q.ky, q.kz));
    const Real u1 = u01<Real>(r.b);
    const Real ca = Mth<Real>::sqrt_(u1), sa = Mth<Real>::sqrt_(Real(1) - u1);
    Real sp, cp;
    Mth<Real>::sincos2pi_u(u01<Real>(r.c), &sp, &cp);
    q.kx = km * sa * cp;
    if (axis == 1) {
        q.ky = km * sn * ca;
        q.kz = km * sa * sp;
    } else {
        q.ky = km * sa * sp;
        q.kz = km * sn * ca;
    }
}

template <typename Real>
__device__ __forceinline__ bool walls(Part<Real>& q, const DevParams& P, const KConst<Real>& K, BlockTally* bt,
                                      int e_base)
{
    int out = -1;
    if (q.x < Real(0)) out = CNT_SRC_OUT;
    else if (q.x > K.Lx) out = CNT_DRN_OUT;
    if (out >= 0) {
        tally_cnt(bt, P, q.e, e_base, out, 1u);
        return true;  // the caller frees the id
    }
    // a reflected coordinate is kept inside the box (a position that was
    // inside needs no clamp)
    if (q.y < Real(0)) {
        q.y = -q.y;
        q.y = q.y > K.Ly ? K.Ly : q.y;
        q.ky = -q.ky;
    } else if (q.y > K.Ly) {
        q.y = Real(2) * K.Ly - q.y;
        q.y = q.y < Real(0) ? Real(0) : q.y;
        const U4 r = q.draw();
        if (u01<Real>(r.a) < K.p_spec) q.ky = -q.ky;
        else diffuse(q, 1, Real(-1), r);
    }
    if (q.z < Real(0)) {
        q.z = -q.z;
        q.z = q.z > K.Lz ? K.Lz : q.z;
        const U4 r = q.draw();
        if (u01<Real>(r.a) < K.p_spec) q.kz = -q.kz;
        else diffuse(q, 2, Real(1), r);
    } else if (q.z > K.Lz) {
        q.z = Real(2) * K.Lz - q.z;
        q.z = q.z < Real(0) ? Real(0) : q.z;
        const U4 r = q.draw();
        if (u01<Real>(r.a) < K.p_spec) q.kz = -q.kz;
        else diffuse(q, 2, Real(-1), r);
    }
    return false;
}

// ----------------------------------------------------------- scatter
// One Philox call per scattering: u0 picks the mechanism against the
// cumulative table row of the current energy bin (lower bin edge; above the
// last entry = self-scattering), u2/u3 the final direction, u1 the next
// flight time -ln(u1)/Gamma0 of the final valley.  Split in two: the
// mechanism choice runs for every scattering, the final state only for real
// ones (the words of u2/u3 are kept raw until then).

// A scattering in progress: the particle plus the draws of its Philox call.
template <typename Real>
struct QEntry {
    Part<Real> q;
    Real u1;
    uint32_t r2, r3;  // Philox words of the final-state uniforms (converted only for real scatterings)
    Real beta2;          // screening of the subcell's temperature
    const Real* ig0;     // 1/Gamma0 per valley used for the next flight time
    int mech;
};

// Mechanism choice.  Returns the mechanism (-1: self-scattering, whose next
// flight time is set here).
template <typename Real>
__device__ __forceinline__ int choose(QEntry<Real>& Q, const DevParams& P, const KConst<Real>& K, const Phys<Real>& ph,
                                      const Real* tab_s, int nbs, const Real* tab_g, BlockTally* bt, int e_base)
{
    Part<Real>& q = Q.q;
    const U4 r = q.draw();
    Real u0 = u01<Real>(r.a);
    Q.u1 = u01<Real>(r.b);
    Q.r2 = r.c;
    Q.r3 = r.d;
    const int v = q.v;
    const Real E = q.E;
    Q.beta2 = ph.beta2;
    Q.ig0 = ph.inv_g0;
    int bn = -1;
    if (P.cell_bin) {
        // per-subcell temperature: the table of the subcell's temperature bin,
        // tried against the ensemble's Gamma0 (u0 Gamma0_ens / Gamma0_bin)
        bn = P.cell_bin[(size_t)q.e * K.ncell + cell_of<Real>(K, q.x, q.y, q.z)];
        const Phys<Real>& pb = static_cast<const Phys<Real>*>(P.bin_phys)[bn];
        Q.ig0 = static_cast<const Real*>(P.ens_ig0) + (size_t)q.e * NV;
        u0 = u0 * static_cast<const Real*>(P.ens_g0)[(size_t)q.e * NV + v] * pb.inv_g0[v];
        Q.beta2 = pb.beta2;
    }
    const int fb = Mth<Real>::floor_i(E * K.inv_dE);  // a NaN converts to 0: caught below
    int b;
    if (fb >= K.nb) {
        b = K.nb - 1;
        tally_cnt(bt, P, q.e, e_base, CNT_OVERFLOW, 1u);
    } else {
        b = fb >= 0 ? fb : 0;
    }
    if (!(E == E)) atomicOr(P.err, ERR_NAN);
    const Real* row = (bn >= 0) ? static_cast<const Real*>(P.bin_table) + (((size_t)bn * NV + v) * K.nb + b) * NM
                    : (b < nbs) ? tab_s + ((size_t)v * nbs + b) * NM : tab_g + ((size_t)v * K.nb + b) * NM;
    int mech = -1;
    if (u0 < row[NM - 1]) {
        // the row (NM = 10 entries) as five aligned pairs
        using V2 = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
        const V2* r2 = reinterpret_cast<const V2*>(row);
        int cnt = 0;
#pragma unroll
        for (int m = 0; m < NM / 2; ++m) {
            const V2 pr = r2[m];
            cnt += (pr.x <= u0) + (pr.y <= u0);
        }
        mech = cnt;
    }
    if (mech >= 0) {
        // final energy; a channel that cannot conserve energy counts as self
        Real Ep;
        if (mech == 0 || mech == 3) Ep = E;
        else if (mech == 1) Ep = E + ph.hw_lo;
        else if (mech == 2) Ep = E - ph.hw_lo;
        else {
            const int j = (mech - 4) >> 1;
            Ep = E + ((mech & 1) == 0 ? ph.hw_iv : -ph.hw_iv) - (ph.Ec[j] - ph.Ec[v]);
        }
        if (!(Ep > Real(0))) {
            tally_cnt(bt, P, q.e, e_base, CNT_REJECT, 1u);
            mech = -1;
        }
    }
    if (mech < 0) {
        tally_cnt(bt, P, q.e, e_base, CNT_SELF0 + v, 1u);
        q.tr = Mth<Real>::neglog_u(Q.u1) * Q.ig0[v];
    }
    Q.mech = mech;
    return mech;
}

// Final state of a real scattering (mech >= 0) and the next flight time.
template <typename Real, bool NW>
__device__ __forceinline__ void final_state(QEntry<Real>& Q, const DevParams& P, const KConst<Real>& K,
                                            const Phys<Real>& ph, BlockTally* bt, int e_base)
{
    Part<Real>& q = Q.q;
    const int mech = Q.mech, v = q.v;
    const Real E = q.E, u2 = u01<Real>(Q.r2);
    int j = v;
    Real Ep;
    if (mech == 0 || mech == 3) {
        Ep = E;
    } else if (mech == 1) {
        Ep = E + ph.hw_lo;
    } else if (mech == 2) {
        Ep = E - ph.hw_lo;
    } else {
        j = (mech - 4) >> 1;
        Ep = E + ((mech & 1) == 0 ? ph.hw_iv : -ph.hw_iv) - (ph.Ec[j] - ph.Ec[v]);
    }
    const Real k2 = norm2(q.kx, q.ky, q.kz);
    const Real km = Mth<Real>::sqrt_(k2);
    const Real kp = Mth<Real>::sqrt_(Ep * fma_(ph.alpha[j], Ep, Real(1)) / ph.ck[j]);
    Real ct;
    bool rel = true;
    if (mech == 0) {
        // Brooks-Herring: P(cos) ~ 1 / (2k^2 (1 - cos) + beta^2)^2
        ct = Real(1) - Real(2) * u2 / (Real(1) + Real(4) * k2 * (Real(1) - u2) / Q.beta2);
    } else if (mech <= 2) {
        // Froehlich: P(cos) ~ 1 / (k^2 + k'^2 - 2 k k' cos)
        const Real d = km - kp;
        const Real xi = Real(2) * km * kp / (d * d);
        ct = (xi >= Real(1e-6)) ? ((Real(1) + xi) - Mth<Real>::pow_(Real(1) + Real(2) * xi, u2)) / xi
                                : Real(1) - Real(2) * u2;
    } else {
        ct = Real(1) - Real(2) * u2;  // isotropic
        rel = false;
    }
    Real sp, cp;
    Mth<Real>::sincos2pi_u(u01<Real>(Q.r3), &sp, &cp);
    const Real st = Mth<Real>::sqrt_(Mth<Real>::max_(Real(0), fma_(-ct, ct, Real(1))));
    Real dx, dy, dz;
    if (rel) {
        // frame of k: branchless orthonormal basis (Duff et al., JCGT 2017)
        Real nx = 0, ny = 0, nz = 1;
        if (km > Real(0)) {
            const Real ik = Real(1) / km;
            nx = q.kx * ik;
            ny = q.ky * ik;
            nz = q.kz * ik;
        }
        const Real sg = Mth<Real>::copysign_(Real(1), nz);
        const Real aa = Real(-1) / (sg + nz);
        const Real bb = nx * ny * aa;
        const Real e1x = fma_(sg * nx * nx, aa, Real(1)), e1y = sg * bb, e1z = -sg * nx;
        const Real e2x = bb, e2y = fma_(ny * ny, aa, sg), e2z = -ny;
        const Real sc = st * cp, ss = st * sp;
        dx = fma_(ct, nx, fma_(ss, e2x, sc * e1x));
        dy = fma_(ct, ny, fma_(ss, e2y, sc * e1y));
        dz = fma_(ct, nz, fma_(ss, e2z, sc * e1z));
    } else {
        dx = st * cp;
        dy = st * sp;
        dz = ct;
    }
    q.kx = kp * dx;
    q.ky = kp * dy;
    q.kz = kp * dz;
    q.E = Ep;
    q.f = ph.vk[j] / fma_(Real(2) * ph.alpha[j], Ep, Real(1));
    if (NW) {
        // real events per (subcell, valley, mechanism): the subcell heat map
        // (net phonon emission) and the mechanism statistics both follow
        const int c = cell_of<Real>(K, q.x, q.y, q.z);
        EMC_CHECK(P.err, q.e >= 0 && q.e < P.n_ens && c >= 0 && c < K.ncell && v >= 0 && v < NV && mech >= 0 &&
                             mech < NM);
        agg_inc_u64(P.events, ((unsigned long long)q.e * K.ncell + c) * (NV * NM) + v * NM + mech);
    } else {
        const int w = q.e - e_base;
        if (w >= 0 && w < WE)
            atomicAdd(&bt->ev[w][v * NM + mech], 1u);
        else
            atomicAdd(&P.events[((size_t)q.e * NV + v) * NM + mech], 1ull);
    }
    q.v = j;
    q.tr = Mth<Real>::neglog_u(Q.u1) * Q.ig0[j];
}

// Per-thread samples of one ensemble.  When threads move on to another
// ensemble, the warp flushes them together: the threads holding the same
// ensemble are summed across the warp (float tree of the compensated sums,
// integer warp reduction of the counts) and one of them adds the result to
// the block window (or global memory), so no two lanes of a warp contend for
// one tally word.
template <typename Real>
__device__ __forceinline__ Real warp_sum(Real x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <typename Real>
struct Samples {
    Acc<Real> v[3], E, Et;
    // particle-steps per valley, 21 bits each (a lane flushes long before
    // 2^21 of them: at every change of ensemble and at the end of a launch)
    unsigned long long nv = 0ull;
    int e = -1;

    __device__ __forceinline__ void count_valley(int vv, unsigned int n) { nv += (unsigned long long)n << (21 * vv); }
    __device__ __forceinline__ unsigned int nvalley(int vv) const { return unsigned((nv >> (21 * vv)) & 0x1FFFFFull); }

    // Called by all 32 lanes of the warp; lanes with `need` set hand over
    // their samples and counts and start afresh.
    __device__ __forceinline__ void flush_warp(const DevParams& P, BlockTally* bt, int e_base, bool need)
    {
        const bool mine = need && e >= 0 && nv != 0ull;
        unsigned pending = __ballot_sync(0xffffffffu, mine);
        while (pending) {
            const int key = __shfl_sync(0xffffffffu, e, __ffs(pending) - 1);
            const bool in = mine && e == key;
            const unsigned grp = __ballot_sync(0xffffffffu, in);
            double vals[5];
            vals[0] = double(warp_sum<Real>(in ? v[0].s : Real(0))) - double(warp_sum<Real>(in ? v[0].comp() : Real(0)));
            vals[1] = double(warp_sum<Real>(in ? v[1].s : Real(0))) - double(warp_sum<Real>(in ? v[1].comp() : Real(0)));
            vals[2] = double(warp_sum<Real>(in ? v[2].s : Real(0))) - double(warp_sum<Real>(in ? v[2].comp() : Real(0)));
            vals[3] = double(warp_sum<Real>(in ? E.s : Real(0))) - double(warp_sum<Real>(in ? E.comp() : Real(0)));
            vals[4] = double(warp_sum<Real>(in ? Et.s : Real(0))) - double(warp_sum<Real>(in ? Et.comp() : Real(0)));
            const unsigned int c0 = __reduce_add_sync(0xffffffffu, in ? nvalley(0) : 0u);
            const unsigned int c1 = __reduce_add_sync(0xffffffffu, in ? nvalley(1) : 0u);
            const unsigned int c2 = __reduce_add_sync(0xffffffffu, in ? nvalley(2) : 0u);
            if ((threadIdx.x & 31) == __ffs(grp) - 1) {
                const unsigned int cnt[3] = {c0, c1, c2};
                const int w = key - e_base;
                if (w >= 0 && w < WE) {
                    for (int i = 0; i < 5; ++i)
                        if (vals[i] != 0.0) atomicAdd(&bt->sums[w][i], vals[i]);
                    for (int i = 0; i < NV; ++i)
                        if (cnt[i]) atomicAdd(&bt->cnt[w][CNT_V0 + i], cnt[i]);
                    atomicAdd(&bt->cnt[w][CNT_SAMPLES], c0 + c1 + c2);
                } else {
                    for (int i = 0; i < 5; ++i)
                        if (vals[i] != 0.0) atomicAdd(&P.sums[(size_t)key * NSUM + i], vals[i]);
                    for (int i = 0; i < NV; ++i)
                        if (cnt[i]) atomicAdd(&P.cnt[(size_t)key * NCNT + CNT_V0 + i], (unsigned long long)cnt[i]);
                    atomicAdd(&P.cnt[(size_t)key * NCNT + CNT_SAMPLES], (unsigned long long)(c0 + c1 + c2));
                }
            }
            pending &= ~grp;
        }
        if (need) {
            for (int i = 0; i < 3; ++i) v[i].clear();
            E.clear();
            Et.clear();
            nv = 0ull;
        }
    }
};

// Samples of one particle over the steps of a launch.  Float build: plain
// float partial sums over the (at most a few tens of) steps, folded into the
// thread's compensated accumulators once per particle; double build: added
// to the accumulators directly, in step order.
template <typename Real>
struct StepSums {
    // the total energy's valley-edge part is added once per stretch of steps
    // in one valley (add_ec), not per step
    Real v0 = 0, v1 = 0, v2 = 0, E = 0, Ec = 0;
    __device__ __forceinline__ void add(Samples<Real>&, Real a, Real b, Real c, Real d, Real)
    {
        v0 += a;
        v1 += b;
        v2 += c;
        E += d;
    }
    __device__ __forceinline__ void add_ec(Real x) { Ec += x; }
    __device__ __forceinline__ void fold(Samples<Real>& S) const
    {
        S.v[0].add(v0);
        S.v[1].add(v1);
        S.v[2].add(v2);
        S.E.add(E);
        S.Et.add(E + Ec);
    }
};
template <>
struct StepSums<double> {
    __device__ __forceinline__ void add(Samples<double>& S, double a, double b, double c, double d, double e)
    {
        S.v[0].add(a);
        S.v[1].add(b);
        S.v[2].add(c);
        S.E.add(d);
        S.Et.add(e);
    }
    __device__ __forceinline__ void add_ec(double) {}  // added per step, in step order
    __device__ __forceinline__ void fold(Samples<double>&) const {}
};

// -------------------------------------------------------------- flight
// Persistent blocks, no block-level barriers after set-up: warp g of the
// grid advances the 32-slot chunks g, g + W, g + 2W, ... (W warps in the
// grid), one particle per lane, with coalesced state loads and stores.  The
// round robin spreads every stretch of the slot range over all warps, so a
// sorted range (neighbouring slots in neighbouring subcells, a hot drain end
// and a cool source end) still balances.  Every free flight carries the
// particle to its next event -- the end of its step or a scattering --
// through one shared drift and wall check; the lanes of a warp need not be
// in the same step (the field is fixed within a launch), and scatterings
// wait until enough lanes have one (below).  Block tallies in
// shared memory are indexed by ensemble (the first WE ensembles; others go
// straight to global atomics).  The rate table of a single table set is
// staged in shared memory for bins [0, nbs); the per-table-set physics for
// up to 64 table sets.
__device__ __forceinline__ void flush_window(const DevParams& P, BlockTally* bt)
{
    for (int i = threadIdx.x; i < WE * NV * NM; i += blockDim.x) {
        const int w = i / (NV * NM), j = i - w * NV * NM;
        const unsigned int n = bt->ev[w][j];  // bulk only (one subcell per ensemble)
        if (n && w < P.n_ens) atomicAdd(&P.events[(size_t)w * NV * NM + j], (unsigned long long)n);
    }
    for (int i = threadIdx.x; i < WE * NCNT; i += blockDim.x) {
        const int w = i / NCNT, j = i - w * NCNT;
        const unsigned int n = bt->cnt[w][j];
        if (n && w < P.n_ens) {
            atomicAdd(&P.cnt[(size_t)w * NCNT + j], (unsigned long long)n);
            if (j == CNT_SRC_OUT || j == CNT_DRN_OUT)
                atomicAdd(reinterpret_cast<unsigned long long*>(&P.alive[w]), (unsigned long long)(-(long long)n));
        }
    }
    for (int i = threadIdx.x; i < WE * NSUM; i += blockDim.x) {
        const int w = i / NSUM, j = i - w * NSUM;
        const double x = bt->sums[w][j];
        if (x != 0.0 && w < P.n_ens) atomicAdd(&P.sums[(size_t)w * NSUM + j], x);
    }
}

// The flight of one context's particles by the blocks blk = 0 .. nblk - 1 of
// a launch (a launch may run two contexts side by side, each on its own
// blocks: k_flight_pair).
template <typename Real, bool NW>
__device__ __forceinline__ void flight_body(const DevParams& P, const KConst<Real>& K, int n_steps, int count_charge,
                                            unsigned char* sm, int blk, int nblk)
{
    const int nbs = K.nbs;
    Real* tab_s = reinterpret_cast<Real*>(sm);
    size_t off = ((size_t)NV * nbs * NM * sizeof(Real) + 15) & ~size_t(15);
    Phys<Real>* ph_s = reinterpret_cast<Phys<Real>*>(sm + off);
    off += ((size_t)K.n_tab_s * sizeof(Phys<Real>) + 15) & ~size_t(15);
    BlockTally* bt = reinterpret_cast<BlockTally*>(sm + off);

    const Real* tab_all = static_cast<const Real*>(P.table);
    const Phys<Real>* ph_g = static_cast<const Phys<Real>*>(P.phys);
    for (int i = threadIdx.x; i < NV * nbs * NM; i += blockDim.x) {
        const int v = i / (nbs * NM), rr = i - v * nbs * NM;
        tab_s[i] = tab_all[(size_t)v * K.nb * NM + rr];
    }
    for (int i = threadIdx.x; i < K.n_tab_s * (int)(sizeof(Phys<Real>) / sizeof(Real)); i += blockDim.x)
        reinterpret_cast<Real*>(ph_s)[i] = reinterpret_cast<const Real*>(ph_g)[i];
    for (int i = threadIdx.x; i < (int)(sizeof(BlockTally) / 4); i += blockDim.x)
        reinterpret_cast<unsigned int*>(bt)[i] = 0u;
    __syncthreads();

    const Real dt = K.dt;
    const int nbs1 = (K.n_tab == 1) ? nbs : 0;
    const int e_base = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)nblk * (blockDim.x >> 5);
    const int64_t n_chunks = (P.n_slots + 31) >> 5;
    Samples<Real> S;
    // runs of kChunkRun consecutive chunks per warp, the runs dealt round
    // robin: a lane's next particle is most often of the same ensemble, so
    // its samples are handed over (a warp-wide reduction) once per run.
    // Two measured fastest on the sorted 21 x 200,000 sweep (1.76e9 real
    // events/s against 1.74e9 for one, 1.61e9 for four, 1.50e9 for eight:
    // longer runs put too much of a sorted stretch on one warp)
    const int64_t w0 = (int64_t)blk * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t c0 = w0 * kChunkRun; c0 < n_chunks; c0 += warps * kChunkRun)
    for (int64_t c = c0; c < c0 + kChunkRun && c < n_chunks; ++c) {
        const int64_t p = c * 32 + lane;
        const uint32_t tg = (p < P.n_slots) ? P.tag[p] : uint32_t(DEAD);
        const bool valid = (tg & 0xFFu) != DEAD;
        // lanes whose samples belong to another ensemble than their new
        // particle hand them over (warp-wide, all lanes converged here)
        const bool need = valid && int(tg >> 8) != S.e;
        if (__any_sync(0xffffffffu, need)) S.flush_warp(P, bt, e_base, need);
        QEntry<Real> Q;
        Part<Real>& q = Q.q;
        q.e = valid ? int(tg >> 8) : 0;
        q.v = valid ? int(tg & 0xFFu) : 0;
        q.kx = q.ky = q.kz = q.x = q.y = q.z = q.tr = q.E = q.f = Real(0);
        q.ctr = 0;
        q.id = 0;
        q.seed = 0;
        if (valid) {
            S.e = q.e;
            q.kx = static_cast<const Real*>(P.kx)[p];
            q.ky = static_cast<const Real*>(P.ky)[p];
            q.kz = static_cast<const Real*>(P.kz)[p];
            if (NW) {
                q.x = static_cast<const Real*>(P.x)[p];
                q.y = static_cast<const Real*>(P.y)[p];
                q.z = static_cast<const Real*>(P.z)[p];
            }
            q.tr = static_cast<const Real*>(P.tr)[p];
            q.ctr = P.ctr[p];
            q.id = gid_of(P, q.e, P.id[p]);
            q.seed = P.seed[q.e];
        }
        const int ts = P.tabset[q.e];
        const Phys<Real>& ph = (ts < K.n_tab_s) ? ph_s[ts] : ph_g[ts];
        const Real* tab_g = tab_all + (size_t)ts * NV * K.nb * NM;
        if (valid) {
            q.E = kane_E(ph.ck[q.v] * norm2(q.kx, q.ky, q.kz), ph.alpha[q.v]);
            q.f = ph.vk[q.v] / fma_(Real(2) * ph.alpha[q.v], q.E, Real(1));
        }
        Real f4[4] = {Real(0), Real(0), Real(0), Real(0)};
        int cell = -1;
        if (valid) {
            if (NW) {
                // the field of the subcell at the start of a step (reloaded
                // only when the particle has changed subcell)
                cell = cell_of<Real>(K, q.x, q.y, q.z);
                load4<Real>(static_cast<const Real*>(P.acc_cell) + 4 * ((size_t)q.e * K.ncell + cell), f4);
            } else {
                load4<Real>(static_cast<const Real*>(P.acc_bulk) + 4 * (size_t)q.e, f4);
            }
        }
        StepSums<Real> ss;
        unsigned int nsv = 0u;  // step ends in the particle's current valley, not yet counted
        // The warp runs in step: each round the lanes without a pending
        // scattering take one free flight (to the end of their step or to
        // their next scattering, through the walls); the pending scatterings
        // (mechanism choice, final state) run once at least a third of the
        // lanes still working wait for one, so that code runs with many
        // lanes of the warp instead of with the few that scatter in a given
        // step (a third measured fastest: a half or more leaves too many
        // lanes idle in the flights, a quarter or less runs the scatterings
        // with too few).  A particle's own sequence of flights, draws and
        // tallies is the same as step by step.
        bool live = true, done = !valid || n_steps <= 0, pending = false;
        int s = 0, it = 0;
        Real tleft = dt;
        for (;;) {
            if (!done && !pending) {
                bool step_end = false;
                if (it >= MAX_FLIGHTS_PER_STEP) {
                    atomicOr(P.err, ERR_FLIGHTS);
                    step_end = true;  // the step ends where the particle is
                } else {
                    ++it;
                    const bool to_end = q.tr >= tleft;
                    drift<Real, NW>(q, ph, f4, to_end ? tleft : q.tr);
                    if (NW && walls(q, P, K, bt, e_base)) {
                        live = false;
                        done = true;
                    } else if (to_end) {
                        q.tr -= tleft;
                        step_end = true;
                    } else {
                        tleft -= q.tr;
                        pending = true;
                    }
                }
                if (step_end) {
                    ss.add(S, q.f * q.kx, q.f * q.ky, q.f * q.kz, q.E, q.E + ph.Ec[q.v]);
                    ++nsv;
                    ++s;
                    it = 0;
                    tleft = dt;
                    if (s >= n_steps) {
                        done = true;
                    } else if (NW) {
                        const int cc = cell_of<Real>(K, q.x, q.y, q.z);
                        if (cc != cell) {
                            load4<Real>(static_cast<const Real*>(P.acc_cell) + 4 * ((size_t)q.e * K.ncell + cc), f4);
                            cell = cc;
                        }
                    }
                }
            }
            const unsigned pend = __ballot_sync(0xffffffffu, pending);
            const unsigned work = __ballot_sync(0xffffffffu, !done);
            if (work == 0u) break;
            if (3 * __popc(pend) < __popc(work)) continue;
            if (pending) {
                if (choose<Real>(Q, P, K, ph, tab_s, nbs1, tab_g, bt, e_base) >= 0) {
                    if (Q.mech >= 4) {  // intervalley: the step ends so far were in the old valley
                        S.count_valley(q.v, nsv);
                        ss.add_ec(Real(nsv) * ph.Ec[q.v]);
                        nsv = 0u;
                    }
                    final_state<Real, NW>(Q, P, K, ph, bt, e_base);
                }
                pending = false;
            }
        }
        if (valid) {
            S.count_valley(q.v, nsv);
            ss.add_ec(Real(nsv) * ph.Ec[q.v]);
            ss.fold(S);
            store<Real>(P, p, q, NW);
            P.tag[p] = (uint32_t(q.e) << 8) | (live ? uint32_t(q.v) : DEAD);
            if (NW && !live) {
                // left through a contact: its id is free for the refill
                const uint32_t i = P.id[p];
                atomicOr(&P.dead_bits[P.bits_off[q.e] + (i >> 5)], 1u << (i & 31u));
            }
        }
        if (NW && count_charge && valid && live)
            agg_add_i(P.charge, q.e * K.ncell + cell_of<Real>(K, q.x, q.y, q.z));
    }
    S.flush_warp(P, bt, e_base, true);
    __syncthreads();
    flush_window(P, bt);
}

template <typename Real, bool NW>
__global__ void __launch_bounds__(256, 4)
    k_flight(const DevParams P, const KConst<Real> K, int n_steps, int count_charge)
{
    extern __shared__ __align__(16) unsigned char sm[];
    flight_body<Real, NW>(P, K, n_steps, count_charge, sm, blockIdx.x, gridDim.x);
}

// Two contexts in one launch: blocks [0, nblk0) fly context 0, the others
// context 1 (the mixed bulk + nanowire batch: one context per geometry).
template <typename Real, bool NW0, bool NW1>
__global__ void __launch_bounds__(256, 4)
    k_flight_pair(const DevParams P0, const KConst<Real> K0, int n_steps0, int count0, const DevParams P1,
                  const KConst<Real> K1, int n_steps1, int count1, int nblk0)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if ((int)blockIdx.x < nblk0)
        flight_body<Real, NW0>(P0, K0, n_steps0, count0, sm, blockIdx.x, nblk0);
    else
        flight_body<Real, NW1>(P1, K1, n_steps1, count1, sm, (int)blockIdx.x - nblk0, (int)gridDim.x - nblk0);
}

// ---------------------------------------------------------------- init
template <typename Real, bool NW>
__global__ void k_init(const DevParams P)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n_slots) return;
    int lo = 0, hi = P.n_ens - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.ens_off[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    const int e = lo;
    const uint32_t id = uint32_t(s - P.ens_off[e]);
    P.id[s] = id;
    P.slot_of_id[s] = uint32_t(s);
    Part<Real> q;
    q.e = e;
    q.id = gid_of(P, e, id);
    q.seed = P.seed[e];
    q.ctr = 0;
    if ((int64_t)id < P.ens_n0[e]) {
        const Phys<Real>* ph = static_cast<const Phys<Real>*>(P.phys) + P.tabset[e];
        const Real lo3[3] = {0, 0, 0};
        const Real len3[3] = {Real(P.Lx), Real(P.Ly), Real(P.Lz)};
        new_electron<Real, NW>(q, ph, lo3, len3, P.err);
        store<Real>(P, s, q, NW);
        P.tag[s] = uint32_t(e) << 8;
    } else {
        q.kx = q.ky = q.kz = q.x = q.y = q.z = q.tr = Real(0);
        store<Real>(P, s, q, NW);
        P.tag[s] = (uint32_t(e) << 8) | DEAD;
        atomicOr(&P.dead_bits[P.bits_off[e] + (id >> 5)], 1u << (id & 31u));
    }
}

// --------------------------------------------------------------- inject
// Refill each contact subcell (the x = 0 layer first, then x = Lx, cells in
// (y, z) order) up to n_target electrons, taking free ids of the wire in
// increasing global order: the r-th free id fills the r-th missing electron.
// The global order ranks the free initial-electron ids (global ids < N) of
// all shards first, shard by shard, then the free spare ids, shard by shard;
// unsharded, it is the order of the local ids.  One block per ensemble.
// Threads own contiguous words of the free-id bitmap; a block scan of the
// words' population counts (initial-electron and spare ids apart) gives
// each free id its rank, ids are gathered by rank into shared memory (INJ
// per round) and the new electrons are drawn in parallel.  The subcell
// charge grows by the wire's refill of each contact subcell, which the
// deficits and the wire's free-id count fix, so every shard ends with the
// wire's count.  Dynamic shared memory: a scan buffer (blockDim 64-bit
// words), the deficit prefix sums (2 ny nz + 1 ints) and INJ ids.
constexpr int INJ = 1024;

// free ids among local ids [32 w, 32 w + 32) below n0 (initial-electron
// ids) and at or above it (spare ids)
__device__ __forceinline__ void free_split(uint32_t word, int64_t w, int64_t n0, int& a, int& b)
{
    const int64_t lo = 32 * w;
    uint32_t ma;
    if (lo + 32 <= n0) ma = 0xFFFFFFFFu;
    else if (lo >= n0) ma = 0u;
    else ma = (1u << uint32_t(n0 - lo)) - 1u;
    a = __popc(word & ma);
    b = __popc(word & ~ma);
}

template <typename Real>
__global__ void __launch_bounds__(1024) k_inject(const DevParams P)
{
    extern __shared__ long long shl[];
    const int e = blockIdx.x;
    const int nface = P.ny * P.nz, ncon = 2 * nface;
    long long* scan = shl;
    int* pre = reinterpret_cast<int*>(scan + blockDim.x);
    uint32_t* ids = reinterpret_cast<uint32_t*>(pre + ncon + 1);
    __shared__ int n_src, n_drn;
    // deficits of the contact cells, loaded in parallel, then their prefix
    // sums (pre[t] = electrons missing in contacts 0 .. t-1)
    for (int t = threadIdx.x; t < ncon; t += blockDim.x) {
        const int side = t / nface, rem = t - side * nface;
        const int ix = side ? P.nx - 1 : 0;
        const int need = P.n_target[e] - P.charge[(size_t)e * P.ncell + ix * nface + rem];
        pre[t + 1] = need > 0 ? need : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int t = 0; t < ncon; ++t) pre[t + 1] += pre[t];
        n_src = 0;
        n_drn = 0;
    }
    __syncthreads();
    const int D = pre[ncon];
    if (D == 0) return;
    const int64_t n0 = P.ens_n0[e];
    const int64_t words = (P.ens_cap[e] + 31) / 32;
    uint32_t* bits = P.dead_bits + P.bits_off[e];
    const int64_t per = (words + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = (int64_t)threadIdx.x * per;
    const int64_t w1 = w0 + per < words ? w0 + per : words;
    int mine_a = 0, mine_b = 0;
    for (int64_t w = w0; w < w1; ++w) {
        int a, b;
        free_split(bits[w], w, n0, a, b);
        mine_a += a;
        mine_b += b;
    }
    const long long mine = ((long long)mine_a << 32) | (long long)mine_b;
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const long long x = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += x;
        __syncthreads();
    }
    const long long last = scan[blockDim.x - 1], incl = scan[threadIdx.x];
    const long long loc_a = last >> 32, loc_b = last & 0xFFFFFFFFll;
    long long off_a = 0, off_b = 0, tot_a = loc_a, tot_b = loc_b;
    bool lead = true;
    if (P.shard) {
        const long long* sh = P.shard + 5 * (size_t)e;
        off_a = sh[0];
        off_b = sh[1];
        tot_a = sh[2];
        tot_b = sh[3];
        lead = sh[4] != 0;
    }
    const long long total = tot_a + tot_b;
    const int Deff = D < total ? D : int(total);
    if (threadIdx.x == 0 && lead && total < D)
        atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_STARVED], (unsigned long long)(D - total));
    // wire ranks of this thread's first free initial-electron id and first
    // free spare id; along the thread's words the ranks rise, and every
    // spare rank is above every initial-electron rank
    const long long base_a = off_a + (incl >> 32) - mine_a;
    const long long base_b = tot_a + off_b + (incl & 0xFFFFFFFFll) - mine_b;
    const long long own_a0 = off_a, own_a1 = off_a + loc_a;
    const long long own_b0 = tot_a + off_b, own_b1 = tot_a + off_b + loc_b;
    const Phys<Real>* ph = static_cast<const Phys<Real>*>(P.phys) + P.tabset[e];
    const Real len3[3] = {Real(P.dx), Real(P.dy), Real(P.dz)};
    for (int r0 = 0; r0 < Deff; r0 += INJ) {
        const int r1 = min(Deff, r0 + INJ);
        // (block-uniform) no id of this shard has a rank in [r0, r1)
        if (!(own_a0 < r1 && r0 < own_a1) && !(own_b0 < r1 && r0 < own_b1)) continue;
        // gather the ids of ranks [r0, r1) by rank
        long long rank = base_a;
        bool in_b = false;
        for (int64_t w = w0; w < w1 && rank < r1; ++w) {
            uint32_t word = bits[w];
            while (word && rank < r1) {
                const int bit = __ffs(word) - 1;
                word &= word - 1u;
                const int64_t i = w * 32 + bit;
                if (i >= n0 && !in_b) {
                    in_b = true;
                    rank = base_b;
                    if (rank >= r1) break;
                }
                if (rank >= r0) ids[rank - r0] = uint32_t(i);
                ++rank;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < r1 - r0; k += blockDim.x) {
            const long long rk = r0 + k;
            if (!((rk >= own_a0 && rk < own_a1) || (rk >= own_b0 && rk < own_b1))) continue;
            const uint32_t id = ids[k];
            int lo = 0, hi = ncon - 1;  // contact t with pre[t] <= rk < pre[t + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= rk) lo = mid;
                else hi = mid - 1;
            }
            const int t = lo;
            const int side = t / nface, rem = t - side * nface;
            const int ix = side ? P.nx - 1 : 0, iy = rem / P.nz, iz = rem - iy * P.nz;
            EMC_CHECK(P.err, (int64_t)id < P.ens_cap[e] && t >= 0 && t < ncon);
            const int64_t slot = P.slot_of_id[P.ens_off[e] + id];
            EMC_CHECK(P.err, slot >= P.ens_off[e] && slot < P.ens_off[e] + P.ens_cap[e]);
            Part<Real> q;
            q.e = e;
            q.id = gid_of(P, e, id);
            q.seed = P.seed[e];
            q.ctr = P.ctr[slot];
            const Real lo3[3] = {Real(ix * P.dx), Real(iy * P.dy), Real(iz * P.dz)};
            const Phys<Real>* pi = ph;
            Phys<Real> pt;
            if (P.cell_bin) {
                // thermal at the subcell's temperature; first flight with the ensemble's Gamma0
                pt = static_cast<const Phys<Real>*>(P.bin_phys)[P.cell_bin[(size_t)e * P.ncell + ix * nface + rem]];
                for (int vv = 0; vv < NV; ++vv) pt.inv_g0[vv] = static_cast<const Real*>(P.ens_ig0)[(size_t)e * NV + vv];
                pi = &pt;
            }
            new_electron<Real, true>(q, pi, lo3, len3, P.err);
            store<Real>(P, slot, q, true);
            P.tag[slot] = uint32_t(e) << 8;
            atomicAdd(side ? &n_drn : &n_src, 1);
        }
        __syncthreads();
    }
    // the wire's refill of each contact subcell: the missing electrons of
    // contact t whose ranks are below Deff
    for (int t = threadIdx.x; t < ncon; t += blockDim.x) {
        int got = Deff - pre[t];
        const int need = pre[t + 1] - pre[t];
        got = got < 0 ? 0 : (got > need ? need : got);
        if (got > 0) {
            const int side = t / nface, rem = t - side * nface;
            const int ix = side ? P.nx - 1 : 0;
            P.charge[(size_t)e * P.ncell + ix * nface + rem] += got;
        }
    }
    // clear the bits of the ids taken (ranks below Deff).  The whole
    // ensemble is one block, so every thread's scan of the bitmap above has
    // finished before any bit changes (several blocks per ensemble would
    // rank against a bitmap that others are already clearing)
    long long rank = base_a;
    bool in_b = false;
    for (int64_t w = w0; w < w1 && rank < Deff; ++w) {
        uint32_t word = bits[w], clear = 0u;
        while (word && rank < Deff) {
            const int bit = __ffs(word) - 1;
            word &= word - 1u;
            if (w * 32 + bit >= n0 && !in_b) {
                in_b = true;
                rank = base_b;
                if (rank >= Deff) break;
            }
            clear |= 1u << bit;
            ++rank;
        }
        bits[w] &= ~clear;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_SRC_IN], (unsigned long long)n_src);
        atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_DRN_IN], (unsigned long long)n_drn);
        atomicAdd(reinterpret_cast<unsigned long long*>(&P.alive[e]), (unsigned long long)(n_src + n_drn));
    }
}

// Free ids of each ensemble among its initial-electron ids and among its
// spare ids (out[e][0], out[e][1]); one block per ensemble.
template <typename Real>
__global__ void __launch_bounds__(256) k_free_counts(const DevParams P, long long* out)
{
    __shared__ long long ra[256], rb[256];
    const int e = blockIdx.x;
    const int64_t n0 = P.ens_n0[e];
    const int64_t words = (P.ens_cap[e] + 31) / 32;
    const uint32_t* bits = P.dead_bits + P.bits_off[e];
    long long sa = 0, sb = 0;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
        int a, b;
        free_split(bits[w], w, n0, a, b);
        sa += a;
        sb += b;
    }
    ra[threadIdx.x] = sa;
    rb[threadIdx.x] = sb;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            ra[threadIdx.x] += ra[threadIdx.x + h];
            rb[threadIdx.x] += rb[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * e] = ra[0];
        out[2 * e + 1] = rb[0];
    }
}

// ----------------------------------------------------------------- sort
// Counting sort of the particle slots by key (ensemble, valley, subcell),
// free slots (valley DEAD) last within each ensemble's range, so that the
// ranges stay where they are.  Key pass: histogram; the host-side scan gives
// the offsets; scatter pass: every slot moves to offset[key] + rank (the rank
// order inside a key does not matter: every particle carries its own id and
// Philox stream).
template <typename Real, bool NW>
__global__ void k_sort_keys(const DevParams P, const KConst<Real> K, uint32_t* key, unsigned int* hist)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_slots) return;
    const uint32_t tg = P.tag[p];
    const int e = int(tg >> 8);
    const int v = (tg & 0xFFu) == DEAD ? NV : int(tg & 0xFFu);
    int c = 0;
    if (NW && v < NV)
        c = cell_of<Real>(K, static_cast<const Real*>(P.x)[p], static_cast<const Real*>(P.y)[p],
                          static_cast<const Real*>(P.z)[p]);
    const uint32_t kk = (uint32_t)(((size_t)e * (NV + 1) + v) * K.ncell + c);
    key[p] = kk;
    const unsigned peers = __match_any_sync(__activemask(), kk);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[kk], (unsigned)__popc(peers));
}

template <typename Real, bool NW>
__global__ void k_sort_scatter(const DevParams P, const uint32_t* key, const unsigned int* offs,
                               unsigned int* cursor, DevParams Q)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_slots) return;
    const uint32_t kk = key[p];
    // one cursor claim per group of lanes with the same key
    const unsigned peers = __match_any_sync(__activemask(), kk);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&cursor[kk], (unsigned)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t d = (int64_t)offs[kk] + base + __popc(peers & ((1u << lane) - 1u));
    EMC_CHECK(P.err, d >= 0 && d < P.n_slots);
    static_cast<Real*>(Q.kx)[d] = static_cast<const Real*>(P.kx)[p];
    static_cast<Real*>(Q.ky)[d] = static_cast<const Real*>(P.ky)[p];
    static_cast<Real*>(Q.kz)[d] = static_cast<const Real*>(P.kz)[p];
    if (NW) {
        static_cast<Real*>(Q.x)[d] = static_cast<const Real*>(P.x)[p];
        static_cast<Real*>(Q.y)[d] = static_cast<const Real*>(P.y)[p];
        static_cast<Real*>(Q.z)[d] = static_cast<const Real*>(P.z)[p];
    }
    static_cast<Real*>(Q.tr)[d] = static_cast<const Real*>(P.tr)[p];
    Q.ctr[d] = P.ctr[p];
    Q.tag[d] = P.tag[p];
    const uint32_t id = P.id[p];
    Q.id[d] = id;
    P.slot_of_id[P.ens_off[P.tag[p] >> 8] + id] = uint32_t(d);
}

// After a change of an ensemble's Gamma0 (new subcell temperatures) the
// residual flight times are rescaled by Gamma0_old / Gamma0_new of their
// valley: an exponential residual of rate G_old times G_old / G_new is an
// exponential of rate G_new, so no redraw is needed.
template <typename Real>
__global__ void k_rescale_flights(const DevParams P, int e, const double* ratio)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ens_cap[e]) return;
    const int64_t s = P.ens_off[e] + i;
    const uint32_t tg = P.tag[s];
    if ((tg & 0xFFu) == DEAD) return;
    static_cast<Real*>(P.tr)[s] = static_cast<Real*>(P.tr)[s] * Real(ratio[tg & 0xFFu]);
}

// --------------------------------------------------------------- launch
template <typename Real>
size_t flight_smem_bytes(int nb_smem, int n_tab_s)
{
    return (((size_t)NV * nb_smem * NM * sizeof(Real) + 15) & ~size_t(15)) +
           (((size_t)n_tab_s * sizeof(Phys<Real>) + 15) & ~size_t(15)) + sizeof(BlockTally);
}

// The dynamic shared-memory limit is an attribute of the kernel on the
// current device, shared by every context: it is only ever raised (to the
// largest request seen on the device), so a context that needs less never
// lowers the limit under another one that is still alive.
template <typename Real>
cudaError_t flight_set_smem(size_t bytes)
{
    static std::mutex mu;
    static std::map<int, size_t> raised;
    int dev = 0;
    cudaError_t a = cudaGetDevice(&dev);
    if (a != cudaSuccess) return a;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = raised[dev];
    if (bytes <= cur) return cudaSuccess;
    a = cudaFuncSetAttribute(k_flight<Real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (a != cudaSuccess) return a;
    a = cudaFuncSetAttribute(k_flight<Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (a == cudaSuccess) cur = bytes;
    return a;
}

// resident flight blocks per SM for this shared-memory size
template <typename Real>
int flight_blocks_per_sm(bool nw, int block, size_t smem)
{
    int n = 0;
    if (nw)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_flight<Real, true>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_flight<Real, false>, block, smem);
    return n > 0 ? n : 1;
}

template <typename Real>
KConst<Real> flight_consts(const DevParams& P)
{
    KConst<Real> K;
    K.Lx = Real(P.Lx);
    K.Ly = Real(P.Ly);
    K.Lz = Real(P.Lz);
    K.inv_dx = Real(1.0 / P.dx);
    K.inv_dy = Real(1.0 / P.dy);
    K.inv_dz = Real(1.0 / P.dz);
    K.p_spec = Real(P.p_spec);
    K.dt = Real(P.dt);
    K.inv_dE = Real(P.inv_dE);
    K.nx = P.nx;
    K.ny = P.ny;
    K.nz = P.nz;
    K.ncell = P.ncell;
    K.nb = P.nb;
    K.nbs = P.nb_smem;
    K.n_tab = P.n_tab;
    K.n_tab_s = P.n_tab <= 64 ? P.n_tab : 0;
    K.per_block = 0;
    K.err = P.err;
    return K;
}

template <typename Real>
void launch_flight(const DevParams& P, bool nw, int n_steps, int count_charge, int block, int grid_cap,
                   cudaStream_t st)
{
    if (P.n_slots <= 0) return;
    const KConst<Real> K = flight_consts<Real>(P);
    const int64_t tiles = (P.n_slots + block - 1) / block;
    const int64_t g = tiles < grid_cap ? tiles : grid_cap;
    const size_t smem = flight_smem_bytes<Real>(K.nbs, K.n_tab_s);
    if (nw)
        k_flight<Real, true><<<(unsigned)g, block, smem, st>>>(P, K, n_steps, count_charge);
    else
        k_flight<Real, false><<<(unsigned)g, block, smem, st>>>(P, K, n_steps, count_charge);
}

// Shared memory and resident blocks per SM of the two-context launch.
template <typename Real>
cudaError_t pair_prepare(const DevParams& P0, bool nw0, const DevParams& P1, bool nw1, int block, size_t* smem,
                         int* blocks_per_sm)
{
    const KConst<Real> K0 = flight_consts<Real>(P0), K1 = flight_consts<Real>(P1);
    const size_t s0 = flight_smem_bytes<Real>(K0.nbs, K0.n_tab_s), s1 = flight_smem_bytes<Real>(K1.nbs, K1.n_tab_s);
    *smem = s0 > s1 ? s0 : s1;
    const void* fn = nw0 ? (nw1 ? (const void*)k_flight_pair<Real, true, true> : (const void*)k_flight_pair<Real, true, false>)
                         : (nw1 ? (const void*)k_flight_pair<Real, false, true> : (const void*)k_flight_pair<Real, false, false>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    *blocks_per_sm = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, *smem);
}

// Both contexts in one launch of `grid` blocks, split in proportion to
// their particle slots (at least one block each).
template <typename Real>
void launch_flight_pair(const DevParams& P0, bool nw0, int n_steps0, int count0, const DevParams& P1, bool nw1,
                        int n_steps1, int count1, int block, int grid, size_t smem, cudaStream_t st)
{
    const KConst<Real> K0 = flight_consts<Real>(P0), K1 = flight_consts<Real>(P1);
    const double f = double(P0.n_slots) / double(P0.n_slots + P1.n_slots);
    int g = grid < 2 ? 2 : grid;
    int n0 = (int)(f * g + 0.5);
    n0 = n0 < 1 ? 1 : (n0 > g - 1 ? g - 1 : n0);
    if (nw0 && nw1)
        k_flight_pair<Real, true, true><<<g, block, smem, st>>>(P0, K0, n_steps0, count0, P1, K1, n_steps1, count1, n0);
    else if (nw0)
        k_flight_pair<Real, true, false><<<g, block, smem, st>>>(P0, K0, n_steps0, count0, P1, K1, n_steps1, count1, n0);
    else if (nw1)
        k_flight_pair<Real, false, true><<<g, block, smem, st>>>(P0, K0, n_steps0, count0, P1, K1, n_steps1, count1, n0);
    else
        k_flight_pair<Real, false, false><<<g, block, smem, st>>>(P0, K0, n_steps0, count0, P1, K1, n_steps1, count1, n0);
}
template <typename Real>
void launch_sort(const DevParams& P, const DevParams& alt, bool nw, uint32_t* key, unsigned int* hist,
                 const unsigned int* offs, unsigned int* cursor, int phase, cudaStream_t st)
{
    if (P.n_slots <= 0) return;
    KConst<Real> K{};
    K.inv_dx = Real(1.0 / P.dx);
    K.inv_dy = Real(1.0 / P.dy);
    K.inv_dz = Real(1.0 / P.dz);
    K.nx = P.nx;
    K.ny = P.ny;
    K.nz = P.nz;
    K.ncell = P.ncell;
    K.err = P.err;
    const unsigned grid = (unsigned)((P.n_slots + 255) / 256);
    if (phase == 0) {
        if (nw) k_sort_keys<Real, true><<<grid, 256, 0, st>>>(P, K, key, hist);
        else k_sort_keys<Real, false><<<grid, 256, 0, st>>>(P, K, key, hist);
    } else {
        if (nw) k_sort_scatter<Real, true><<<grid, 256, 0, st>>>(P, key, offs, cursor, alt);
        else k_sort_scatter<Real, false><<<grid, 256, 0, st>>>(P, key, offs, cursor, alt);
    }
}

template <typename Real>
void launch_rescale(const DevParams& P, int e, int64_t cap, const double* ratio, cudaStream_t st)
{
    if (cap <= 0) return;
    k_rescale_flights<Real><<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(P, e, ratio);
}

template <typename Real>
void launch_init(const DevParams& P, bool nw, cudaStream_t st)
{
    if (P.n_slots <= 0) return;
    const unsigned grid = (unsigned)((P.n_slots + 255) / 256);
    if (nw)
        k_init<Real, true><<<grid, 256, 0, st>>>(P);
    else
        k_init<Real, false><<<grid, 256, 0, st>>>(P);
}

template <typename Real>
void launch_inject(const DevParams& P, cudaStream_t st)
{
    // one block per ensemble (the bitmap is ranked and cleared by one block):
    // the widest block shortens each thread's stretch of the bitmap
    // (measured: 1024 threads 0.9% faster per Poisson period than 256)
    const int block = 1024;
    const size_t smem = sizeof(long long) * block + sizeof(int) * (2 * P.ny * P.nz + 1 + INJ);
    k_inject<Real><<<P.n_ens, block, smem, st>>>(P);
}

template <typename Real>
void launch_free_counts(const DevParams& P, long long* out, cudaStream_t st)
{
    k_free_counts<Real><<<P.n_ens, 256, 0, st>>>(P, out);
}

}  // namespace emc
