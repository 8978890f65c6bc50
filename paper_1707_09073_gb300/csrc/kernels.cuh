// Templated particle kernels of libemc: the fused flight/scatter step, the
// initial ensemble, and the contact re-injection.  Real = float is the
// production path, Real = double the parity build.
//
// Method (Hao et al., arXiv:1707.09073; the paragraphs opening "In such
// simulations" and "For Si-doped GaN nanowires"): every electron is tracked
// through free flights under the local field with the Kane dispersion
// E(1 + aE) = hbar^2 k^2 / 2m, interrupted by scatterings chosen against a
// constant total rate Gamma0 per valley (self-scattering fills the gap to the
// real rates); the subcells count electrons for the Poisson update and the
// net energy handed to phonons.
#pragma once
#include "common.cuh"

namespace emc {

// ------------------------------------------------------------- math
template <typename Real>
struct Mth;
template <>
struct Mth<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float pow_(float b, float e) { return exp2f(e * log2f(b)); }
    static __device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
    static __device__ __forceinline__ float cospi_(float x) { return cospif(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
};
template <>
struct Mth<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double pow_(double b, double e) { return pow(b, e); }
    static __device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }
    static __device__ __forceinline__ double cospi_(double x) { return cospi(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
};

// Kinetic energy whose Kane gamma is g: the positive root of E(1 + aE) = g,
// written as 2g / (1 + sqrt(1 + 4ag)) (exact for a = 0, no cancellation).
template <typename Real>
__device__ __forceinline__ Real kane_E(Real g, Real a)
{
    return Real(2) * g / (Real(1) + Mth<Real>::sqrt_(Real(1) + Real(4) * a * g));
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
};
template <>
struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

struct BlockTally {
    unsigned int ev[WE][NV * NM];
    unsigned int cnt[WE][NCNT];
    double sums[WE][NSUM];
};

__device__ __forceinline__ void tally_cnt(BlockTally* bt, const DevParams& P, int e, int e_base,
                                          int idx, unsigned int n)
{
    const int w = e - e_base;
    if (w >= 0 && w < WE)
        atomicAdd(&bt->cnt[w][idx], n);
    else
        atomicAdd(&P.cnt[(size_t)e * NCNT + idx], (unsigned long long)n);
}

// ------------------------------------------------------------ particle
template <typename Real>
struct Part {
    Real kx, ky, kz, x, y, z, tr;
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

template <typename Real>
__device__ __forceinline__ int cell_of(const DevParams& P, Real x, Real y, Real z)
{
    Real fx = Mth<Real>::floor_(x / Real(P.dx));
    Real fy = Mth<Real>::floor_(y / Real(P.dy));
    Real fz = Mth<Real>::floor_(z / Real(P.dz));
    int ix = fx >= Real(0) ? (fx < Real(P.nx) ? int(fx) : P.nx - 1) : 0;
    int iy = fy >= Real(0) ? (fy < Real(P.ny) ? int(fy) : P.ny - 1) : 0;
    int iz = fz >= Real(0) ? (fz < Real(P.nz) ? int(fz) : P.nz - 1) : 0;
    return (ix * P.ny + iy) * P.nz + iz;
}

// Kane-Maxwellian g(E) exp(-E/kT) in valley 0 by rejection: proposal
// -kT (ln u0 + ln u1 cos^2(pi u2 / 2)) ~ Gamma(3/2, kT), accepted when
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
    Real st = Mth<Real>::sqrt_(fmax(Real(0), Real(1) - ct * ct));
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
// k advances linearly (hbar dk/dt = force); in the nanowire the position
// moves along the force by the energy gained over the force and across it by
// the mean of the start and end group velocities times t.
template <typename Real, bool NW>
__device__ __forceinline__ void drift(Part<Real>& q, const Phys<Real>* ph, const Real a[3],
                                      const Real ah[3], Real inv_hF, Real t)
{
    const Real k0x = q.kx, k0y = q.ky, k0z = q.kz;
    q.kx = k0x + a[0] * t;
    q.ky = k0y + a[1] * t;
    q.kz = k0z + a[2] * t;
    if (NW) {
        const int v = q.v;
        const Real ck = ph->ck[v], al = ph->alpha[v], vk = ph->vk[v];
        const Real E0 = kane_E(ck * (k0x * k0x + k0y * k0y + k0z * k0z), al);
        const Real E1 = kane_E(ck * (q.kx * q.kx + q.ky * q.ky + q.kz * q.kz), al);
        const Real f0 = vk / (Real(1) + Real(2) * al * E0);
        const Real f1 = vk / (Real(1) + Real(2) * al * E1);
        const Real h = Real(0.5) * t;
        Real dx = h * (f0 * k0x + f1 * q.kx);
        Real dy = h * (f0 * k0y + f1 * q.ky);
        Real dz = h * (f0 * k0z + f1 * q.kz);
        if (inv_hF > Real(0)) {
            const Real d = (E1 - E0) * inv_hF - (dx * ah[0] + dy * ah[1] + dz * ah[2]);
            dx += d * ah[0];
            dy += d * ah[1];
            dz += d * ah[2];
        }
        q.x += dx;
        q.y += dy;
        q.z += dz;
    }
}

// ------------------------------------------------------------- walls
// Contacts absorb at x < 0 (source) and x > Lx (drain).  Plane A (y = 0) is a
// symmetry plane: always specular.  The outer side (y = Ly), bottom and top
// walls reflect specularly with probability p, else diffusely with a
// cosine-weighted inward direction and |k| kept.  Returns true if absorbed.
template <typename Real>
__device__ __forceinline__ void diffuse(Part<Real>& q, int axis, Real sn, U4 r)
{
    const Real km = Mth<Real>::sqrt_(q.kx * q.kx + q.ky * q.ky + q.kz * q.kz);
    const Real u1 = u01<Real>(r.b);
    const Real ca = Mth<Real>::sqrt_(u1), sa = Mth<Real>::sqrt_(Real(1) - u1);
    Real sp, cp;
    Mth<Real>::sincospi_(Real(2) * u01<Real>(r.c), &sp, &cp);
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
__device__ __forceinline__ bool walls(Part<Real>& q, const DevParams& P, BlockTally* bt, int e_base)
{
    const Real Lx = Real(P.Lx), Ly = Real(P.Ly), Lz = Real(P.Lz), ps = Real(P.p_spec);
    int out = -1;
    if (q.x < Real(0)) out = CNT_SRC_OUT;
    else if (q.x > Lx) out = CNT_DRN_OUT;
    if (out >= 0) {
        tally_cnt(bt, P, q.e, e_base, out, 1u);
        atomicOr(&P.dead_bits[P.bits_off[q.e] + (q.id >> 5)], 1u << (q.id & 31u));
        return true;
    }
    if (q.y < Real(0)) {
        q.y = -q.y;
        q.ky = -q.ky;
    } else if (q.y > Ly) {
        q.y = Real(2) * Ly - q.y;
        U4 r = q.draw();
        if (u01<Real>(r.a) < ps) q.ky = -q.ky;
        else diffuse(q, 1, Real(-1), r);
    }
    q.y = q.y < Real(0) ? Real(0) : (q.y > Ly ? Ly : q.y);
    if (q.z < Real(0)) {
        q.z = -q.z;
        U4 r = q.draw();
        if (u01<Real>(r.a) < ps) q.kz = -q.kz;
        else diffuse(q, 2, Real(1), r);
    } else if (q.z > Lz) {
        q.z = Real(2) * Lz - q.z;
        U4 r = q.draw();
        if (u01<Real>(r.a) < ps) q.kz = -q.kz;
        else diffuse(q, 2, Real(-1), r);
    }
    q.z = q.z < Real(0) ? Real(0) : (q.z > Lz ? Lz : q.z);
    return false;
}

// ----------------------------------------------------------- scatter
// One Philox call per scattering: u0 picks the mechanism against the
// cumulative table row of the current energy bin (lower bin edge; above the
// last entry = self-scattering), u2/u3 the final direction, u1 the next
// flight time -ln(u1)/Gamma0 of the final valley.
template <typename Real, bool NW>
__device__ __forceinline__ void scatter(Part<Real>& q, const DevParams& P, const Phys<Real>* ph,
                                        const Real* tab_s, int nbs, const Real* tab_g, BlockTally* bt,
                                        int e_base)
{
    const U4 r = q.draw();
    const Real u0 = u01<Real>(r.a), u1 = u01<Real>(r.b), u2 = u01<Real>(r.c), u3 = u01<Real>(r.d);
    const int v = q.v;
    const Real k2 = q.kx * q.kx + q.ky * q.ky + q.kz * q.kz;
    const Real E = kane_E(ph->ck[v] * k2, ph->alpha[v]);
    const Real fb = Mth<Real>::floor_(E * Real(P.inv_dE));
    int b;
    if (fb >= Real(P.nb)) {
        b = P.nb - 1;
        tally_cnt(bt, P, q.e, e_base, CNT_OVERFLOW, 1u);
    } else if (fb >= Real(0)) {
        b = int(fb);
    } else {
        b = 0;
        if (!(E == E)) atomicOr(P.err, ERR_NAN);
    }
    const Real* row = (b < nbs) ? tab_s + ((size_t)v * nbs + b) * NM
                                : tab_g + ((size_t)v * P.nb + b) * NM;
    int mech = -1;
    if (u0 < row[NM - 1]) {
#pragma unroll
        for (int m = 0; m < NM; ++m)
            if (mech < 0 && u0 < row[m]) mech = m;
    }
    int vn = v;
    if (mech >= 0) {
        int j = v;
        Real Ep;
        if (mech == 0 || mech == 3) {
            Ep = E;
        } else if (mech == 1) {
            Ep = E + ph->hw_lo;
        } else if (mech == 2) {
            Ep = E - ph->hw_lo;
        } else {
            j = (mech - 4) >> 1;
            Ep = E + ((mech & 1) == 0 ? ph->hw_iv : -ph->hw_iv) - (ph->Ec[j] - ph->Ec[v]);
        }
        if (!(Ep > Real(0))) {
            tally_cnt(bt, P, q.e, e_base, CNT_REJECT, 1u);
            mech = -1;
        } else {
            const Real km = Mth<Real>::sqrt_(k2);
            const Real kp = Mth<Real>::sqrt_(Ep * (Real(1) + ph->alpha[j] * Ep) / ph->ck[j]);
            Real ct;
            bool rel = true;
            if (mech == 0) {
                // Brooks-Herring: P(cos) ~ 1 / (2k^2 (1 - cos) + beta^2)^2
                ct = Real(1) - Real(2) * u2 / (Real(1) + Real(4) * k2 * (Real(1) - u2) / ph->beta2);
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
            Mth<Real>::sincospi_(Real(2) * u3, &sp, &cp);
            const Real st = Mth<Real>::sqrt_(fmax(Real(0), Real(1) - ct * ct));
            Real dx, dy, dz;
            if (rel) {
                // frame of k: branchless orthonormal basis (Duff et al., JCGT 2017)
                Real nx = 0, ny = 0, nz = 1;
                if (km > Real(0)) {
                    nx = q.kx / km;
                    ny = q.ky / km;
                    nz = q.kz / km;
                }
                const Real sg = copysign(Real(1), nz);
                const Real aa = Real(-1) / (sg + nz);
                const Real bb = nx * ny * aa;
                const Real e1x = Real(1) + sg * nx * nx * aa, e1y = sg * bb, e1z = -sg * nx;
                const Real e2x = bb, e2y = sg + ny * ny * aa, e2z = -ny;
                dx = st * cp * e1x + st * sp * e2x + ct * nx;
                dy = st * cp * e1y + st * sp * e2y + ct * ny;
                dz = st * cp * e1z + st * sp * e2z + ct * nz;
            } else {
                dx = st * cp;
                dy = st * sp;
                dz = ct;
            }
            q.kx = kp * dx;
            q.ky = kp * dy;
            q.kz = kp * dz;
            vn = j;
            const int w = q.e - e_base;
            if (w >= 0 && w < WE)
                atomicAdd(&bt->ev[w][v * NM + mech], 1u);
            else
                atomicAdd(&P.events[((size_t)q.e * NV + v) * NM + mech], 1ull);
            if (NW && mech != 0 && mech != 3) {
                const int c = cell_of<Real>(P, q.x, q.y, q.z);
                // net emission: mech 1 absorbs, 2 emits; 4+2j absorbs, 5+2j emits
                const long long d = (mech == 1) ? -1 : (mech == 2 ? 1 : ((mech & 1) ? 1 : -1));
                atomicAdd(reinterpret_cast<unsigned long long*>(
                              &P.heat[((size_t)q.e * P.ncell + c) * 2 + (mech <= 2 ? 0 : 1)]),
                          (unsigned long long)d);
            }
        }
    }
    if (mech < 0) tally_cnt(bt, P, q.e, e_base, CNT_SELF0 + v, 1u);
    q.v = vn;
    q.tr = -Mth<Real>::log_(u1) * ph->inv_g0[vn];
}

// -------------------------------------------------------------- flight
// One thread per particle slot; n_steps time steps fused.  Tables of a
// single table set are staged in shared memory for bins [0, nb_smem).
template <typename Real, bool NW>
__global__ void __launch_bounds__(512) k_flight(const DevParams P, int n_steps, int count_charge)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int nbs = P.nb_smem;
    Real* tab_s = reinterpret_cast<Real*>(sm);
    size_t tbytes = ((size_t)NV * nbs * NM * sizeof(Real) + 15) & ~size_t(15);
    BlockTally* bt = reinterpret_cast<BlockTally*>(sm + tbytes);
    const Real* tab_all = static_cast<const Real*>(P.table);
    for (int i = threadIdx.x; i < NV * nbs * NM; i += blockDim.x) {
        const int v = i / (nbs * NM), rr = i - v * nbs * NM;
        tab_s[i] = tab_all[(size_t)v * P.nb * NM + rr];
    }
    for (int i = threadIdx.x; i < (int)(sizeof(BlockTally) / 4); i += blockDim.x)
        reinterpret_cast<unsigned int*>(bt)[i] = 0u;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int e_base = int(P.tag[(int64_t)blockIdx.x * blockDim.x] >> 8);
    __syncthreads();

    Acc<Real> s_v[3], s_E, s_Et;
    unsigned int n_v[NV] = {0u, 0u, 0u};
    int e = e_base;
    bool live = false;
    if (p < P.n_slots) {
        const uint32_t tg = P.tag[p];
        e = int(tg >> 8);
        live = (tg & 0xFFu) != DEAD;
        if (live) {
            Part<Real> q;
            q.e = e;
            q.v = int(tg & 0xFFu);
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
            q.id = P.id[p];
            q.seed = P.seed[e];
            const int ts = P.tabset[e];
            const Phys<Real>* ph = static_cast<const Phys<Real>*>(P.phys) + ts;
            const Real* tab_g = tab_all + (size_t)ts * NV * P.nb * NM;
            const int nbs_e = (P.n_tab == 1) ? nbs : 0;
            const Real dt = Real(P.dt);
            Real a[3], ah[3] = {0, 0, 0}, inv_hF = 0;
            if (!NW) {
                const Real* ab = static_cast<const Real*>(P.acc_bulk) + 3 * (size_t)e;
                a[0] = ab[0];
                a[1] = ab[1];
                a[2] = ab[2];
            }
            for (int s = 0; s < n_steps; ++s) {
                if (NW) {
                    const int c = cell_of<Real>(P, q.x, q.y, q.z);
                    const Real* ac = static_cast<const Real*>(P.acc_cell) + 3 * ((size_t)e * P.ncell + c);
                    a[0] = ac[0];
                    a[1] = ac[1];
                    a[2] = ac[2];
                    const Real am = Mth<Real>::sqrt_(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                    if (am > Real(0)) {
                        ah[0] = a[0] / am;
                        ah[1] = a[1] / am;
                        ah[2] = a[2] / am;
                        inv_hF = Real(1) / (Real(kHbarEVfs) * am);
                    } else {
                        inv_hF = Real(0);
                    }
                }
                Real tleft = dt;
                bool died = false;
                for (int it = 0;; ++it) {
                    if (it >= MAX_FLIGHTS_PER_STEP) {
                        atomicOr(P.err, ERR_FLIGHTS);
                        break;
                    }
                    if (q.tr >= tleft) {
                        drift<Real, NW>(q, ph, a, ah, inv_hF, tleft);
                        q.tr -= tleft;
                        if (NW) died = walls(q, P, bt, e_base);
                        break;
                    }
                    drift<Real, NW>(q, ph, a, ah, inv_hF, q.tr);
                    tleft -= q.tr;
                    if (NW && walls(q, P, bt, e_base)) {
                        died = true;
                        break;
                    }
                    scatter<Real, NW>(q, P, ph, tab_s, nbs_e, tab_g, bt, e_base);
                }
                if (died) {
                    live = false;
                    break;
                }
                const int v = q.v;
                const Real E = kane_E(ph->ck[v] * (q.kx * q.kx + q.ky * q.ky + q.kz * q.kz), ph->alpha[v]);
                const Real f = ph->vk[v] / (Real(1) + Real(2) * ph->alpha[v] * E);
                s_v[0].add(f * q.kx);
                s_v[1].add(f * q.ky);
                s_v[2].add(f * q.kz);
                s_E.add(E);
                s_Et.add(E + ph->Ec[v]);
                n_v[v] += 1u;
            }
            store<Real>(P, p, q, NW);
            P.tag[p] = (uint32_t(e) << 8) | (live ? uint32_t(q.v) : DEAD);
            if (NW && count_charge && live) atomicAdd(&P.charge[(size_t)e * P.ncell + cell_of<Real>(P, q.x, q.y, q.z)], 1);
        }
    }
    // ---- block reduction of the per-step samples
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    double vals[NSUM] = {s_v[0].value(), s_v[1].value(), s_v[2].value(), s_E.value(), s_Et.value(), 0.0, 0.0, 0.0};
    unsigned int cnts[NV + 1] = {n_v[0], n_v[1], n_v[2], n_v[0] + n_v[1] + n_v[2]};
    const int e0 = __shfl_sync(FULL, e, 0);
    const bool uniform = __all_sync(FULL, e == e0);
    if (uniform) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int i = 0; i < 5; ++i) vals[i] += __shfl_xor_sync(FULL, vals[i], o);
#pragma unroll
            for (int i = 0; i < NV + 1; ++i) cnts[i] += __shfl_xor_sync(FULL, cnts[i], o);
        }
    }
    if (!uniform || lane == 0) {
        if (cnts[NV] > 0u) {
            const int w = e - e_base;
            if (w >= 0 && w < WE) {
                for (int i = 0; i < 5; ++i) atomicAdd(&bt->sums[w][i], vals[i]);
                for (int i = 0; i < NV; ++i) atomicAdd(&bt->cnt[w][CNT_V0 + i], cnts[i]);
                atomicAdd(&bt->cnt[w][CNT_SAMPLES], cnts[NV]);
            } else {
                for (int i = 0; i < 5; ++i) atomicAdd(&P.sums[(size_t)e * NSUM + i], vals[i]);
                for (int i = 0; i < NV; ++i)
                    atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_V0 + i], (unsigned long long)cnts[i]);
                atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_SAMPLES], (unsigned long long)cnts[NV]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < WE * NV * NM; i += blockDim.x) {
        const int w = i / (NV * NM), j = i - w * NV * NM;
        const unsigned int n = bt->ev[w][j];
        if (n && e_base + w < P.n_ens) atomicAdd(&P.events[(size_t)(e_base + w) * NV * NM + j], (unsigned long long)n);
    }
    for (int i = threadIdx.x; i < WE * NCNT; i += blockDim.x) {
        const int w = i / NCNT, j = i - w * NCNT;
        const unsigned int n = bt->cnt[w][j];
        if (n && e_base + w < P.n_ens) atomicAdd(&P.cnt[(size_t)(e_base + w) * NCNT + j], (unsigned long long)n);
    }
    for (int i = threadIdx.x; i < WE * NSUM; i += blockDim.x) {
        const int w = i / NSUM, j = i - w * NSUM;
        const double x = bt->sums[w][j];
        if (x != 0.0 && e_base + w < P.n_ens) atomicAdd(&P.sums[(size_t)(e_base + w) * NSUM + j], x);
    }
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
    q.id = id;
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
// (y, z) order) up to n_target electrons, taking free ids of the ensemble in
// increasing order.  One block per ensemble; dynamic shared memory holds the
// deficit prefix sums (2 ny nz + 1 ints) and a scan buffer (blockDim ints).
template <typename Real>
__global__ void __launch_bounds__(256) k_inject(const DevParams P)
{
    extern __shared__ int shi[];
    const int e = blockIdx.x;
    const int nface = P.ny * P.nz, ncon = 2 * nface;
    int* pre = shi;
    int* scan = shi + ncon + 1;
    if (threadIdx.x == 0) {
        int acc = 0;
        pre[0] = 0;
        for (int t = 0; t < ncon; ++t) {
            const int side = t / nface, rem = t - side * nface;
            const int ix = side ? P.nx - 1 : 0;
            const int cell = ix * nface + rem;
            const int need = P.n_target[e] - P.charge[(size_t)e * P.ncell + cell];
            acc += need > 0 ? need : 0;
            pre[t + 1] = acc;
        }
    }
    __syncthreads();
    const int D = pre[ncon];
    if (D == 0) return;
    const int64_t words = (P.ens_cap[e] + 31) / 32;
    uint32_t* bits = P.dead_bits + P.bits_off[e];
    const int64_t per = (words + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = (int64_t)threadIdx.x * per;
    const int64_t w1 = w0 + per < words ? w0 + per : words;
    int mine = 0;
    for (int64_t w = w0; w < w1; ++w) mine += __popc(bits[w]);
    // block exclusive scan
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int x = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += x;
        __syncthreads();
    }
    const int total = scan[blockDim.x - 1];
    int rank = scan[threadIdx.x] - mine;
    if (threadIdx.x == 0 && total < D)
        atomicAdd(&P.cnt[(size_t)e * NCNT + CNT_STARVED], (unsigned long long)(D - total));
    const Phys<Real>* ph = static_cast<const Phys<Real>*>(P.phys) + P.tabset[e];
    const Real len3[3] = {Real(P.dx), Real(P.dy), Real(P.dz)};
    for (int64_t w = w0; w < w1 && rank < D; ++w) {
        uint32_t word = bits[w];
        uint32_t clear = 0u;
        while (word && rank < D) {
            const int bit = __ffs(word) - 1;
            word &= word - 1u;
            const uint32_t id = uint32_t(w * 32 + bit);
            // contact t with pre[t] <= rank < pre[t + 1]
            int lo = 0, hi = ncon - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= rank) lo = mid;
                else hi = mid - 1;
            }
            const int t = lo;
            const int side = t / nface, rem = t - side * nface;
            const int ix = side ? P.nx - 1 : 0, iy = rem / P.nz, iz = rem - iy * P.nz;
            const int64_t slot = P.slot_of_id[P.ens_off[e] + id];
            Part<Real> q;
            q.e = e;
            q.id = id;
            q.seed = P.seed[e];
            q.ctr = P.ctr[slot];
            const Real lo3[3] = {Real(ix * P.dx), Real(iy * P.dy), Real(iz * P.dz)};
            new_electron<Real, true>(q, ph, lo3, len3, P.err);
            store<Real>(P, slot, q, true);
            P.tag[slot] = uint32_t(e) << 8;
            atomicAdd(&P.charge[(size_t)e * P.ncell + ix * nface + rem], 1);
            atomicAdd(&P.cnt[(size_t)e * NCNT + (side ? CNT_DRN_IN : CNT_SRC_IN)], 1ull);
            clear |= 1u << bit;
            ++rank;
        }
        bits[w] &= ~clear;
    }
}

// --------------------------------------------------------------- launch
template <typename Real>
size_t flight_smem_bytes(int nb_smem)
{
    return (((size_t)NV * nb_smem * NM * sizeof(Real) + 15) & ~size_t(15)) + sizeof(BlockTally);
}

template <typename Real>
cudaError_t flight_set_smem(size_t bytes)
{
    cudaError_t a = cudaFuncSetAttribute(k_flight<Real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (a != cudaSuccess) return a;
    return cudaFuncSetAttribute(k_flight<Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename Real>
void launch_flight(const DevParams& P, bool nw, int n_steps, int count_charge, int block, cudaStream_t st)
{
    if (P.n_slots <= 0) return;
    const unsigned grid = (unsigned)((P.n_slots + block - 1) / block);
    const size_t smem = flight_smem_bytes<Real>(P.nb_smem);
    if (nw)
        k_flight<Real, true><<<grid, block, smem, st>>>(P, n_steps, count_charge);
    else
        k_flight<Real, false><<<grid, block, smem, st>>>(P, n_steps, count_charge);
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
    const int block = 256;
    const size_t smem = sizeof(int) * (2 * P.ny * P.nz + 1 + block);
    k_inject<Real><<<P.n_ens, block, smem, st>>>(P);
}

}  // namespace emc
