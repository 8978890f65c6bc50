// Phonon Monte Carlo of the transistor region (include/emc.h,
// emc_phonon_solve): energy-based deviational phonon bundles (Peraud and
// Hadjiconstantinou, 2011) of the paper's phonon model (three identical sine
// branches, the relaxation times of the phonon-model paragraph, Table II,
// optionally Eq. (1) and a boundary term; the interface of Eq. (2)) flying
// through the subcell grid of the half wire.  Every bundle carries the same
// share of the power sum |q| V, with the sign of the heat of the subcell it
// starts in (negative heat: a phonon deficit); the signed time the bundles
// spend in a subcell is its deviational energy and so its temperature rise.
//
// One thread per bundle at a time; a thread that finishes a bundle takes the
// next one from a global counter, so the warps stay full until the work
// runs out.  Per segment the bundle flies to the nearest of: its next
// scattering (the optical depth left over the subcell's rate), a face of its
// subcell (then the neighbouring subcell, with its own rate table), a face of
// the domain (specular, rough, isothermal or interface).  Each lane first
// runs the segments that need no random numbers (subcell, specular and
// isothermal faces: a few dozen instructions each) up to its next
// scattering or rough / interface face; the draws and new directions of
// those events, and the emissions of new bundles, then run with most lanes
// of the warp together instead of once per segment for the few lanes that
// happen to scatter in it.  Residence times,
// scatterings and emissions are tallied per subcell in shared memory (time
// as a 64-bit two's-complement fixed-point count of 2^-24 ps, so the sums do
// not depend on the order of the additions) and added to global memory at
// the end.
//
// Random numbers: Philox4x32-10 keyed by (seed, bundle id), counter words
// (n, 0, 0, 1) (the electrons use word 3 = 0), n = 0, 1, ... per bundle:
//   emission: call 0 -> subcell, position (x, y, z) in it; call 1 -> bin,
//             cos(theta) = 2u - 1, phi = 2 pi u, optical depth -ln u;
//   scattering: bin, cos(theta), phi, optical depth;
//   rough or interface face: specular (u < p) or transmitted (u < tau12),
//             then a cosine-law direction (cos(theta) = sqrt(u), phi = 2 pi u).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace emc {

enum { PH_SPECULAR = 0, PH_ROUGH = 1, PH_ISOTHERMAL = 2, PH_INTERFACE = 3 };
constexpr double kPhTimeScale = 16777216.0;  // fixed-point residence: 2^24 per ps

struct PhParams {
    int nx, ny, nz, ncell, nb, pad_;
    double hx, hy, hz;             // subcell edges, nm
    const void* vg;                // Real[nb] group velocity, nm/ps
    const void* rate;              // Real[nt][nb] 1/tau, 1/ps
    const void* cdf;               // Real[nt][nb] cumulative of C / tau (last 1)
    const int* tix;                // [C] rate table of each subcell
    const void* cell_cdf;          // Real[C] cumulative |heat| of the subcells (last 1)
    const int* cell_neg;           // [C] 1 where the heat is negative
    const void* tau12;             // Real[nb] interface transmissivity
    int face[6];                   // x=0, x=Lx, y=0, y=Ly, z=0, z=Lz
    double p_spec[6];
    uint32_t seed, pad2_;
    long long n_bundles, first, max_segments;
    unsigned long long* next;      // bundles handed out
    unsigned long long* t_res;     // [C] fixed-point residence time
    unsigned long long* scat;      // [C]
    unsigned long long* emit;      // [C]
    unsigned long long* out;       // [8]: absorbed per face (6), segments, capped
    int* err;                      // device error word (checked build: ERR_BOUNDS)
    int nt, pad3_;                 // rate tables
};

template <typename Real>
struct PhM;
template <>
struct PhM<float> {
    static __device__ __forceinline__ float neglog(float u) { return fmaxf(0.f, -__logf(u)); }
    // sin and cos of 2 pi u, u in (0,1): the hardware approximation at
    // 2 pi (u - 1/2) in (-pi, pi), negated
    static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c)
    {
        float ss, cc;
        __sincosf(6.283185307179586f * (u - 0.5f), &ss, &cc);
        *s = -ss;
        *c = -cc;
    }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    // a 32-bit conversion where it fits (under 256 ps): the 64-bit one runs
    // on the double-precision pipe
    static __device__ __forceinline__ unsigned long long fixed(float t)
    {
        const float x = t * float(kPhTimeScale);
        return x < 4.0e9f ? (unsigned long long)__float2uint_rn(x) : __float2ull_rn(x);
    }
};
template <>
struct PhM<double> {
    static __device__ __forceinline__ double neglog(double u) { return -log(u); }
    static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ unsigned long long fixed(double t) { return __double2ull_rn(t * kPhTimeScale); }
};

// Products, sums and quotients of the flight arithmetic.  In the parity
// build every operation is rounded by itself (no fused multiply-add, IEEE
// division), as the oracle rounds it: a bundle that grazes a subcell face
// splits its time between the two subcells at a point that a one-ulp
// difference can move visibly.  The production build lets the compiler fuse
// products and sums, divides with the hardware approximation and times the
// faces with reciprocals kept per direction (ph_faces_ahead).
template <typename Real>
struct PhA {
    static __device__ __forceinline__ Real mul(Real a, Real b) { return a * b; }
    static __device__ __forceinline__ Real add(Real a, Real b) { return a + b; }
    static __device__ __forceinline__ Real sub(Real a, Real b) { return a - b; }
    static __device__ __forceinline__ Real div(Real a, Real b) { return __fdividef(a, b); }
};
template <>
struct PhA<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

// a fixed-point time, negated (two's complement) for a negative bundle
__device__ __forceinline__ unsigned long long ph_signed(unsigned long long t, bool neg) { return neg ? 0ull - t : t; }

// smallest i in [0, n) with cdf[i] > u
template <typename Real>
__device__ __forceinline__ int ph_inverse_cdf(const Real* cdf, int n, Real u)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) > u) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

struct PhStream {
    uint32_t seed, id;
    uint32_t n;
    __device__ __forceinline__ U4 draw()
    {
        U4 c{n, 0u, 0u, 1u};
        ++n;
        return philox10(c, seed, id);
    }
};

template <typename Real>
__device__ __forceinline__ void ph_isotropic(Real u1, Real u2, Real& dx, Real& dy, Real& dz)
{
    using A = PhA<Real>;
    const Real ct = A::sub(A::mul(Real(2), u1), Real(1));
    const Real st = PhM<Real>::sqrt_(fmax(Real(0), A::sub(Real(1), A::mul(ct, ct))));
    Real s, c;
    PhM<Real>::sincos2pi(u2, &s, &c);
    dx = st * c;
    dy = st * s;
    dz = ct;
}

// cosine-law direction into the domain through face f (axis f/2, low face
// for even f); tangent axes (axis+1) % 3 and (axis+2) % 3
template <typename Real>
__device__ __forceinline__ void ph_lambert(int f, Real u1, Real u2, Real d[3])
{
    const int a = f >> 1;
    const Real ct = PhM<Real>::sqrt_(u1), st = PhM<Real>::sqrt_(Real(1) - u1);
    Real s, c;
    PhM<Real>::sincos2pi(u2, &s, &c);
    const Real n = (f & 1) ? -ct : ct;
    const Real t1 = st * c, t2 = st * s;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int rel = (k - a + 3) % 3;  // 0: normal, 1: first tangent, 2: second
        d[k] = rel == 0 ? n : (rel == 1 ? t1 : t2);
    }
}


// Production build: per axis the coordinate of the subcell face ahead and
// the reciprocal of the velocity component, set whenever the direction, the
// frequency bin or the subcell changes, so that a flight segment needs no
// division for the faces (a zero component gives an infinite reciprocal and
// a time that is never the earliest).
template <typename Real>
__device__ __forceinline__ void ph_faces_ahead(Real v, const Real d[3], const int ix[3], const Real h[3], Real inv[3],
                                               Real bnd[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        inv[a] = __fdividef(Real(1), v * d[a]);
        bnd[a] = Real(ix[a] + (d[a] > Real(0) ? 1 : 0)) * h[a];
    }
}

// Dynamic shared memory: t_res (u64) [C], then scatterings and emissions
// (u32) [C] each.
template <typename Real>
__global__ void __launch_bounds__(256) k_phonon(const PhParams P)
{
    extern __shared__ unsigned long long ph_sh[];
    const int C = P.ncell;
    unsigned long long* s_t = ph_sh;
    unsigned int* s_scat = reinterpret_cast<unsigned int*>(ph_sh + C);
    unsigned int* s_emit = s_scat + C;
    __shared__ unsigned long long s_out[8];
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        s_t[i] = 0ull;
        s_scat[i] = 0u;
        s_emit[i] = 0u;
    }
    if (threadIdx.x < 8) s_out[threadIdx.x] = 0ull;
    __syncthreads();

    const Real* vg = static_cast<const Real*>(P.vg);
    const Real* rate = static_cast<const Real*>(P.rate);
    const Real* cdf = static_cast<const Real*>(P.cdf);
    const Real* ccdf = static_cast<const Real*>(P.cell_cdf);
    const Real* tau12 = static_cast<const Real*>(P.tau12);
    const Real h[3] = {Real(P.hx), Real(P.hy), Real(P.hz)};
    const int nc[3] = {P.nx, P.ny, P.nz};
    const int nb = P.nb;
    const Real INF = Real(INFINITY);
    using A = PhA<Real>;

    unsigned long long n_seg = 0, n_cap = 0;
    // Per lane: ev = 3 wants a new bundle, 1 a scattering (or, right after
    // an emission, the first frequency and direction), 2 a rough or
    // interface face f; 0 flies.  The whole warp runs the loop in step: each
    // round the flying lanes run one segment, and the pending events run
    // (one draw each) once at least half of the lanes with work wait.
    bool neg = false, done = false, fresh = false;
    int ev = 3, f = 0;
    PhStream st{P.seed, 0u, 0u};
    Real p[3], d[3], depth = Real(0);
    Real inv[3] = {Real(0), Real(0), Real(0)}, bnd[3] = {Real(0), Real(0), Real(0)};  // production build
    constexpr bool kFast = std::is_same<Real, float>::value;
    int ix[3] = {0, 0, 0}, c = 0, b = 0;
    long long seg = 0;
    for (;;) {
        if (!done && ev == 0) {
            // one flight segment (needs no random numbers)
            if (seg >= P.max_segments) {
                ++n_cap;
                ev = 3;
            } else {
                ++seg;
                ++n_seg;
                EMC_CHECK(P.err, c >= 0 && c < C && b >= 0 && b < nb && ix[0] >= 0 && ix[0] < nc[0] && ix[1] >= 0 &&
                                     ix[1] < nc[1] && ix[2] >= 0 && ix[2] < nc[2] && __ldg(P.tix + c) < P.nt);
                const Real v = __ldg(vg + b);
                const Real rr = __ldg(rate + (size_t)__ldg(P.tix + c) * nb + b);
                // time to the faces of the subcell, the earliest axis first
                int ax = 0;
                Real t_exit = INF;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Real ta = INF;
                    if constexpr (kFast) {
                        ta = (bnd[a] - p[a]) * inv[a];  // NaN only for a zero component: never taken
                    } else {
                        if (d[a] > Real(0)) ta = A::div(A::sub(A::mul(Real(ix[a] + 1), h[a]), p[a]), A::mul(v, d[a]));
                        else if (d[a] < Real(0)) ta = A::div(A::sub(A::mul(Real(ix[a]), h[a]), p[a]), A::mul(v, d[a]));
                    }
                    if (ta < Real(0)) ta = Real(0);
                    if (ta < t_exit) {
                        t_exit = ta;
                        ax = a;
                    }
                }
                const Real t_scat = rr > Real(0) ? A::div(depth, rr) : INF;
                const bool scat = t_scat < t_exit;
                const Real t = scat ? t_scat : t_exit;
#pragma unroll
                for (int a = 0; a < 3; ++a) p[a] = A::add(p[a], A::mul(A::mul(v, d[a]), t));
                atomicAdd(&s_t[c], ph_signed(PhM<Real>::fixed(t), neg));
                if (scat) {
                    ev = 1;
                } else {
                    depth = A::sub(depth, A::mul(rr, t_exit));
                    if (depth < Real(0)) depth = Real(0);
                    // onto the face of axis ax (constant indices only: registers)
                    bool up = false, inside = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (a == ax) {
                            up = d[a] > Real(0);
                            p[a] = A::mul(Real(ix[a] + (up ? 1 : 0)), h[a]);
                            const int nxt = ix[a] + (up ? 1 : -1);
                            inside = nxt >= 0 && nxt < nc[a];
                            if (inside) {
                                ix[a] = nxt;
                                if constexpr (kFast) bnd[a] = Real(nxt + (up ? 1 : 0)) * h[a];
                            }
                        }
                    }
                    if (inside) {
                        c = (ix[0] * P.ny + ix[1]) * P.nz + ix[2];
                    } else {
                        f = 2 * ax + (up ? 1 : 0);
                        const int kind = P.face[f];
                        if (kind == PH_ISOTHERMAL) {
                            atomicAdd(&s_out[f], 1ull);
                            ev = 3;
                        } else if (kind == PH_SPECULAR) {
#pragma unroll
                            for (int a = 0; a < 3; ++a)
                                if (a == ax) {
                                    d[a] = -d[a];
                                    if constexpr (kFast) {
                                        inv[a] = -inv[a];
                                        bnd[a] = Real(ix[a] + (up ? 0 : 1)) * h[a];
                                    }
                                }
                        } else {
                            ev = 2;
                        }
                    }
                }
            }
        }
        const unsigned pend = __ballot_sync(0xFFFFFFFFu, !done && ev != 0);
        const unsigned live = __ballot_sync(0xFFFFFFFFu, !done);
        if (live == 0u) break;
        if (2 * __popc(pend) < __popc(live)) continue;
        // the pending events
        // the lanes that want a new bundle take consecutive ids with one
        // atomic per warp
        const unsigned want = __ballot_sync(0xFFFFFFFFu, !done && ev == 3);
        unsigned long long base = 0ull;
        if (want) {
            if ((threadIdx.x & 31) == __ffs(want) - 1) base = atomicAdd(P.next, (unsigned long long)__popc(want));
            base = __shfl_sync(0xFFFFFFFFu, base, __ffs(want) - 1);
        }
        if (!done && ev == 3) {
            const unsigned long long i = base + __popc(want & ((1u << (threadIdx.x & 31)) - 1u));
            if (i >= (unsigned long long)P.n_bundles) {
                done = true;
            } else {
                st.id = uint32_t(P.first + (long long)i);
                st.n = 0u;
                const U4 r = st.draw();
                c = ph_inverse_cdf<Real>(ccdf, C, u01<Real>(r.a));
                ix[0] = c / (P.ny * P.nz);
                ix[1] = (c / P.nz) % P.ny;
                ix[2] = c % P.nz;
                p[0] = A::mul(A::add(Real(ix[0]), u01<Real>(r.b)), h[0]);
                p[1] = A::mul(A::add(Real(ix[1]), u01<Real>(r.c)), h[1]);
                p[2] = A::mul(A::add(Real(ix[2]), u01<Real>(r.d)), h[2]);
                atomicAdd(&s_emit[c], 1u);
                neg = __ldg(P.cell_neg + c) != 0;
                seg = 0;
                fresh = true;
                ev = 1;
            }
        }
        if (!done && (ev == 1 || ev == 2)) {
            const U4 r = st.draw();
            const Real u0 = u01<Real>(r.a);
            if (ev == 1) {
                // a scattering, or the first flight of a new bundle
                if (!fresh) atomicAdd(&s_scat[c], 1u);
                fresh = false;
                b = ph_inverse_cdf<Real>(cdf + (size_t)__ldg(P.tix + c) * nb, nb, u0);
                ph_isotropic<Real>(u01<Real>(r.b), u01<Real>(r.c), d[0], d[1], d[2]);
                depth = PhM<Real>::neglog(u01<Real>(r.d));
                if constexpr (kFast) ph_faces_ahead<Real>(__ldg(vg + b), d, ix, h, inv, bnd);
                ev = 0;
            } else {
                const int ax = f >> 1;
                bool diffuse = true;
                ev = 0;
                if (P.face[f] == PH_INTERFACE) {
                    if (u0 < __ldg(tau12 + b)) {
                        atomicAdd(&s_out[f], 1ull);
                        diffuse = false;
                        ev = 3;
                    }
                } else if (u0 < Real(P.p_spec[f])) {  // rough: specular part
                    diffuse = false;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (a == ax) d[a] = -d[a];
                }
                if (diffuse) ph_lambert<Real>(f, u01<Real>(r.b), u01<Real>(r.c), d);
                if constexpr (kFast) {
                    if (ev == 0) ph_faces_ahead<Real>(__ldg(vg + b), d, ix, h, inv, bnd);
                }
            }
        }
    }
    atomicAdd(&s_out[6], n_seg);
    atomicAdd(&s_out[7], n_cap);
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        if (s_t[i]) atomicAdd(P.t_res + i, s_t[i]);
        if (s_scat[i]) atomicAdd(P.scat + i, (unsigned long long)s_scat[i]);
        if (s_emit[i]) atomicAdd(P.emit + i, (unsigned long long)s_emit[i]);
    }
    if (threadIdx.x < 8 && s_out[threadIdx.x]) atomicAdd(P.out + threadIdx.x, s_out[threadIdx.x]);
}

template <typename Real>
inline size_t ph_smem_bytes(int ncell)
{
    return (size_t)ncell * (sizeof(unsigned long long) + 2 * sizeof(unsigned int));
}

}  // namespace emc
