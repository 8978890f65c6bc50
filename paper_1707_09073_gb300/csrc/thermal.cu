// Thermal side of the electrothermal loop (include/emc.h, emc_thermal_*):
// steady Fourier conduction on the subcell grid of the half nanowire with
// kappa(T) from the phonon model of the paper (three identical sine-shaped
// acoustic branches, 1/tau = A w^4 + B1 w^2 T exp(-B2/T), Table II) and a
// boundary-scattering length (the size-modified mean free paths).
//
// Per subcell: sum over faces g_f (T_c - T_n) + boundary terms g_b (T_c -
// T_sink) = q_c, with g_f = harmonic-mean kappa / h^2, the contact faces
// (x = 0, x = L) at T_sink half a cell away, the bottom face (z = 0) through
// a conductance h_bottom in series with the half cell, and every other face
// adiabatic.  kappa(T) is handled by Picard iteration; each linear solve is
// FP64 conjugate gradients.  One block per ensemble, everything in shared
// memory.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/emc.h"
#include "common.cuh"

namespace emc {
// accessors of the context (defined in emc.cu)
cudaStream_t ctx_stream(emc_ctx* ctx);
int ctx_grid(emc_ctx* ctx, int* nx, int* ny, int* nz, double* Lx, double* Ly, double* Lz, int* n_ens);
emc_status ctx_fail(emc_ctx* ctx, emc_status s, const char* msg);
void ctx_count_launches(emc_ctx* ctx, int64_t n);
}  // namespace emc

using namespace emc;

namespace {

constexpr double kTLo = 150.0, kTStep = 0.5;
constexpr int kNT = 2701;  // 150 .. 1500 K
constexpr int kMaxThermalCells = 2048;

// kappa(T) of the GaN column of Table II on the grid above (midpoint rule in
// the wave vector, 4000 points)
std::vector<double> kappa_table_build(const emc_thermal_config& tc)
{
    const double q0 = tc.k0_per_m, wm = tc.omega_max_rad_s;
    std::vector<double> out(kNT);
    const int nq = 4000;
    for (int t = 0; t < kNT; ++t) {
        const double T = kTLo + kTStep * t;
        double acc = 0.0;
        for (int i = 0; i < nq; ++i) {
            const double q = (i + 0.5) * q0 / nq;
            const double w = wm * std::sin(kPi * q / (2.0 * q0));
            const double vg = wm * kPi / (2.0 * q0) * std::cos(kPi * q / (2.0 * q0));
            const double x = kHbar * w / (kKB * T);
            const double em1 = std::expm1(x);
            const double dndT = x * std::exp(x) / (em1 * em1) / T;
            double rate = tc.A_s3 * w * w * w * w + tc.B1_s_per_K * w * w * T * std::exp(-tc.B2_K / T);
            if (tc.L_boundary > 0.0) rate += vg / tc.L_boundary;
            acc += kHbar * w * dndT * vg * vg / rate * q * q / (2.0 * kPi * kPi);
        }
        out[t] = acc * q0 / nq;
    }
    return out;
}

// tables are cached per phonon parameter set (the quadrature costs ~0.3 s)
std::vector<double> kappa_table(const emc_thermal_config& tc)
{
    static std::mutex mu;
    static std::map<std::tuple<double, double, double, double, double, double>, std::vector<double>> cache;
    const auto key = std::make_tuple(tc.k0_per_m, tc.omega_max_rad_s, tc.A_s3, tc.B1_s_per_K, tc.B2_K, tc.L_boundary);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, kappa_table_build(tc)).first;
    return it->second;
}

struct TGeo {
    int nx, ny, nz, n;
    double hx, hy, hz, T_sink, h_bottom, tol;
    int max_picard, max_cg;
};

__device__ __forceinline__ double kap_at(const double* tab, double T)
{
    double f = (T - kTLo) / kTStep;
    f = fmin(fmax(f, 0.0), double(kNT - 1) - 1e-9);
    const int i = int(f);
    const double a = f - i;
    return tab[i] * (1.0 - a) + tab[i + 1] * a;
}

// y = A(kappa) x on the grid; bnd[c] receives the boundary conductance sum
__device__ void apply(const TGeo& G, const double* kap, const double* x, double* y, double* bnd)
{
    for (int c = threadIdx.x; c < G.n; c += blockDim.x) {
        const int i = c / (G.ny * G.nz), j = (c / G.nz) % G.ny, l = c % G.nz;
        const double kc = kap[c], xc = x[c];
        double acc = 0.0, gb = 0.0;
        auto face = [&](int nb, double h) {
            const double g = 2.0 * kc * kap[nb] / (kc + kap[nb]) / (h * h);
            acc += g * (xc - x[nb]);
        };
        if (i > 0) face(c - G.ny * G.nz, G.hx); else gb += 2.0 * kc / (G.hx * G.hx);
        if (i < G.nx - 1) face(c + G.ny * G.nz, G.hx); else gb += 2.0 * kc / (G.hx * G.hx);
        if (j > 0) face(c - G.nz, G.hy);
        if (j < G.ny - 1) face(c + G.nz, G.hy);
        if (l > 0) face(c - 1, G.hz); else gb += 1.0 / (G.hz * (G.hz / (2.0 * kc) + 1.0 / G.h_bottom));
        if (l < G.nz - 1) face(c + 1, G.hz);
        y[c] = acc + gb * xc;
        if (bnd) bnd[c] = gb;
    }
}

__device__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ double block_max(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, red[i]);
    return s;
}

// one block per ensemble: Picard over kappa(T), CG for each linear system
__global__ void __launch_bounds__(512) k_thermal(TGeo G, const double* __restrict__ tab, const double* q, double* T,
                                                 int* iters)
{
    extern __shared__ double sh[];
    double* x = sh;
    double* kap = sh + G.n;
    double* r = sh + 2 * G.n;
    double* p = sh + 3 * G.n;
    double* Ap = sh + 4 * G.n;
    __shared__ double red[32];
    const int e = blockIdx.x;
    const double* qe = q + (size_t)e * G.n;
    double* Te = T + (size_t)e * G.n;
    for (int c = threadIdx.x; c < G.n; c += blockDim.x) x[c] = Te[c];
    __syncthreads();
    int pic = 0, total = 0;
    for (; pic < G.max_picard; ++pic) {
        for (int c = threadIdx.x; c < G.n; c += blockDim.x) {
            kap[c] = kap_at(tab, x[c]);
            p[c] = x[c];  // previous Picard iterate
        }
        __syncthreads();
        // r = b - A x with b = q + g_b T_sink
        apply(G, kap, x, Ap, r);
        __syncthreads();
        double rr = 0.0, bb = 0.0;
        for (int c = threadIdx.x; c < G.n; c += blockDim.x) {
            const double b = qe[c] + r[c] * G.T_sink;
            r[c] = b - Ap[c];
            rr += r[c] * r[c];
            bb += b * b;
        }
        rr = block_sum(rr, red);
        bb = block_sum(bb, red);
        // keep the previous iterate in Ap's place for the convergence test
        double* prev = Ap;
        for (int c = threadIdx.x; c < G.n; c += blockDim.x) prev[c] = p[c];
        __syncthreads();
        // CG with direction d (stored in p) and A d in a scratch: reuse kap? no:
        // directions go to p, products to the tail of the buffer
        double* d = p;
        double* Ad = sh + 5 * G.n;
        for (int c = threadIdx.x; c < G.n; c += blockDim.x) d[c] = r[c];
        __syncthreads();
        const double stop = 1e-26 * fmax(bb, 1e-300);
        for (int it = 0; it < G.max_cg && rr > stop; ++it, ++total) {
            apply(G, kap, d, Ad, nullptr);
            __syncthreads();
            double dAd = 0.0;
            for (int c = threadIdx.x; c < G.n; c += blockDim.x) dAd += d[c] * Ad[c];
            dAd = block_sum(dAd, red);
            const double al = rr / dAd;
            double rn = 0.0;
            for (int c = threadIdx.x; c < G.n; c += blockDim.x) {
                x[c] += al * d[c];
                r[c] -= al * Ad[c];
                rn += r[c] * r[c];
            }
            rn = block_sum(rn, red);
            const double be = rn / rr;
            rr = rn;
            for (int c = threadIdx.x; c < G.n; c += blockDim.x) d[c] = r[c] + be * d[c];
            __syncthreads();
        }
        double md = 0.0;
        for (int c = threadIdx.x; c < G.n; c += blockDim.x) md = fmax(md, fabs(x[c] - prev[c]));
        md = block_max(md, red);
        if (md < G.tol) {
            ++pic;
            break;
        }
    }
    for (int c = threadIdx.x; c < G.n; c += blockDim.x) Te[c] = x[c];
    if (threadIdx.x == 0 && iters) {
        iters[2 * e] = pic;
        iters[2 * e + 1] = total;
    }
}

}  // namespace

extern "C" {

emc_status emc_kappa(const emc_thermal_config* tc, const double* T, double* kappa, int32_t n)
{
    if (!tc || n < 0 || (n > 0 && (!T || !kappa))) return EMC_EINVAL;
    const std::vector<double> tab = kappa_table(*tc);
    for (int i = 0; i < n; ++i) {
        double f = (T[i] - kTLo) / kTStep;
        f = std::fmin(std::fmax(f, 0.0), double(kNT - 1) - 1e-9);
        const int k = int(f);
        const double a = f - k;
        kappa[i] = tab[k] * (1.0 - a) + tab[k + 1] * a;
    }
    return EMC_OK;
}

emc_status emc_thermal_solve(emc_ctx* ctx, const emc_thermal_config* tc, const double* q, double* T, int32_t* iters)
{
    if (!ctx || !tc || !q || !T) return EMC_EINVAL;
    int nx, ny, nz, ne;
    double Lx, Ly, Lz;
    if (!ctx_grid(ctx, &nx, &ny, &nz, &Lx, &Ly, &Lz, &ne))
        return ctx_fail(ctx, EMC_ESTATE, "emc_thermal_solve needs the nanowire geometry");
    const int n = nx * ny * nz;
    if (n > kMaxThermalCells) return ctx_fail(ctx, EMC_EINVAL, "emc_thermal_solve: at most 2048 subcells");
    if (!(tc->T_sink > 0) || !(tc->h_bottom > 0) || tc->max_picard <= 0 || tc->max_cg <= 0)
        return ctx_fail(ctx, EMC_EINVAL, "emc_thermal_solve: invalid configuration");
    cudaStream_t st = ctx_stream(ctx);
    const std::vector<double> tab = kappa_table(*tc);
    double *d_tab = nullptr, *d_q = nullptr, *d_T = nullptr;
    int* d_it = nullptr;
    const size_t bytes = sizeof(double) * (size_t)ne * n;
#define TCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return ctx_fail(ctx, EMC_ECUDA, cudaGetErrorString(e_)); \
    } while (0)
    TCK(cudaMallocAsync(&d_tab, sizeof(double) * kNT, st));
    TCK(cudaMallocAsync(&d_q, bytes, st));
    TCK(cudaMallocAsync(&d_T, bytes, st));
    TCK(cudaMallocAsync(&d_it, sizeof(int) * 2 * ne, st));
    TCK(cudaMemcpyAsync(d_tab, tab.data(), sizeof(double) * kNT, cudaMemcpyHostToDevice, st));
    TCK(cudaMemcpyAsync(d_q, q, bytes, cudaMemcpyHostToDevice, st));
    TCK(cudaMemcpyAsync(d_T, T, bytes, cudaMemcpyHostToDevice, st));
    TGeo G{nx, ny, nz, n, Lx / nx, Ly / ny, Lz / nz, tc->T_sink, tc->h_bottom, tc->tol_K, tc->max_picard, tc->max_cg};
    const size_t smem = sizeof(double) * 6 * n;
    TCK(cudaFuncSetAttribute(k_thermal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_thermal<<<ne, 512, smem, st>>>(G, d_tab, d_q, d_T, d_it);
    ctx_count_launches(ctx, 1);
    TCK(cudaGetLastError());
    TCK(cudaMemcpyAsync(T, d_T, bytes, cudaMemcpyDeviceToHost, st));
    if (iters) TCK(cudaMemcpyAsync(iters, d_it, sizeof(int) * 2 * ne, cudaMemcpyDeviceToHost, st));
    TCK(cudaFreeAsync(d_tab, st));
    TCK(cudaFreeAsync(d_q, st));
    TCK(cudaFreeAsync(d_T, st));
    TCK(cudaFreeAsync(d_it, st));
    TCK(cudaStreamSynchronize(st));
#undef TCK
    return EMC_OK;
}

}  // extern "C"
