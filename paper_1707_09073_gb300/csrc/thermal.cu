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
#include <vector>

#include "../../include/emc.h"
#include "common.cuh"
#include "phonon.cuh"
#include "trace.h"

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

// Normalised Fermi-Dirac integral of order 1/2, F(eta) = (2/sqrt(pi))
// int_0^inf sqrt(x) / (1 + e^(x - eta)) dx, with x = t^2 and the midpoint
// rule in t; dF/deta (the order -1/2 integral) from the same points.
void fermi_half(double eta, double* F, double* dF)
{
    const int n = 1200;
    const double tmax = std::sqrt(std::fmax(eta, 0.0) + 80.0), h = tmax / n;
    double acc = 0.0, dacc = 0.0;
    for (int i = 0; i < n; ++i) {
        const double t = (i + 0.5) * h, z = t * t - eta;
        const double occ = z > 0.0 ? std::exp(-z) / (1.0 + std::exp(-z)) : 1.0 / (1.0 + std::exp(z));
        acc += 2.0 * t * t * occ;
        dacc += 2.0 * t * t * occ * (1.0 - occ);
    }
    *F = acc * h * 2.0 / std::sqrt(kPi);
    *dF = dacc * h * 2.0 / std::sqrt(kPi);
}

// Fermi level (J from the band edge) of n electrons per m^3 in a parabolic
// band of DOS mass m_rel m0 at T: n = N_c F_1/2(E_F / kT).  Newton on
// ln F(eta) from the non-degenerate or degenerate limit, kept inside a
// shrinking bracket (bisection when a step leaves it).
double fermi_level(double n, double T, double m_rel)
{
    const double Nc = 2.0 * std::pow(m_rel * kM0 * kKB * T / (2.0 * kPi * kHbar * kHbar), 1.5);
    const double target = std::log(n / Nc);
    double lo = -200.0, hi = 400.0;
    double eta = target < 0.0 ? target : std::pow(0.75 * std::sqrt(kPi) * std::exp(target), 2.0 / 3.0);
    eta = std::fmin(std::fmax(eta, lo), hi);
    for (int it = 0; it < 200; ++it) {
        double F, dF;
        fermi_half(eta, &F, &dF);
        const double g = std::log(F) - target;
        if (g < 0.0) lo = eta;
        else hi = eta;
        double next = eta - g * F / dF;
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (std::fabs(next - eta) < 1e-13 * (1.0 + std::fabs(eta))) {
            eta = next;
            break;
        }
        eta = next;
    }
    return eta * kKB * T;
}

// Phonon-electron scattering rate of Eq. (1) (1/s).  The braces
// hbar w / kT - ln[(1 + e^(a+y)) / (1 + e^(a-y))] (hbar w / kT = 2y) are
// evaluated with ln(1 + e^z) = max(z, 0) + ln(1 + e^-|z|), the 2y cancelling
// exactly, so non-degenerate values (a >> 1) keep their precision.
double tau_e_inv(double w, double T, double E_F, const emc_thermal_config& tc)
{
    const double m = tc.m_e_rel * kM0, v = tc.vg_e_m_s, kT = kKB * T;
    const double Da = tc.Da_eV * kQ;
    const double half = 0.5 * m * v * v;
    const double pre = Da * Da * m * m * m * v / (4.0 * kPi * kHbar * kHbar * kHbar * kHbar * tc.rho_kg_m3) * kT / half;
    const double a = (half - E_F) / kT + (kHbar * w) * (kHbar * w) / (8.0 * m * v * v * kT);
    const double y = kHbar * w / (2.0 * kT);
    auto sp = [](double z) { return std::log1p(std::exp(-std::fabs(z))); };
    double br;
    if (a - y >= 0.0) br = sp(a - y) - sp(a + y);
    else if (a + y <= 0.0) br = 2.0 * y - sp(a + y) + sp(a - y);
    else br = (y - a) - sp(a + y) + sp(a - y);
    return pre * br;
}

// the phonon-electron parameters are either off (n_e = 0) or all positive
bool electrons_ok(const emc_thermal_config& tc)
{
    if (tc.n_e_m3 == 0.0) return true;
    return tc.n_e_m3 > 0.0 && tc.m_e_rel > 0.0 && tc.Da_eV > 0.0 && tc.rho_kg_m3 > 0.0 && tc.vg_e_m_s > 0.0;
}

// kappa(T) of the GaN column of Table II on the grid above (midpoint rule in
// the wave vector, 4000 points), with the boundary term and, when n_e > 0,
// the phonon-electron term of Eq. (1)
std::vector<double> kappa_table_build(const emc_thermal_config& tc)
{
    const double q0 = tc.k0_per_m, wm = tc.omega_max_rad_s;
    std::vector<double> out(kNT);
    const int nq = 4000;
    for (int t = 0; t < kNT; ++t) {
        const double T = kTLo + kTStep * t;
        const double E_F = tc.n_e_m3 > 0.0 ? fermi_level(tc.n_e_m3, T, tc.m_e_rel) : 0.0;
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
            if (tc.n_e_m3 > 0.0) rate += tau_e_inv(w, T, E_F, tc);
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
    static std::map<std::vector<double>, std::vector<double>> cache;
    const std::vector<double> key = {tc.k0_per_m, tc.omega_max_rad_s, tc.A_s3, tc.B1_s_per_K, tc.B2_K, tc.L_boundary,
                                     tc.n_e_m3, tc.m_e_rel, tc.Da_eV, tc.rho_kg_m3, tc.vg_e_m_s};
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, kappa_table_build(tc)).first;
    return it->second;
}

// 1/R_K(T) of Eq. (3) per unit interface area on the kappa grid.  With the
// sine branches, v_g D = q^2 / (2 pi^2) per branch, so Eq. (2) is
// tau_12 = q_2(w)^2 / (q_1(w)^2 + q_2(w)^2) (zero above the substrate's
// omega_max) and Eq. (3) is, over the wire's wave vector q_1 (dw = v_g dq),
// (3/4) int hbar w (q_1^2 / 2 pi^2) dn/dT tau_12 v_g dq_1 (midpoint rule, up
// to the wave vector at which the substrate runs out of states).
double dmm_tau12(double w, const emc_thermal_config& tc)
{
    const double w1 = tc.omega_max_rad_s, w2 = tc.sub_omega_max_rad_s;
    if (!(w > 0.0) || !(w < w2)) return 0.0;  // no substrate states
    if (!(w < w1)) return 1.0;                // substrate states only
    const double q1 = 2.0 * tc.k0_per_m / kPi * std::asin(w / w1);
    const double q2 = 2.0 * tc.sub_k0_per_m / kPi * std::asin(w / w2);
    return q2 * q2 / (q1 * q1 + q2 * q2);
}

std::vector<double> interface_table_build(const emc_thermal_config& tc)
{
    const double q0 = tc.k0_per_m, wm = tc.omega_max_rad_s;
    const double qtop = tc.sub_omega_max_rad_s < wm ? 2.0 * q0 / kPi * std::asin(tc.sub_omega_max_rad_s / wm) : q0;
    const int nq = 8000;
    std::vector<double> out(kNT);
    for (int t = 0; t < kNT; ++t) {
        const double T = kTLo + kTStep * t;
        double acc = 0.0;
        for (int i = 0; i < nq; ++i) {
            const double q = (i + 0.5) * qtop / nq;
            const double w = wm * std::sin(kPi * q / (2.0 * q0));
            const double vg = wm * kPi / (2.0 * q0) * std::cos(kPi * q / (2.0 * q0));
            const double x = kHbar * w / (kKB * T);
            const double em1 = std::expm1(x);
            const double dndT = x * std::exp(x) / (em1 * em1) / T;
            acc += kHbar * w * q * q / (2.0 * kPi * kPi) * dndT * dmm_tau12(w, tc) * vg;
        }
        out[t] = 0.75 * acc * qtop / nq;
    }
    return out;
}

bool dmm_ok(const emc_thermal_config& tc)
{
    return tc.k0_per_m > 0.0 && tc.omega_max_rad_s > 0.0 && tc.sub_k0_per_m > 0.0 && tc.sub_omega_max_rad_s > 0.0;
}

std::vector<double> interface_table(const emc_thermal_config& tc)
{
    static std::mutex mu;
    static std::map<std::vector<double>, std::vector<double>> cache;
    const std::vector<double> key = {tc.k0_per_m, tc.omega_max_rad_s, tc.sub_k0_per_m, tc.sub_omega_max_rad_s};
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, interface_table_build(tc)).first;
    return it->second;
}

double table_at(const std::vector<double>& tab, double T)
{
    double f = (T - kTLo) / kTStep;
    f = std::fmin(std::fmax(f, 0.0), double(kNT - 1) - 1e-9);
    const int k = int(f);
    const double a = f - k;
    return tab[k] * (1.0 - a) + tab[k + 1] * a;
}

struct TGeo {
    int nx, ny, nz, n;
    double hx, hy, hz, T_sink, h_bottom, tol;
    int max_picard, max_cg;
    const double* g_if;    // interface conductance table (area ratio applied), or null
};

__device__ __forceinline__ double kap_at(const double* tab, double T)
{
    double f = (T - kTLo) / kTStep;
    f = fmin(fmax(f, 0.0), double(kNT - 1) - 1e-9);
    const int i = int(f);
    const double a = f - i;
    return tab[i] * (1.0 - a) + tab[i + 1] * a;
}

// y = A(kappa) x on the grid; bnd[c] receives the boundary conductance sum.
// gif[c]: the interface conductance of a bottom subcell (0: none)
__device__ void apply(const TGeo& G, const double* kap, const double* gif, const double* x, double* y, double* bnd)
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
        if (l > 0) {
            face(c - 1, G.hz);
        } else {
            double r = G.hz / (2.0 * kc) + (G.h_bottom > 0.0 ? 1.0 / G.h_bottom : 0.0);
            if (gif[c] > 0.0) r += 1.0 / gif[c];
            gb += 1.0 / (G.hz * r);
        }
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
    double* gif = sh + 6 * G.n;
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
            gif[c] = (G.g_if && c % G.nz == 0) ? kap_at(G.g_if, x[c]) : 0.0;
            p[c] = x[c];  // previous Picard iterate
        }
        __syncthreads();
        // r = b - A x with b = q + g_b T_sink
        apply(G, kap, gif, x, Ap, r);
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
            apply(G, kap, gif, d, Ad, nullptr);
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


// ------------------------------------------------------------ phonon MC
// Spectral tables of the phonon Monte Carlo: nb equal wave-vector bins of
// (0, q0), each standing for its centre q_b, w_b = w_max sin(pi q_b / 2 q0),
// v_b = (pi w_max / 2 q0) cos(pi q_b / 2 q0), heat capacity per unit volume
// of three branches C_b = 3 hbar w_b dn/dT q_b^2 dq / (2 pi^2); per distinct
// whole-kelvin temperature the rates 1/tau_b and the cumulative of
// C_b / tau_b (the re-emission distribution).
struct PhTables {
    std::vector<double> vg;       // [nb] nm/ps
    std::vector<double> rate;     // [nt][nb] 1/ps
    std::vector<double> cdf;      // [nt][nb]
    std::vector<double> ctot;     // [nt] J/(m^3 K)
    std::vector<int> tix;         // [C]
    std::vector<double> tau12;    // [nb]
};

const char* ph_tables(const emc_thermal_config& tc, int nb, const std::vector<double>& T_cells, bool interface,
                      PhTables* out)
{
    const double q0 = tc.k0_per_m, wm = tc.omega_max_rad_s, dq = q0 / nb;
    std::vector<double> w(nb), v(nb), modes(nb);
    out->vg.resize(nb);
    out->tau12.assign(nb, 0.0);
    for (int i = 0; i < nb; ++i) {
        const double q = (i + 0.5) * dq;
        w[i] = wm * std::sin(kPi * q / (2.0 * q0));
        v[i] = wm * kPi / (2.0 * q0) * std::cos(kPi * q / (2.0 * q0));
        modes[i] = q * q * dq / (2.0 * kPi * kPi);
        out->vg[i] = v[i] * 1e-3;
        if (interface) out->tau12[i] = dmm_tau12(w[i], tc);
    }
    std::map<long long, int> key_of;
    out->tix.resize(T_cells.size());
    for (double T : T_cells) key_of.emplace((long long)std::floor(T + 0.5), 0);
    int nt = 0;
    for (auto& kv : key_of) kv.second = nt++;
    for (size_t c = 0; c < T_cells.size(); ++c) out->tix[c] = key_of[(long long)std::floor(T_cells[c] + 0.5)];
    out->rate.assign((size_t)nt * nb, 0.0);
    out->cdf.assign((size_t)nt * nb, 0.0);
    out->ctot.assign(nt, 0.0);
    for (const auto& kv : key_of) {
        const double T = double(kv.first);
        const int t = kv.second;
        const double EF = tc.n_e_m3 > 0.0 ? fermi_level(tc.n_e_m3, T, tc.m_e_rel) : 0.0;
        double acc = 0.0, ct = 0.0;
        for (int i = 0; i < nb; ++i) {
            double r = tc.A_s3 * std::pow(w[i], 4) + tc.B1_s_per_K * w[i] * w[i] * T * std::exp(-tc.B2_K / T);
            if (tc.L_boundary > 0.0) r += v[i] / tc.L_boundary;
            if (tc.n_e_m3 > 0.0) r += tau_e_inv(w[i], T, EF, tc);
            const double x = kHbar * w[i] / (kKB * T);
            double dndT = 0.0;
            if (x < 700.0) {
                const double em1 = std::expm1(x);
                dndT = x * std::exp(x) / (em1 * em1) / T;
            }
            const double cb = 3.0 * kHbar * w[i] * dndT * modes[i];
            out->rate[(size_t)t * nb + i] = r * 1e-12;
            acc += cb * r;
            out->cdf[(size_t)t * nb + i] = acc;
            ct += cb;
        }
        if (!(acc > 0.0) || !std::isfinite(acc)) return "phonon MC: no scattering weight at some temperature";
        for (int i = 0; i < nb; ++i) out->cdf[(size_t)t * nb + i] /= acc;
        out->cdf[(size_t)t * nb + nb - 1] = 1.0;
        out->ctot[t] = ct;
    }
    return nullptr;
}

template <typename Real>
std::vector<Real> as_real(const std::vector<double>& a)
{
    return std::vector<Real>(a.begin(), a.end());
}

template <typename Real>
emc_status phonon_run(emc_ctx* ctx, const emc_phonon_config& pc, const PhTables& tb, const std::vector<double>& ccdf,
                      const std::vector<int>& neg,
                      int nx, int ny, int nz, double Lx, double Ly, double Lz, int64_t n, int64_t first,
                      std::vector<unsigned long long>* t_res, std::vector<unsigned long long>* scat,
                      std::vector<unsigned long long>* emit, unsigned long long out8[8], float* ms)
{
    cudaStream_t st = ctx_stream(ctx);
    const int C = nx * ny * nz, nb = pc.n_bins, nt = (int)tb.ctot.size();
#define PCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return ctx_fail(ctx, EMC_ECUDA, cudaGetErrorString(e_)); \
    } while (0)
    const std::vector<Real> vg = as_real<Real>(tb.vg), rate = as_real<Real>(tb.rate), cdf = as_real<Real>(tb.cdf),
                            cc = as_real<Real>(ccdf), t12 = as_real<Real>(tb.tau12);
    Real *d_vg, *d_rate, *d_cdf, *d_cc, *d_t12;
    int *d_tix, *d_neg;
    unsigned long long* d_u;  // next, out[8], t_res[C], scat[C], emit[C]
    PCK(cudaMallocAsync(&d_vg, sizeof(Real) * nb, st));
    PCK(cudaMallocAsync(&d_rate, sizeof(Real) * nt * nb, st));
    PCK(cudaMallocAsync(&d_cdf, sizeof(Real) * nt * nb, st));
    PCK(cudaMallocAsync(&d_cc, sizeof(Real) * C, st));
    PCK(cudaMallocAsync(&d_t12, sizeof(Real) * nb, st));
    PCK(cudaMallocAsync(&d_tix, sizeof(int) * C, st));
    PCK(cudaMallocAsync(&d_neg, sizeof(int) * C, st));
    const size_t nu = 10 + 3 * (size_t)C;  // next, out[8], error word, tallies
    PCK(cudaMallocAsync(&d_u, sizeof(unsigned long long) * nu, st));
    PCK(cudaMemcpyAsync(d_vg, vg.data(), sizeof(Real) * nb, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_rate, rate.data(), sizeof(Real) * nt * nb, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_cdf, cdf.data(), sizeof(Real) * nt * nb, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_cc, cc.data(), sizeof(Real) * C, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_t12, t12.data(), sizeof(Real) * nb, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_tix, tb.tix.data(), sizeof(int) * C, cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_neg, neg.data(), sizeof(int) * C, cudaMemcpyHostToDevice, st));
    PCK(cudaMemsetAsync(d_u, 0, sizeof(unsigned long long) * nu, st));
    PhParams P{};
    P.nx = nx; P.ny = ny; P.nz = nz; P.ncell = C; P.nb = nb;
    P.hx = Lx * 1e9 / nx; P.hy = Ly * 1e9 / ny; P.hz = Lz * 1e9 / nz;
    P.vg = d_vg; P.rate = d_rate; P.cdf = d_cdf; P.tix = d_tix; P.cell_cdf = d_cc; P.tau12 = d_t12;
    P.cell_neg = d_neg;
    for (int f = 0; f < 6; ++f) {
        P.face[f] = pc.face[f];
        P.p_spec[f] = pc.p_specular[f];
    }
    P.seed = pc.seed;
    P.n_bundles = n; P.first = first; P.max_segments = pc.max_segments;
    P.next = d_u; P.out = d_u + 1; P.err = reinterpret_cast<int*>(d_u + 9);
    P.t_res = d_u + 10; P.scat = d_u + 10 + C; P.emit = d_u + 10 + 2 * (size_t)C;
    P.nt = nt;
    const int block = pc.block_size ? pc.block_size : 256;
    const size_t smem = ph_smem_bytes<Real>(C);
    PCK(cudaFuncSetAttribute(k_phonon<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PCK(cudaFuncSetAttribute(k_phonon<Real>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared));
    int dev = 0, nsm = 0, occ = 0;
    PCK(cudaGetDevice(&dev));
    PCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_phonon<Real>, block, smem));
    long long grid = (long long)nsm * (occ > 0 ? occ : 1);
    const long long need = (n + block - 1) / block;
    if (grid > need) grid = need;
    cudaEvent_t e0, e1;
    PCK(cudaEventCreate(&e0));
    PCK(cudaEventCreate(&e1));
    PCK(cudaEventRecord(e0, st));
    k_phonon<Real><<<(unsigned)grid, block, smem, st>>>(P);
    ctx_count_launches(ctx, 1);
    PCK(cudaGetLastError());
    PCK(cudaEventRecord(e1, st));
    std::vector<unsigned long long> u(nu);
    PCK(cudaMemcpyAsync(u.data(), d_u, sizeof(unsigned long long) * nu, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    PCK(cudaEventElapsedTime(ms, e0, e1));
    PCK(cudaEventDestroy(e0));
    PCK(cudaEventDestroy(e1));
    for (void* ptr : {(void*)d_vg, (void*)d_rate, (void*)d_cdf, (void*)d_cc, (void*)d_t12, (void*)d_tix, (void*)d_neg,
                      (void*)d_u})
        PCK(cudaFreeAsync(ptr, st));
    PCK(cudaStreamSynchronize(st));
#undef PCK
    for (int k = 0; k < 8; ++k) out8[k] = u[1 + k];
    t_res->assign(u.begin() + 10, u.begin() + 10 + C);
    scat->assign(u.begin() + 10 + C, u.begin() + 10 + 2 * C);
    emit->assign(u.begin() + 10 + 2 * C, u.begin() + 10 + 3 * C);
    if (u[9] != 0ull) return ctx_fail(ctx, EMC_EOVERFLOW, "phonon Monte Carlo: index out of range (checked build)");
    return EMC_OK;
}

}  // namespace

extern "C" {

emc_status emc_kappa(const emc_thermal_config* tc, const double* T, double* kappa, int32_t n)
{
    if (!tc || n < 0 || (n > 0 && (!T || !kappa)) || !electrons_ok(*tc)) return EMC_EINVAL;
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

emc_status emc_dmm_transmissivity(const emc_thermal_config* tc, const double* omega, double* tau12, int32_t n)
{
    if (!tc || n < 0 || (n > 0 && (!omega || !tau12)) || !dmm_ok(*tc)) return EMC_EINVAL;
    for (int i = 0; i < n; ++i) tau12[i] = dmm_tau12(omega[i], *tc);
    return EMC_OK;
}

emc_status emc_interface_conductance(const emc_thermal_config* tc, const double* T, double* G_K, int32_t n)
{
    if (!tc || n < 0 || (n > 0 && (!T || !G_K)) || !dmm_ok(*tc)) return EMC_EINVAL;
    const std::vector<double> tab = interface_table(*tc);
    for (int i = 0; i < n; ++i) G_K[i] = table_at(tab, T[i]);
    return EMC_OK;
}

emc_status emc_thermal_solve(emc_ctx* ctx, const emc_thermal_config* tc, const double* q, double* T, int32_t* iters)
{
    EMC_TRACE("emc_thermal_solve");
    if (!ctx || !tc || !q || !T) return EMC_EINVAL;
    int nx, ny, nz, ne;
    double Lx, Ly, Lz;
    if (!ctx_grid(ctx, &nx, &ny, &nz, &Lx, &Ly, &Lz, &ne))
        return ctx_fail(ctx, EMC_ESTATE, "emc_thermal_solve needs the nanowire geometry");
    const int n = nx * ny * nz;
    if (n > kMaxThermalCells) return ctx_fail(ctx, EMC_EINVAL, "emc_thermal_solve: at most 2048 subcells");
    const bool dmm = tc->interface_dmm != 0;
    if (!(tc->T_sink > 0) || !(dmm || tc->h_bottom > 0) || tc->max_picard <= 0 || tc->max_cg <= 0 ||
        !electrons_ok(*tc) || (dmm && (!dmm_ok(*tc) || !(tc->interface_area_ratio > 0))))
        return ctx_fail(ctx, EMC_EINVAL, "emc_thermal_solve: invalid configuration");
    cudaStream_t st = ctx_stream(ctx);
    const std::vector<double> tab = kappa_table(*tc);
    double *d_tab = nullptr, *d_q = nullptr, *d_T = nullptr, *d_gif = nullptr;
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
    std::vector<double> gtab;
    if (dmm) {
        gtab = interface_table(*tc);
        for (double& g : gtab) g *= tc->interface_area_ratio;
        TCK(cudaMallocAsync(&d_gif, sizeof(double) * kNT, st));
        TCK(cudaMemcpyAsync(d_gif, gtab.data(), sizeof(double) * kNT, cudaMemcpyHostToDevice, st));
    }
    TCK(cudaMemcpyAsync(d_q, q, bytes, cudaMemcpyHostToDevice, st));
    TCK(cudaMemcpyAsync(d_T, T, bytes, cudaMemcpyHostToDevice, st));
    TGeo G{nx, ny, nz, n, Lx / nx, Ly / ny, Lz / nz, tc->T_sink, tc->h_bottom, tc->tol_K, tc->max_picard, tc->max_cg,
           d_gif};
    const size_t smem = sizeof(double) * 7 * n;
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
    if (d_gif) TCK(cudaFreeAsync(d_gif, st));
    TCK(cudaStreamSynchronize(st));
#undef TCK
    return EMC_OK;
}

emc_status emc_phonon_solve(emc_ctx* ctx, const emc_thermal_config* tc, const emc_phonon_config* pc,
                            const double* q, const double* T_cells, int64_t n_bundles, int64_t first,
                            double* dT, double* t_res_ps, uint64_t* scatterings, uint64_t* emitted,
                            emc_phonon_tally* tally)
{
    EMC_TRACE("emc_phonon_solve");
    if (!ctx || !tc || !pc || !q) return EMC_EINVAL;
    int nx, ny, nz, ne;
    double Lx, Ly, Lz;
    if (!ctx_grid(ctx, &nx, &ny, &nz, &Lx, &Ly, &Lz, &ne))
        return ctx_fail(ctx, EMC_ESTATE, "emc_phonon_solve needs the nanowire geometry");
    const int C = nx * ny * nz;
    if (C > 4096) return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: at most 4096 subcells");
    bool absorbing = false, interface = false;
    for (int f = 0; f < 6; ++f) {
        if (pc->face[f] < EMC_PH_SPECULAR || pc->face[f] > EMC_PH_INTERFACE || !(pc->p_specular[f] >= 0.0) ||
            !(pc->p_specular[f] <= 1.0))
            return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: face kinds and p_specular in [0, 1]");
        absorbing |= pc->face[f] == EMC_PH_ISOTHERMAL || pc->face[f] == EMC_PH_INTERFACE;
        interface |= pc->face[f] == EMC_PH_INTERFACE;
    }
    if (!absorbing) return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: no isothermal or interface face");
    if (pc->n_bins < 1 || pc->n_bins > 65536 || pc->max_segments < 1 || pc->max_segments > 1000000000 ||
        (pc->precision != EMC_FP32 && pc->precision != EMC_FP64) ||
        (pc->block_size != 0 && (pc->block_size < 32 || pc->block_size > 256 || pc->block_size % 32)))
        return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: n_bins, max_segments, precision or block_size");
    if (n_bundles < 1 || first < 0 || first + n_bundles > (int64_t(1) << 32))
        return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: bundle ids first .. first + n - 1 must lie in [0, 2^32)");
    if (!(tc->k0_per_m > 0) || !(tc->omega_max_rad_s > 0) || tc->A_s3 < 0 || tc->B1_s_per_K < 0 || tc->B2_K < 0 ||
        tc->L_boundary < 0 || !electrons_ok(*tc) || (interface && !dmm_ok(*tc)))
        return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: invalid phonon model");
    double qsum = 0.0;  // sum |q|
    std::vector<int> neg(C);
    for (int c = 0; c < C; ++c) {
        if (!std::isfinite(q[c])) return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: q must be finite");
        qsum += std::fabs(q[c]);
        neg[c] = q[c] < 0.0 ? 1 : 0;
    }
    if (!(qsum > 0.0)) return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: no heat");
    std::vector<double> Tc(C, tc->T_sink);
    if (T_cells)
        for (int c = 0; c < C; ++c) Tc[c] = T_cells[c];
    for (int c = 0; c < C; ++c)
        if (!(Tc[c] >= 1.0 && Tc[c] <= 1e5)) return ctx_fail(ctx, EMC_EINVAL, "emc_phonon_solve: temperatures in [1, 1e5] K");
    PhTables tb;
    if (const char* e = ph_tables(*tc, pc->n_bins, Tc, interface, &tb)) return ctx_fail(ctx, EMC_EINVAL, e);
    std::vector<double> ccdf(C);
    double acc = 0.0;
    for (int c = 0; c < C; ++c) {
        acc += std::fabs(q[c]);
        ccdf[c] = acc / qsum;
    }
    ccdf[C - 1] = 1.0;
    std::vector<unsigned long long> tr, sc, em;
    unsigned long long out8[8];
    float ms = 0.f;
    const emc_status s =
        pc->precision == EMC_FP64
            ? phonon_run<double>(ctx, *pc, tb, ccdf, neg, nx, ny, nz, Lx, Ly, Lz, n_bundles, first, &tr, &sc, &em, out8, &ms)
            : phonon_run<float>(ctx, *pc, tb, ccdf, neg, nx, ny, nz, Lx, Ly, Lz, n_bundles, first, &tr, &sc, &em, out8, &ms);
    if (s != EMC_OK) return s;
    const double Vc = Lx * Ly * Lz / C, power = qsum * Vc;
    uint64_t nscat = 0;
    for (int c = 0; c < C; ++c) {
        const double t_ps = double((long long)tr[c]) / kPhTimeScale;  // two's complement: signed
        if (t_res_ps) t_res_ps[c] = t_ps;
        if (dT) dT[c] = power * (t_ps * 1e-12) / double(n_bundles) / (tb.ctot[tb.tix[c]] * Vc);
        if (scatterings) scatterings[c] = sc[c];
        if (emitted) emitted[c] = em[c];
        nscat += sc[c];
    }
    if (tally) {
        for (int f = 0; f < 6; ++f) tally->absorbed[f] = out8[f];
        tally->segments = out8[6];
        tally->capped = out8[7];
        tally->scatterings = nscat;
        tally->power_W = power;
        tally->kernel_ms = ms;
    }
    return EMC_OK;
}

}  // extern "C"
