// libemc host side: the C ABI of include/emc.h, device memory, rate tables,
// Poisson update and the step loop.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/emc.h"
#include "common.cuh"
#include "trace.h"

namespace emc {
template <typename Real> void launch_flight(const DevParams&, bool, int, int, int, int, cudaStream_t);
template <typename Real> void launch_init(const DevParams&, bool, cudaStream_t);
template <typename Real> void launch_inject(const DevParams&, cudaStream_t);
template <typename Real> void launch_free_counts(const DevParams&, long long*, cudaStream_t);
template <typename Real>
cudaError_t pair_prepare(const DevParams&, bool, const DevParams&, bool, int, size_t*, int*);
template <typename Real>
void launch_flight_pair(const DevParams&, bool, int, int, const DevParams&, bool, int, int, int, int, size_t,
                        cudaStream_t);
template <typename Real> cudaError_t flight_set_smem(size_t);
template <typename Real> size_t flight_smem_bytes(int, int);
template <typename Real> int flight_blocks_per_sm(bool, int, size_t);
template <typename Real> void launch_rescale(const DevParams&, int, int64_t, const double*, cudaStream_t);
template <typename Real>
void launch_sort(const DevParams&, const DevParams&, bool, uint32_t*, unsigned int*, const unsigned int*, unsigned int*,
                 int, cudaStream_t);
}  // namespace emc

using namespace emc;

namespace {

// FP64 iterative-refinement sweeps per Poisson update: the FP32 inverse
// contracts the error by ~kappa * 2^-24 ~ 4e-4 per sweep, and the update is
// warm-started from the previous potential, so three sweeps reach the FP64
// residual floor; a cold start (standalone solve) takes five.
constexpr int kPoissonSweeps = 3;
// FP32 production steps: the potential is warm-started from the previous
// Poisson period, and one FP64-refined sweep with the FP32 inverse leaves a
// relative error of ~1e-7 (the precision of the FP32 field) even after a
// 10% change; the parity build, the first solve and bias changes keep three
constexpr int kPoissonSweepsStepF32 = 1;
constexpr int kSmemTableKiB = 32;  // default rate-table bytes staged per block
constexpr int kMaxCells = 8192;                 // dense FP64 Poisson inverse limit

// Golden-rule prefactors of one table set in device units (nm, fs, eV).
struct RateConst {
    double ck[NV], alpha[NV], Ec[NV];
    double hw_lo, hw_iv, N_lo, N_iv;
    double pop_K;   // (e^2/eps0) hw_lo (1/eps_inf - 1/eps_s) / 2        eV^2 nm
    double ac_K;    // Da^2 kT / (rho vs^2)                               eV^2 nm^3
    double iv_K;    // hbar^2 Dij^2 / (2 rho hw_iv)                       eV^2 nm^3
    double imp_K;   // N_I (e^2 / (eps_s eps0))^2                         eV^2 / nm
    double beta2;   // Debye screening wave vector^2                     1/nm^2
    int Z[NV];
    uint32_t mask;
};

template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct emc_ctx {
    cudaStream_t st = nullptr;
    std::vector<emc_config> cfg;
    int n_ens = 0, prec = EMC_FP32, geom = EMC_GEOM_BULK;
    int nx = 1, ny = 1, nz = 1, ncell = 1, nb = 0, n_tab = 0, block = 256, spl = 50, K = 10, grid_cap = 1;
    int sort_period = 0;
    int64_t n_slots = 0, steps_done = 0, launches = 0, bits_words = 0;
    // particle sharding: 0 no exchange pending, 1 the initial solve, 2 the
    // refill and Poisson update at the end of a period
    bool sharded = false;
    int shard_pending = 0;
    double dt_fs = 1.0, dE = 0.002;
    double Lx = 1, Ly = 1, Lz = 1, dx = 1, dy = 1, dz = 1;  // nm
    std::vector<int64_t> off, cap, n0;
    std::vector<int32_t> tabset;
    std::vector<RateConst> rc;     // per table set
    std::vector<double> w;         // superparticle weight per ensemble
    std::vector<double> bias;      // [E][3] Vs Vd Vg
    std::vector<double> g0_host;   // [TS][NV] Gamma0, 1/fs
    std::vector<uint8_t> gate_ix;  // [nx]
    std::string err;
    DevParams P{};
    // device buffers
    void *kx = nullptr, *ky = nullptr, *kz = nullptr, *x = nullptr, *y = nullptr, *z = nullptr, *tr = nullptr;
    uint32_t *tag = nullptr, *id = nullptr, *slot_of_id = nullptr, *dead_bits = nullptr;
    uint64_t* ctr = nullptr;
    int64_t *d_off = nullptr, *d_cap = nullptr, *d_n0 = nullptr, *d_bits_off = nullptr;
    uint32_t* d_seed = nullptr;
    int32_t *d_tabset = nullptr, *d_target = nullptr;
    uint32_t* d_gid = nullptr;
    long long *d_shard = nullptr, *d_free = nullptr;
    void *acc_bulk = nullptr, *acc_cell = nullptr, *table = nullptr, *phys = nullptr;
    double* tab64 = nullptr;
    unsigned long long *events = nullptr, *cnt = nullptr;
    double* sums = nullptr;
    int* charge = nullptr;
    long long* alive = nullptr;
    int* d_err = nullptr;
    // Poisson
    double *Lmat = nullptr, *Ginv = nullptr, *phi = nullptr, *rhs = nullptr, *Efield = nullptr, *d_bias = nullptr,
           *d_w = nullptr, *d_Nd = nullptr;
    // emc_tally_async: packed-tally staging buffer and per-ensemble
    // parameters {hw_lo, hw_iv, w, Fx, Fy, Fz}, allocated on first use
    unsigned char* tstage = nullptr;
    double* tpar = nullptr;
    float *G32 = nullptr, *r32 = nullptr, *part = nullptr;
    uint8_t* d_gate = nullptr;
    std::vector<void*> allocs;
    // particle sort (allocated on first use)
    void *akx = nullptr, *aky = nullptr, *akz = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr, *atr = nullptr;
    uint32_t *atag = nullptr, *aid = nullptr, *skey = nullptr;
    uint64_t* actr = nullptr;
    unsigned int *shist = nullptr, *soffs = nullptr, *sblk = nullptr;
    int64_t n_keys = 0;
    int64_t flights_since_sort = 0;
    int64_t sorts = 0;
    // per-subcell temperature (built on the first emc_set_temperature)
    int32_t* cell_bin = nullptr;
    void *bin_table = nullptr, *bin_phys = nullptr, *ens_g0 = nullptr, *ens_ig0 = nullptr;
    double* bin_tab64 = nullptr;
    std::vector<double> bin_g0;         // [NTBIN][NV] Gamma0 of each bin, 1/fs
    std::vector<double> ens_g0_host;    // [E][NV] current Gamma0 of each ensemble
    std::vector<int32_t> cell_bin_host; // [E][C]
    // graph of the per-chunk tail (refill + Poisson update + field)
    cudaGraph_t g_tail = nullptr;
    cudaGraphExec_t g_tail_exec = nullptr;
    int64_t g_tail_launches = 0;
    bool use_graph = true;
    // the context's surrogate network (emc_surrogate_train)
    emc_mlp* sur = nullptr;
    // flight-kernel timing
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

namespace {

emc_status fail(emc_ctx* c, emc_status s, const std::string& m)
{
    if (c) c->err = m;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, EMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

template <typename T>
cudaError_t dalloc(emc_ctx* ctx, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
        ctx->allocs.push_back(q);
        cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(T), ctx->st);
        *p = static_cast<T*>(q);
    }
    return e;
}

// --------------------------------------------------------------- rates
__device__ double dos(const RateConst& R, int v, double E)
{
    const double g = E * (1.0 + R.alpha[v] * E);
    return pow(1.0 / R.ck[v], 1.5) * sqrt(g) * (1.0 + 2.0 * R.alpha[v] * E) / (4.0 * kPi * kPi);
}

// total out-scattering rate (1/fs) of mechanism m in valley v at energy E (eV)
__device__ double rate(const RateConst& R, int v, int m, double E)
{
    if (!((R.mask >> m) & 1u) || E < 0.0) return 0.0;
    const double two_pi_hbar = 2.0 * kPi / kHbarEVfs;
    if (m == 0) {
        if (E <= 0.0) return 0.0;
        const double k = sqrt(E * (1.0 + R.alpha[v] * E) / R.ck[v]);
        const double k2dkdE = k * (1.0 + 2.0 * R.alpha[v] * E) / (2.0 * R.ck[v]);
        return R.imp_K * k2dkdE / (kPi * kHbarEVfs * R.beta2 * (4.0 * k * k + R.beta2));
    }
    if (m == 1 || m == 2) {
        const double Ep = (m == 1) ? E + R.hw_lo : E - R.hw_lo;
        if (Ep <= 0.0) return 0.0;
        const double occ = (m == 1) ? R.N_lo : R.N_lo + 1.0;
        const double k = sqrt(E * (1.0 + R.alpha[v] * E) / R.ck[v]);
        const double kp = sqrt(Ep * (1.0 + R.alpha[v] * Ep) / R.ck[v]);
        const double Lk = (k > 0.0) ? log(fabs((k + kp) / (k - kp))) / k : 2.0 / kp;
        return R.pop_K * occ * (1.0 + 2.0 * R.alpha[v] * Ep) * Lk / (4.0 * kPi * kHbarEVfs * R.ck[v]);
    }
    if (m == 3) return two_pi_hbar * R.ac_K * dos(R, v, E);
    const int j = (m - 4) >> 1;
    const bool absorb = (m & 1) == 0;
    const int Zf = R.Z[j] - (j == v ? 1 : 0);
    if (Zf <= 0) return 0.0;
    const double Ep = E + (absorb ? R.hw_iv : -R.hw_iv) - (R.Ec[j] - R.Ec[v]);
    if (Ep <= 0.0) return 0.0;
    const double occ = absorb ? R.N_iv : R.N_iv + 1.0;
    return two_pi_hbar * R.iv_K * Zf * occ * dos(R, j, Ep);
}

// cumulative rates at the lower edge of every bin: tab64[ts][v][b][m]
__global__ void k_rates(const RateConst* rc, int n_tab, int nb, double dE, double* tab64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_tab * NV * nb) return;
    const int ts = int(i / (NV * nb));
    const int v = int((i / nb) % NV);
    const int b = int(i % nb);
    const RateConst R = rc[ts];
    const double E = b * dE;
    double acc = 0.0;
    double* row = tab64 + (size_t)i * NM;
    for (int m = 0; m < NM; ++m) {
        acc += rate(R, v, m, E);
        row[m] = acc;
    }
}

// Gamma0 = max over bins of the total; one block per (ts, v)
__global__ void k_gamma0(const double* tab64, int nb, double* g0)
{
    __shared__ double red[256];
    const double* base = tab64 + (size_t)blockIdx.x * nb * NM;
    double mx = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) mx = fmax(mx, base[(size_t)b * NM + NM - 1]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) g0[blockIdx.x] = red[0];
}

template <typename Real>
__global__ void k_normalise(double* tab64, const double* g0, int nb, int64_t n, Real* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t tv = i / ((int64_t)nb * NM);
    const double g = g0[tv];
    const double x = g > 0.0 ? tab64[i] / g : 0.0;
    tab64[i] = x;
    out[i] = Real(x);
}

// -------------------------------------------------------------- Poisson
// L = -(7-point Laplacian) on cell centres (nm^-2), Dirichlet faces half a
// cell away: source/drain x faces always, gate faces (outer side y = Ly and
// top z = Lz) where the cell's x centre is gated.  Neumann elsewhere.
__global__ void k_build_L(double* L, int nx, int ny, int nz, double ax, double ay, double az, const uint8_t* gate)
{
    const int n = nx * ny * nz;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = c / (ny * nz), j = (c / nz) % ny, l = c % nz;
    double* row = L + (size_t)c * n;
    double d = 0.0;
    auto nb = [&](int cc, double a) {
        row[cc] -= a;
        d += a;
    };
    if (i > 0) nb(c - ny * nz, ax); else d += 2.0 * ax;
    if (i < nx - 1) nb(c + ny * nz, ax); else d += 2.0 * ax;
    if (j > 0) nb(c - nz, ay);
    if (j < ny - 1) nb(c + nz, ay); else if (gate[i]) d += 2.0 * ay;
    if (l > 0) nb(c - 1, az);
    if (l < nz - 1) nb(c + 1, az); else if (gate[i]) d += 2.0 * az;
    row[c] += d;
}

// one Gauss-Jordan pivot step of the in-place inversion (no pivoting: L is SPD)
__global__ void k_gj(const double* A, double* B, int n, int k)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= n) return;
    const double p = 1.0 / A[(size_t)k * n + k];
    double out;
    if (i == k && j == k) out = p;
    else if (i == k) out = A[(size_t)k * n + j] * p;
    else if (j == k) out = -A[(size_t)i * n + k] * p;
    else out = A[(size_t)i * n + j] - A[(size_t)i * n + k] * (A[(size_t)k * n + j] * p);
    B[(size_t)i * n + j] = out;
}

__global__ void k_to_f32(const double* a, float* b, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = float(a[i]);
}

struct PoisGeo {
    int nx, ny, nz, n;
    double ax, ay, az;
    const uint8_t* gate;
};

// rhs = rho / (eps_s eps0) + Dirichlet face terms (V/nm^2).  rho from the
// subcell count (charge != null) or from a given density rho_in (C/m^3).
__global__ void k_rhs(PoisGeo G, int n_ens, const int* charge, const double* rho_in, const double* w,
                      const double* Nd_nm, double Vcell, double e2eps, const double* bias, double* rhs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_ens * G.n) return;
    const int e = int(i / G.n), c = int(i % G.n);
    const int ix = c / (G.ny * G.nz), iy = (c / G.nz) % G.ny, iz = c % G.nz;
    double r;
    if (charge) r = e2eps * (Nd_nm[e] - w[e] * charge[i] / Vcell);
    else r = e2eps * rho_in[c] / kQ * 1e-27;
    const double* B = bias + 3 * e;
    if (ix == 0) r += 2.0 * G.ax * B[0];
    if (ix == G.nx - 1) r += 2.0 * G.ax * B[1];
    if (G.gate[ix]) {
        if (iy == G.ny - 1) r += 2.0 * G.ay * B[2];
        if (iz == G.nz - 1) r += 2.0 * G.az * B[2];
    }
    rhs[i] = r;
}

// residual r = rhs - L phi in FP64 (stencil), stored as float for the sweep
__global__ void k_resid(PoisGeo G, int n_ens, const double* rhs, const double* phi, float* r32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_ens * G.n) return;
    const int e = int(i / G.n), c = int(i % G.n);
    const int ix = c / (G.ny * G.nz), iy = (c / G.nz) % G.ny, iz = c % G.nz;
    const double* p = phi + (size_t)e * G.n;
    const double pc = p[c];
    double acc = 0.0;
    const int sx = G.ny * G.nz, sy = G.nz;
    acc += (ix > 0) ? G.ax * (pc - p[c - sx]) : 2.0 * G.ax * pc;
    acc += (ix < G.nx - 1) ? G.ax * (pc - p[c + sx]) : 2.0 * G.ax * pc;
    if (iy > 0) acc += G.ay * (pc - p[c - sy]);
    if (iy < G.ny - 1) acc += G.ay * (pc - p[c + sy]);
    else if (G.gate[ix]) acc += 2.0 * G.ay * pc;
    if (iz > 0) acc += G.az * (pc - p[c - 1]);
    if (iz < G.nz - 1) acc += G.az * (pc - p[c + 1]);
    else if (G.gate[ix]) acc += 2.0 * G.az * pc;
    r32[i] = float(rhs[i] - acc);
}

// phi[e] += Ginv r[e] as a skinny FP32 GEMM: tiles of 64 rows x 32
// ensembles, the columns split into slices of 192 (grid.y) for parallelism.
// A block stages 32 columns of its 64 rows of G (transposed, so a warp reads
// its 8 rows as two broadcast float4) and of the 32 residual vectors in
// shared memory; warp w owns rows 8w..8w+7, lane = ensemble.  Partial sums go
// to part[slice][e][row] and k_sweep_reduce adds them in a fixed order
// (deterministic).
constexpr int kSweepRows = 64, kSweepSlice = 192;

__global__ void __launch_bounds__(256) k_sweep(const float* __restrict__ G32, const float* __restrict__ r32,
                                               float* part, int n, int n_ens, int ldp)
{
    __shared__ __align__(16) float Gt[32][kSweepRows];  // [column][row]
    __shared__ float Rs[32][33];                        // [column][ensemble]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * kSweepRows;
    const int k_beg = blockIdx.y * kSweepSlice;
    const int k_end = min(n, k_beg + kSweepSlice);
    const int e0 = blockIdx.z * 32;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k0 = k_beg; k0 < k_end; k0 += 32) {
        for (int i = threadIdx.x; i < kSweepRows * 32; i += blockDim.x) {
            const int rr = i >> 5, kk = i & 31;  // coalesced along a row of G
            const int gr = r0 + rr, gk = k0 + kk;
            Gt[kk][rr] = (gr < n && gk < k_end) ? G32[(size_t)gr * n + gk] : 0.f;
        }
        for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
            const int ee = i >> 5, kk = i & 31;
            const int gk = k0 + kk;
            Rs[kk][ee] = (e0 + ee < n_ens && gk < k_end) ? r32[(size_t)(e0 + ee) * n + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float rv = Rs[kk][lane];
            const float4 ga = *reinterpret_cast<const float4*>(&Gt[kk][8 * warp]);
            const float4 gb = *reinterpret_cast<const float4*>(&Gt[kk][8 * warp + 4]);
            acc[0] += ga.x * rv;
            acc[1] += ga.y * rv;
            acc[2] += ga.z * rv;
            acc[3] += ga.w * rv;
            acc[4] += gb.x * rv;
            acc[5] += gb.y * rv;
            acc[6] += gb.z * rv;
            acc[7] += gb.w * rv;
        }
        __syncthreads();
    }
    const int e = e0 + lane;
    if (e < n_ens)
        for (int i = 0; i < 8; ++i) {
            const int row = r0 + 8 * warp + i;
            if (row < n) part[((size_t)blockIdx.y * ldp + e) * n + row] = acc[i];
        }
}

__global__ void k_sweep_reduce(const float* part, double* phi, int n, int n_ens, int ldp, int slices)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_ens * n) return;
    double s = 0.0;
    for (int sl = 0; sl < slices; ++sl) s += double(part[(size_t)sl * ldp * n + i]);
    phi[i] += s;
}

int sweep_slices(int n) { return (n + kSweepSlice - 1) / kSweepSlice; }

// part must hold sweep_slices(n) * n_ens * n floats
void launch_sweep(const float* G32, const float* r32, float* part, double* phi, int n, int n_ens, cudaStream_t st)
{
    const dim3 grid((n + kSweepRows - 1) / kSweepRows, sweep_slices(n), (n_ens + 31) / 32);
    k_sweep<<<grid, 256, 0, st>>>(G32, r32, part, n, n_ens, n_ens);
    k_sweep_reduce<<<(unsigned)(((int64_t)n_ens * n + 255) / 256), 256, 0, st>>>(part, phi, n, n_ens, n_ens,
                                                                                 sweep_slices(n));
}

// E = -grad phi (V/nm): central differences, one-sided in boundary cells.
template <typename Real>
__global__ void k_field(PoisGeo G, int n_ens, const double* phi, double hx, double hy, double hz, double* Efield,
                        Real* acc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_ens * G.n) return;
    const int e = int(i / G.n), c = int(i % G.n);
    const int idx[3] = {c / (G.ny * G.nz), (c / G.nz) % G.ny, c % G.nz};
    const int nn[3] = {G.nx, G.ny, G.nz};
    const int st[3] = {G.ny * G.nz, G.nz, 1};
    const double h[3] = {hx, hy, hz};
    const double* p = phi + (size_t)e * G.n;
    double m2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double g;
        if (nn[a] == 1) g = 0.0;
        else if (idx[a] == 0) g = (p[c + st[a]] - p[c]) / h[a];
        else if (idx[a] == nn[a] - 1) g = (p[c] - p[c - st[a]]) / h[a];
        else g = (p[c + st[a]] - p[c - st[a]]) / (2.0 * h[a]);
        const double E = -g;                        // V/nm
        m2 += E * E;
        Efield[i * 3 + a] = E * 1e9;                // V/m
        acc[i * 4 + a] = Real(-E / kHbarEVfs);      // dk/dt of an electron, 1/(nm fs)
    }
    // 1 / (hbar |dk/dt|) = 1 / |E| in nm/V (0 for no field)
    acc[i * 4 + 3] = m2 > 0.0 ? Real(1.0 / sqrt(m2)) : Real(0);
}

__global__ void k_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    U4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    U4 r = philox10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.a;
    out[4 * i + 1] = r.b;
    out[4 * i + 2] = r.c;
    out[4 * i + 3] = r.d;
}

// ------------------------------------------------------------ helpers
unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

bool same_table(const emc_config& a, const emc_config& b)
{
    for (int i = 0; i < 3; ++i)
        if (a.m_rel[i] != b.m_rel[i] || a.Ec_eV[i] != b.Ec_eV[i] || a.alpha_per_eV[i] != b.alpha_per_eV[i] ||
            a.Z[i] != b.Z[i])
            return false;
    return a.eps_s == b.eps_s && a.eps_inf == b.eps_inf && a.rho_kg_m3 == b.rho_kg_m3 && a.Da_eV == b.Da_eV &&
           a.Dij_eV_per_m == b.Dij_eV_per_m && a.hw_lo_eV == b.hw_lo_eV && a.hw_iv_eV == b.hw_iv_eV &&
           a.vs_m_s == b.vs_m_s && a.T_K == b.T_K && a.Nd_m3 == b.Nd_m3 && a.mech_mask == b.mech_mask &&
           a.emax_init_kT == b.emax_init_kT;
}

RateConst make_rc(const emc_config& c)
{
    RateConst R{};
    const double kT = kKB * c.T_K / kQ;  // eV
    for (int v = 0; v < NV; ++v) {
        R.ck[v] = kCk0 / c.m_rel[v];
        R.alpha[v] = c.alpha_per_eV[v];
        R.Ec[v] = c.Ec_eV[v];
        R.Z[v] = c.Z[v];
    }
    R.hw_lo = c.hw_lo_eV;
    R.hw_iv = c.hw_iv_eV;
    R.N_lo = 1.0 / std::expm1(c.hw_lo_eV / kT);
    R.N_iv = 1.0 / std::expm1(c.hw_iv_eV / kT);
    const double rho_vs2 = c.rho_kg_m3 * c.vs_m_s * c.vs_m_s / kQ * 1e-27;  // eV/nm^3
    const double rho_s = c.rho_kg_m3 * 1e-15 / kQ;                           // eV fs^2/nm^5
    const double D = c.Dij_eV_per_m * 1e-9;                                  // eV/nm
    const double Nd_nm = c.Nd_m3 * 1e-27;
    const double e2es = kE2Eps0 / c.eps_s;                                   // eV nm
    R.pop_K = kE2Eps0 * c.hw_lo_eV * (1.0 / c.eps_inf - 1.0 / c.eps_s) / 2.0;
    R.ac_K = c.Da_eV * c.Da_eV * kT / rho_vs2;
    R.iv_K = kHbarEVfs * kHbarEVfs * D * D / (2.0 * rho_s * c.hw_iv_eV);
    R.imp_K = Nd_nm * e2es * e2es;
    R.beta2 = e2es * Nd_nm / kT;
    R.mask = c.mech_mask;
    return R;
}

template <typename Real>
Phys<Real> make_phys(const emc_config& c, const RateConst& R, const double* g0)
{
    Phys<Real> p{};
    const double kT = kKB * c.T_K / kQ;
    for (int v = 0; v < NV; ++v) {
        p.ck[v] = Real(R.ck[v]);
        p.vk[v] = Real(kVk0 / c.m_rel[v]);
        p.alpha[v] = Real(c.alpha_per_eV[v]);
        p.Ec[v] = Real(c.Ec_eV[v]);
        p.inv_g0[v] = Real(g0[v] > 0.0 ? 1.0 / g0[v] : 0.0);
    }
    p.hw_lo = Real(c.hw_lo_eV);
    p.hw_iv = Real(c.hw_iv_eV);
    p.beta2 = Real(R.beta2);
    p.kT = Real(kT);
    const double emax = c.emax_init_kT * kT;
    p.emax_init = Real(emax);
    const double a = c.alpha_per_eV[0];
    p.hmax0 = Real(std::sqrt(1.0 + a * emax) * (1.0 + 2.0 * a * emax));
    return p;
}

emc_status validate(const emc_config* c, int n, emc_ctx* ctx)
{
    if (!c || n <= 0) return fail(ctx, EMC_EINVAL, "no configuration");
    if (n > (1 << 24) - 1) return fail(ctx, EMC_EINVAL, "too many ensembles");
    const emc_config& a = c[0];
    for (int e = 0; e < n; ++e) {
        const emc_config& b = c[e];
        if (b.geometry != a.geometry || b.precision != a.precision || b.dt_s != a.dt_s || b.n_bins != a.n_bins ||
            b.dE_eV != a.dE_eV || b.steps_per_poisson != a.steps_per_poisson || b.nx != a.nx || b.ny != a.ny ||
            b.nz != a.nz || b.Lx != a.Lx || b.Ly != a.Ly || b.Lz != a.Lz || b.gate_on != a.gate_on ||
            b.gate_x0 != a.gate_x0 || b.gate_x1 != a.gate_x1 || b.eps_s != a.eps_s)
            return fail(ctx, EMC_EINVAL, "ensembles of one context must share geometry, grid, precision, dt, table");
        if (b.n_particles < 0 || b.capacity < b.n_particles || b.capacity > 0x7FFFFFFF)
            return fail(ctx, EMC_EINVAL, "need 0 <= n_particles <= capacity < 2^31");
        if (!(b.T_K > 0) || !(b.Nd_m3 > 0) || !(b.dt_s > 0) || !(b.dE_eV > 0) || b.n_bins <= 0)
            return fail(ctx, EMC_EINVAL, "T, Nd, dt, dE and n_bins must be positive");
        for (int v = 0; v < 3; ++v)
            if (!(b.m_rel[v] > 0) || b.alpha_per_eV[v] < 0 || b.Z[v] < 0)
                return fail(ctx, EMC_EINVAL, "invalid valley parameters");
        if (!(b.eps_s > b.eps_inf) || !(b.eps_inf > 0) || !(b.rho_kg_m3 > 0) || !(b.vs_m_s > 0) ||
            !(b.hw_lo_eV > 0) || !(b.hw_iv_eV > 0))
            return fail(ctx, EMC_EINVAL, "invalid material parameters");
        if (b.precision != EMC_FP32 && b.precision != EMC_FP64) return fail(ctx, EMC_EINVAL, "precision");
        if (b.geometry == EMC_GEOM_NANOWIRE) {
            if (b.nx < 2 || b.ny < 1 || b.nz < 1 || (int64_t)b.nx * b.ny * b.nz > kMaxCells)
                return fail(ctx, EMC_EINVAL, "nanowire grid: nx >= 2, ny, nz >= 1, cells <= 8192");
            if (!(b.Lx > 0 && b.Ly > 0 && b.Lz > 0) || b.steps_per_poisson <= 0)
                return fail(ctx, EMC_EINVAL, "nanowire lengths and steps_per_poisson must be positive");
            if (b.p_specular < 0 || b.p_specular > 1) return fail(ctx, EMC_EINVAL, "p_specular in [0,1]");
        } else if (b.geometry != EMC_GEOM_BULK) {
            return fail(ctx, EMC_EINVAL, "geometry");
        }
        if (b.block_size != 0 && (b.block_size < 32 || b.block_size > 256 || b.block_size % 32))
            return fail(ctx, EMC_EINVAL, "block_size: multiple of 32 in [32, 256]");
        if (b.table_smem_kb < 0 || b.table_smem_kb > 200) return fail(ctx, EMC_EINVAL, "table_smem_kb in [0, 200]");
        if (b.steps_per_launch > 1000 || b.steps_per_poisson > 1000)
            return fail(ctx, EMC_EINVAL, "steps_per_launch and steps_per_poisson at most 1000");
        const bool sh = b.shard_n_global != 0 || b.shard_live_base != 0 || b.shard_spare_base != 0;
        if (sh != (a.shard_n_global != 0 || a.shard_live_base != 0 || a.shard_spare_base != 0))
            return fail(ctx, EMC_EINVAL, "shards: every ensemble of a context sharded, or none");
        if (sh) {
            const int64_t spare = std::max<int64_t>(b.capacity, b.n_particles) - b.n_particles;
            if (b.geometry != EMC_GEOM_NANOWIRE) return fail(ctx, EMC_EINVAL, "shards: nanowire only");
            if (b.shard_n_global <= 0 || b.shard_live_base < 0 || b.shard_live_base + b.n_particles > b.shard_n_global ||
                b.shard_spare_base < b.shard_n_global || b.shard_spare_base + spare > 0xFFFFFFFFll)
                return fail(ctx, EMC_EINVAL, "shards: need 0 <= live_base, live_base + n_particles <= N, "
                                             "N <= spare_base, spare_base + spare slots <= 2^32");
        }
    }
    return EMC_OK;
}

template <typename Real>
emc_status build_tables_and_phys(emc_ctx* ctx)
{
    const int TS = ctx->n_tab, nb = ctx->nb;
    RateConst* d_rc = nullptr;
    double* d_g0 = nullptr;
    CK(dalloc(ctx, &d_rc, TS));
    CK(dalloc(ctx, &d_g0, (size_t)TS * NV));
    CK(cudaMemcpyAsync(d_rc, ctx->rc.data(), sizeof(RateConst) * TS, cudaMemcpyHostToDevice, ctx->st));
    const int64_t rows = (int64_t)TS * NV * nb;
    CK(dalloc(ctx, &ctx->tab64, (size_t)rows * NM));
    Real* tabR = nullptr;
    CK(dalloc(ctx, &tabR, (size_t)rows * NM));
    ctx->table = tabR;
    k_rates<<<grid_for(rows, 128), 128, 0, ctx->st>>>(d_rc, TS, nb, ctx->dE, ctx->tab64);
    k_gamma0<<<TS * NV, 256, 0, ctx->st>>>(ctx->tab64, nb, d_g0);
    k_normalise<Real><<<grid_for(rows * NM, 256), 256, 0, ctx->st>>>(ctx->tab64, d_g0, nb, rows * NM, tabR);
    ctx->launches += 3;
    CK(cudaGetLastError());
    ctx->g0_host.assign((size_t)TS * NV, 0.0);
    CK(cudaMemcpyAsync(ctx->g0_host.data(), d_g0, sizeof(double) * TS * NV, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<Phys<Real>> ph(TS);
    std::vector<int> rep(TS, -1);
    for (int e = 0; e < ctx->n_ens; ++e)
        if (rep[ctx->tabset[e]] < 0) rep[ctx->tabset[e]] = e;
    for (int t = 0; t < TS; ++t) {
        for (int v = 0; v < NV; ++v)
            if (!(ctx->g0_host[t * NV + v] > 0.0))
                return fail(ctx, EMC_EINVAL, "a valley has zero total scattering rate (check mech_mask)");
        ph[t] = make_phys<Real>(ctx->cfg[rep[t]], ctx->rc[t], &ctx->g0_host[t * NV]);
    }
    Phys<Real>* d_ph = nullptr;
    CK(dalloc(ctx, &d_ph, TS));
    CK(cudaMemcpyAsync(d_ph, ph.data(), sizeof(Phys<Real>) * TS, cudaMemcpyHostToDevice, ctx->st));
    ctx->phys = d_ph;
    return EMC_OK;
}

template <typename Real>
emc_status alloc_particles(emc_ctx* ctx)
{
    const size_t n = (size_t)ctx->n_slots;
    Real *a, *b, *c, *d, *e, *f, *g;
    CK(dalloc(ctx, &a, n));
    CK(dalloc(ctx, &b, n));
    CK(dalloc(ctx, &c, n));
    CK(dalloc(ctx, &g, n));
    ctx->kx = a; ctx->ky = b; ctx->kz = c; ctx->tr = g;
    if (ctx->geom == EMC_GEOM_NANOWIRE) {
        CK(dalloc(ctx, &d, n));
        CK(dalloc(ctx, &e, n));
        CK(dalloc(ctx, &f, n));
        ctx->x = d; ctx->y = e; ctx->z = f;
    }
    Real *ab = nullptr, *ac = nullptr;
    CK(dalloc(ctx, &ab, (size_t)ctx->n_ens * 4));
    CK(dalloc(ctx, &ac, (size_t)ctx->n_ens * ctx->ncell * 4));
    ctx->acc_bulk = ab;
    ctx->acc_cell = ac;
    // per ensemble (dk/dt of an electron, 1/(nm fs); 4th slot unused in bulk)
    std::vector<Real> hb((size_t)ctx->n_ens * 4, Real(0));
    for (int e = 0; e < ctx->n_ens; ++e)
        for (int i = 0; i < 3; ++i) hb[4 * e + i] = Real(-ctx->cfg[e].field_V_m[i] * 1e-9 / kHbarEVfs);
    CK(cudaMemcpyAsync(ab, hb.data(), sizeof(Real) * hb.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

PoisGeo pgeo(const emc_ctx* ctx)
{
    PoisGeo G;
    G.nx = ctx->nx;
    G.ny = ctx->ny;
    G.nz = ctx->nz;
    G.n = ctx->ncell;
    G.ax = 1.0 / (ctx->dx * ctx->dx);
    G.ay = 1.0 / (ctx->dy * ctx->dy);
    G.az = 1.0 / (ctx->dz * ctx->dz);
    G.gate = ctx->d_gate;
    return G;
}

emc_status poisson_setup(emc_ctx* ctx)
{
    const int n = ctx->ncell;
    const size_t nn = (size_t)n * n;
    CK(dalloc(ctx, &ctx->Lmat, nn));
    CK(dalloc(ctx, &ctx->Ginv, nn));
    CK(dalloc(ctx, &ctx->G32, nn));
    CK(dalloc(ctx, &ctx->phi, (size_t)ctx->n_ens * n));
    CK(dalloc(ctx, &ctx->rhs, (size_t)ctx->n_ens * n));
    CK(dalloc(ctx, &ctx->r32, (size_t)ctx->n_ens * n));
    CK(dalloc(ctx, &ctx->part, (size_t)sweep_slices(n) * ctx->n_ens * n));
    CK(dalloc(ctx, &ctx->Efield, (size_t)ctx->n_ens * n * 3));
    CK(dalloc(ctx, &ctx->d_gate, (size_t)ctx->nx));
    CK(dalloc(ctx, &ctx->d_bias, (size_t)ctx->n_ens * 3));
    CK(dalloc(ctx, &ctx->d_w, (size_t)ctx->n_ens));
    CK(dalloc(ctx, &ctx->d_Nd, (size_t)ctx->n_ens));
    CK(cudaMemcpyAsync(ctx->d_gate, ctx->gate_ix.data(), ctx->nx, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_bias, ctx->bias.data(), sizeof(double) * ctx->bias.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_w, ctx->w.data(), sizeof(double) * ctx->n_ens, cudaMemcpyHostToDevice, ctx->st));
    std::vector<double> Nd(ctx->n_ens);
    for (int e = 0; e < ctx->n_ens; ++e) Nd[e] = ctx->cfg[e].Nd_m3 * 1e-27;
    CK(cudaMemcpyAsync(ctx->d_Nd, Nd.data(), sizeof(double) * ctx->n_ens, cudaMemcpyHostToDevice, ctx->st));
    PoisGeo G = pgeo(ctx);
    k_build_L<<<grid_for(n, 128), 128, 0, ctx->st>>>(ctx->Lmat, ctx->nx, ctx->ny, ctx->nz, G.ax, G.ay, G.az, ctx->d_gate);
    CK(cudaMemcpyAsync(ctx->Ginv, ctx->Lmat, sizeof(double) * nn, cudaMemcpyDeviceToDevice, ctx->st));
    dim3 blk(32, 8), grd(grid_for(n, 32), grid_for(n, 8));
    double *A = ctx->Ginv, *B = ctx->rhs;  // B: temporary (rhs too small) -> use a scratch n*n
    double* scratch = nullptr;
    CK(cudaMalloc(&scratch, sizeof(double) * nn));
    B = scratch;
    for (int k = 0; k < n; ++k) {
        k_gj<<<grd, blk, 0, ctx->st>>>(A, B, n, k);
        std::swap(A, B);
    }
    ctx->launches += 1 + n;
    if (A != ctx->Ginv) CK(cudaMemcpyAsync(ctx->Ginv, A, sizeof(double) * nn, cudaMemcpyDeviceToDevice, ctx->st));
    k_to_f32<<<grid_for((int64_t)nn, 256), 256, 0, ctx->st>>>(ctx->Ginv, ctx->G32, (int64_t)nn);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->st));
    cudaFree(scratch);
    return EMC_OK;
}

// rhs from the subcell counts -> kPoissonSweeps refinement sweeps -> field
template <typename Real>
emc_status poisson_update(emc_ctx* ctx, int sweeps = kPoissonSweeps)
{
    const int n = ctx->ncell, E = ctx->n_ens;
    const int64_t tot = (int64_t)E * n;
    PoisGeo G = pgeo(ctx);
    const double Vcell = ctx->dx * ctx->dy * ctx->dz;
    k_rhs<<<grid_for(tot, 256), 256, 0, ctx->st>>>(G, E, ctx->charge, nullptr, ctx->d_w, ctx->d_Nd, Vcell,
                                                   kE2Eps0 / ctx->cfg[0].eps_s, ctx->d_bias, ctx->rhs);
    for (int s = 0; s < sweeps; ++s) {
        k_resid<<<grid_for(tot, 256), 256, 0, ctx->st>>>(G, E, ctx->rhs, ctx->phi, ctx->r32);
        launch_sweep(ctx->G32, ctx->r32, ctx->part, ctx->phi, n, E, ctx->st);
    }
    k_field<Real><<<grid_for(tot, 256), 256, 0, ctx->st>>>(G, E, ctx->phi, ctx->dx, ctx->dy, ctx->dz, ctx->Efield,
                                                           static_cast<Real*>(ctx->acc_cell));
    ctx->launches += 2 + 3 * sweeps;
    CK(cudaGetLastError());
    return EMC_OK;
}

void fill_params(emc_ctx* ctx)
{
    DevParams& P = ctx->P;
    P.kx = ctx->kx; P.ky = ctx->ky; P.kz = ctx->kz;
    P.x = ctx->x; P.y = ctx->y; P.z = ctx->z; P.tr = ctx->tr;
    P.tag = ctx->tag; P.ctr = ctx->ctr; P.id = ctx->id;
    P.n_slots = ctx->n_slots;
    P.n_ens = ctx->n_ens;
    P.ens_off = ctx->d_off; P.ens_cap = ctx->d_cap; P.ens_n0 = ctx->d_n0;
    P.seed = ctx->d_seed; P.tabset = ctx->d_tabset;
    P.acc_bulk = ctx->acc_bulk; P.acc_cell = ctx->acc_cell;
    P.n_target = ctx->d_target;
    P.ens_gid = ctx->d_gid;
    P.shard = ctx->d_shard;
    P.slot_of_id = ctx->slot_of_id; P.dead_bits = ctx->dead_bits; P.bits_off = ctx->d_bits_off;
    P.table = ctx->table; P.phys = ctx->phys;
    P.n_tab = ctx->n_tab; P.nb = ctx->nb;
    P.inv_dE = 1.0 / ctx->dE;
    P.nx = ctx->nx; P.ny = ctx->ny; P.nz = ctx->nz; P.ncell = ctx->ncell;
    P.Lx = ctx->Lx; P.Ly = ctx->Ly; P.Lz = ctx->Lz;
    P.dx = ctx->dx; P.dy = ctx->dy; P.dz = ctx->dz;
    P.p_spec = ctx->cfg[0].p_specular;
    P.dt = ctx->dt_fs;
    P.events = ctx->events; P.cnt = ctx->cnt; P.sums = ctx->sums; P.charge = ctx->charge;
    P.alive = ctx->alive;
    P.cell_bin = ctx->cell_bin;
    P.bin_table = ctx->bin_table;
    P.bin_phys = ctx->bin_phys;
    P.ens_g0 = ctx->ens_g0;
    P.ens_ig0 = ctx->ens_ig0;
    P.err = ctx->d_err;
    const size_t row = (size_t)NV * NM * (ctx->prec == EMC_FP64 ? 8 : 4);
    const int kib = ctx->cfg[0].table_smem_kb > 0 ? ctx->cfg[0].table_smem_kb : kSmemTableKiB;
    int nbs = (ctx->n_tab == 1) ? (int)std::min<size_t>((size_t)ctx->nb, (size_t)kib * 1024 / row) : 0;
    P.nb_smem = nbs;
}

// exclusive scan of n uint32 (n <= 2048 * 2048): per-block scans of 2048
// elements, a one-block scan of the block totals, then the block offsets
__global__ void k_scan_blocks(const unsigned int* in, unsigned int* out, unsigned int* blk, int64_t n)
{
    __shared__ unsigned int sh[2048];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) sh[i] = (base + i < n) ? in[base + i] : 0u;
    __syncthreads();
    // Hillis-Steele inclusive scan over 2048 with 1024 threads (2 per thread)
    for (int off = 1; off < 2048; off <<= 1) {
        unsigned int a = 0, b = 0;
        const int i0 = threadIdx.x, i1 = threadIdx.x + 1024;
        if (i0 >= off) a = sh[i0 - off];
        if (i1 >= off) b = sh[i1 - off];
        __syncthreads();
        sh[i0] += a;
        sh[i1] += b;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (base + i < n) out[base + i] = (i == 0 ? 0u : sh[i - 1]);
    if (threadIdx.x == 0) blk[blockIdx.x] = sh[2047];
}

__global__ void k_scan_add(unsigned int* out, const unsigned int* blk, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] += blk[i / 2048];
}

template <typename Real>
emc_status sort_particles(emc_ctx* ctx)
{
    const bool nw = ctx->geom == EMC_GEOM_NANOWIRE;
    const size_t n = (size_t)ctx->n_slots;
    if (n == 0) return EMC_OK;
    if (!ctx->skey) {
        Real *a, *b, *c, *g;
        CK(dalloc(ctx, &a, n));
        CK(dalloc(ctx, &b, n));
        CK(dalloc(ctx, &c, n));
        CK(dalloc(ctx, &g, n));
        ctx->akx = a; ctx->aky = b; ctx->akz = c; ctx->atr = g;
        if (nw) {
            Real *d, *e, *f;
            CK(dalloc(ctx, &d, n));
            CK(dalloc(ctx, &e, n));
            CK(dalloc(ctx, &f, n));
            ctx->ax = d; ctx->ay = e; ctx->az = f;
        }
        CK(dalloc(ctx, &ctx->atag, n));
        CK(dalloc(ctx, &ctx->aid, n));
        CK(dalloc(ctx, &ctx->actr, n));
        CK(dalloc(ctx, &ctx->skey, n));
        ctx->n_keys = (int64_t)ctx->n_ens * (NV + 1) * ctx->ncell;
        if (ctx->n_keys > 2048LL * 2048LL) return fail(ctx, EMC_EINVAL, "too many sort keys (ensembles x 4 x cells > 4M)");
        CK(dalloc(ctx, &ctx->shist, (size_t)ctx->n_keys * 2));
        CK(dalloc(ctx, &ctx->soffs, (size_t)ctx->n_keys));
        CK(dalloc(ctx, &ctx->sblk, (size_t)((ctx->n_keys + 2047) / 2048)));
    }
    unsigned int* hist = ctx->shist;
    unsigned int* cursor = ctx->shist + ctx->n_keys;
    CK(cudaMemsetAsync(ctx->shist, 0, sizeof(unsigned int) * 2 * (size_t)ctx->n_keys, ctx->st));
    DevParams alt = ctx->P;
    alt.kx = ctx->akx; alt.ky = ctx->aky; alt.kz = ctx->akz;
    alt.x = ctx->ax; alt.y = ctx->ay; alt.z = ctx->az; alt.tr = ctx->atr;
    alt.tag = ctx->atag; alt.id = ctx->aid; alt.ctr = ctx->actr;
    launch_sort<Real>(ctx->P, alt, nw, ctx->skey, hist, nullptr, nullptr, 0, ctx->st);
    const int64_t nb = (ctx->n_keys + 2047) / 2048;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, ctx->st>>>(hist, ctx->soffs, ctx->sblk, ctx->n_keys);
    if (nb > 1) {
        unsigned int* tmp = cursor;  // cursor is zero; borrow it for the block totals' scan
        k_scan_blocks<<<1, 1024, 0, ctx->st>>>(ctx->sblk, tmp, tmp + nb, nb);
        CK(cudaMemcpyAsync(ctx->sblk, tmp, sizeof(unsigned int) * nb, cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemsetAsync(cursor, 0, sizeof(unsigned int) * (size_t)ctx->n_keys, ctx->st));
        k_scan_add<<<grid_for(ctx->n_keys, 256), 256, 0, ctx->st>>>(ctx->soffs, ctx->sblk, ctx->n_keys);
    }
    launch_sort<Real>(ctx->P, alt, nw, ctx->skey, nullptr, ctx->soffs, cursor, 1, ctx->st);
    const size_t es = sizeof(Real);
    CK(cudaMemcpyAsync(ctx->kx, ctx->akx, es * n, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->ky, ctx->aky, es * n, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->kz, ctx->akz, es * n, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->tr, ctx->atr, es * n, cudaMemcpyDeviceToDevice, ctx->st));
    if (nw) {
        CK(cudaMemcpyAsync(ctx->x, ctx->ax, es * n, cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(ctx->y, ctx->ay, es * n, cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(ctx->z, ctx->az, es * n, cudaMemcpyDeviceToDevice, ctx->st));
    }
    CK(cudaMemcpyAsync(ctx->tag, ctx->atag, 4 * n, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->id, ctx->aid, 4 * n, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->ctr, ctx->actr, 8 * n, cudaMemcpyDeviceToDevice, ctx->st));
    ctx->launches += 2 + (nb > 1 ? 3 : 1);
    ctx->sorts += 1;
    CK(cudaGetLastError());
    return EMC_OK;
}

int temp_bin(double T)
{
    const long k = std::lround((T - TBIN_LO) / TBIN_DT);
    return (int)std::min<long>(NTBIN - 1, std::max<long>(0, k));
}

// rate tables of every temperature bin (the context's single table set)
template <typename Real>
emc_status build_bins(emc_ctx* ctx)
{
    const int nb = ctx->nb;
    std::vector<RateConst> rc(NTBIN);
    for (int k = 0; k < NTBIN; ++k) {
        emc_config c = ctx->cfg[0];
        c.T_K = TBIN_LO + TBIN_DT * k;
        rc[k] = make_rc(c);
    }
    RateConst* d_rc = nullptr;
    double* d_g0 = nullptr;
    CK(cudaMallocAsync(&d_rc, sizeof(RateConst) * NTBIN, ctx->st));
    CK(cudaMallocAsync(&d_g0, sizeof(double) * NTBIN * NV, ctx->st));
    CK(cudaMemcpyAsync(d_rc, rc.data(), sizeof(RateConst) * NTBIN, cudaMemcpyHostToDevice, ctx->st));
    const int64_t rows = (int64_t)NTBIN * NV * nb;
    CK(dalloc(ctx, &ctx->bin_tab64, (size_t)rows * NM));
    Real* tabR = nullptr;
    CK(dalloc(ctx, &tabR, (size_t)rows * NM));
    ctx->bin_table = tabR;
    k_rates<<<grid_for(rows, 128), 128, 0, ctx->st>>>(d_rc, NTBIN, nb, ctx->dE, ctx->bin_tab64);
    k_gamma0<<<NTBIN * NV, 256, 0, ctx->st>>>(ctx->bin_tab64, nb, d_g0);
    k_normalise<Real><<<grid_for(rows * NM, 256), 256, 0, ctx->st>>>(ctx->bin_tab64, d_g0, nb, rows * NM, tabR);
    ctx->launches += 3;
    CK(cudaGetLastError());
    ctx->bin_g0.assign((size_t)NTBIN * NV, 0.0);
    CK(cudaMemcpyAsync(ctx->bin_g0.data(), d_g0, sizeof(double) * NTBIN * NV, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaFreeAsync(d_rc, ctx->st));
    CK(cudaFreeAsync(d_g0, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<Phys<Real>> ph(NTBIN);
    for (int k = 0; k < NTBIN; ++k) {
        emc_config c = ctx->cfg[0];
        c.T_K = TBIN_LO + TBIN_DT * k;
        ph[k] = make_phys<Real>(c, rc[k], &ctx->bin_g0[(size_t)k * NV]);
    }
    Phys<Real>* d_ph = nullptr;
    CK(dalloc(ctx, &d_ph, NTBIN));
    CK(cudaMemcpyAsync(d_ph, ph.data(), sizeof(Phys<Real>) * NTBIN, cudaMemcpyHostToDevice, ctx->st));
    ctx->bin_phys = d_ph;
    Real *g0 = nullptr, *ig0 = nullptr;
    CK(dalloc(ctx, &g0, (size_t)ctx->n_ens * NV));
    CK(dalloc(ctx, &ig0, (size_t)ctx->n_ens * NV));
    ctx->ens_g0 = g0;
    ctx->ens_ig0 = ig0;
    CK(dalloc(ctx, &ctx->cell_bin, (size_t)ctx->n_ens * ctx->ncell));
    // start every ensemble from its own uniform temperature and Gamma0
    ctx->cell_bin_host.assign((size_t)ctx->n_ens * ctx->ncell, 0);
    ctx->ens_g0_host.assign((size_t)ctx->n_ens * NV, 0.0);
    for (int e = 0; e < ctx->n_ens; ++e) {
        const int k = temp_bin(ctx->cfg[e].T_K);
        for (int cc = 0; cc < ctx->ncell; ++cc) ctx->cell_bin_host[(size_t)e * ctx->ncell + cc] = k;
        for (int v = 0; v < NV; ++v) ctx->ens_g0_host[(size_t)e * NV + v] = ctx->g0_host[(size_t)ctx->tabset[e] * NV + v];
    }
    // every ensemble's bins and Gamma0 on the device, not only the ensemble
    // whose temperatures are being set: the flight kernel reads them for all
    std::vector<Real> gR((size_t)ctx->n_ens * NV), igR((size_t)ctx->n_ens * NV);
    for (size_t i = 0; i < gR.size(); ++i) {
        gR[i] = Real(ctx->ens_g0_host[i]);
        igR[i] = Real(1.0 / ctx->ens_g0_host[i]);
    }
    CK(cudaMemcpyAsync(ctx->cell_bin, ctx->cell_bin_host.data(), sizeof(int32_t) * ctx->cell_bin_host.size(),
                       cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(g0, gR.data(), sizeof(Real) * gR.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ig0, igR.data(), sizeof(Real) * igR.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

template <typename Real>
emc_status set_temperature_impl(emc_ctx* ctx, int ens, const double* T, int n)
{
    emc_status s;
    if (!ctx->cell_bin && (s = build_bins<Real>(ctx)) != EMC_OK) return s;
    const int C = ctx->ncell;
    int32_t* cb = &ctx->cell_bin_host[(size_t)ens * C];
    for (int c = 0; c < C; ++c) cb[c] = temp_bin(n == 1 ? T[0] : T[c]);
    // Gamma0 of the ensemble: the largest total rate over the bins it uses
    double g_new[NV] = {0, 0, 0}, ratio[NV];
    std::vector<char> used(NTBIN, 0);
    for (int c = 0; c < C; ++c) used[cb[c]] = 1;
    for (int k = 0; k < NTBIN; ++k)
        if (used[k])
            for (int v = 0; v < NV; ++v) g_new[v] = std::max(g_new[v], ctx->bin_g0[(size_t)k * NV + v]);
    for (int v = 0; v < NV; ++v) {
        ratio[v] = ctx->ens_g0_host[(size_t)ens * NV + v] / g_new[v];
        ctx->ens_g0_host[(size_t)ens * NV + v] = g_new[v];
    }
    Real gR[NV], igR[NV];
    for (int v = 0; v < NV; ++v) {
        gR[v] = Real(g_new[v]);
        igR[v] = Real(1.0 / g_new[v]);
    }
    CK(cudaMemcpyAsync(ctx->cell_bin + (size_t)ens * C, cb, sizeof(int32_t) * C, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(static_cast<Real*>(ctx->ens_g0) + (size_t)ens * NV, gR, sizeof gR, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(static_cast<Real*>(ctx->ens_ig0) + (size_t)ens * NV, igR, sizeof igR, cudaMemcpyHostToDevice,
                       ctx->st));
    double* d_ratio = nullptr;
    CK(cudaMallocAsync(&d_ratio, sizeof ratio, ctx->st));
    CK(cudaMemcpyAsync(d_ratio, ratio, sizeof ratio, cudaMemcpyHostToDevice, ctx->st));
    fill_params(ctx);
    launch_rescale<Real>(ctx->P, ens, ctx->cap[ens], d_ratio, ctx->st);
    ctx->launches += 1;
    CK(cudaFreeAsync(d_ratio, ctx->st));
    CK(cudaGetLastError());
    // the captured chunk tail holds the old kernel parameters
    if (ctx->g_tail_exec) {
        CK(cudaGraphExecDestroy(ctx->g_tail_exec));
        CK(cudaGraphDestroy(ctx->g_tail));
        ctx->g_tail_exec = nullptr;
        ctx->g_tail = nullptr;
    }
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

// bytes of tally `kind` for E ensembles of C subcells (0: unknown kind)
size_t tally_bytes(int E, int C, int kind)
{
    switch (kind) {
    case EMC_TALLY_OBS: return sizeof(emc_obs) * (size_t)E;
    case EMC_TALLY_EVENTS: return 8ull * E * NV * NM;
    case EMC_TALLY_HEAT: return 8ull * E * C * 2;
    case EMC_TALLY_CHARGE: return 8ull * E * C;
    case EMC_TALLY_CROSSINGS: return 8ull * E * 4;
    case EMC_TALLY_PHI: return 8ull * E * C;
    case EMC_TALLY_FIELD: return 8ull * E * C * 3;
    case EMC_TALLY_HEAT_J: return 8ull * E * C;
    case EMC_TALLY_EVENTS_CELL: return 8ull * E * C * NV * NM;
    default: return 0;
    }
}

// bytes of the device staging buffer: the largest tally packed on the device
size_t stage_bytes(int E, int C)
{
    size_t b = 0;
    for (int k : {EMC_TALLY_OBS, EMC_TALLY_EVENTS, EMC_TALLY_HEAT, EMC_TALLY_CHARGE, EMC_TALLY_CROSSINGS,
                  EMC_TALLY_PHI, EMC_TALLY_FIELD, EMC_TALLY_HEAT_J})
        b = std::max(b, tally_bytes(E, C, k));
    return b;
}

// A tally in its ABI layout, computed on the device from the accumulators:
// observations and crossings per ensemble, event counts per ensemble (summed
// over subcells), subcell charge (bulk: live count), net phonon emissions per
// subcell and their energy (from the per-subcell event counts: polar optical
// emissions 2 minus absorptions 1; intervalley emissions 5, 7, 9 minus
// absorptions 4, 6, 8), and the zero potential and uniform field of bulk
// ensembles.  par[E][6] = {hw_lo, hw_iv, w, Fx, Fy, Fz}.
__device__ __forceinline__ void net_phonons(const unsigned long long* ev, long long* pop, long long* iv)
{
    long long a = 0, b = 0;
    for (int v = 0; v < NV; ++v) {
        const unsigned long long* r = ev + v * NM;
        a += (long long)r[2] - (long long)r[1];
        for (int j = 0; j < NV; ++j) b += (long long)r[5 + 2 * j] - (long long)r[4 + 2 * j];
    }
    *pop = a;
    *iv = b;
}

__global__ void k_tally_pack(int kind, int E, int C, int nw, const unsigned long long* cnt, const double* sums,
                             const long long* alive, const int* charge, const unsigned long long* events,
                             const double* par, long long steps_done, void* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kind == EMC_TALLY_OBS) {
        if (i >= E) return;
        const unsigned long long* c = cnt + i * NCNT;
        const double* sm = sums + i * NSUM;
        emc_obs q;
        for (int k = 0; k < 3; ++k) q.sum_v[k] = sm[SUM_VX + k] * 1e6;
        q.sum_E = sm[SUM_E] * kQ;
        q.sum_Etot = sm[SUM_ETOT] * kQ;
        q.n_samples = (int64_t)c[CNT_SAMPLES];
        for (int k = 0; k < 3; ++k) {
            q.valley_steps[k] = (int64_t)c[CNT_V0 + k];
            q.self_events[k] = (int64_t)c[CNT_SELF0 + k];
        }
        q.overflow = (int64_t)c[CNT_OVERFLOW];
        q.steps_done = steps_done;
        q.n_alive = (int64_t)alive[i];
        q.inject_starved = (int64_t)c[CNT_STARVED];
        static_cast<emc_obs*>(out)[i] = q;
    } else if (kind == EMC_TALLY_CROSSINGS) {
        if (i >= E) return;
        int64_t* o = static_cast<int64_t*>(out) + 4 * i;
        const unsigned long long* c = cnt + i * NCNT;
        o[0] = (int64_t)c[CNT_SRC_OUT];
        o[1] = (int64_t)c[CNT_DRN_OUT];
        o[2] = (int64_t)c[CNT_SRC_IN];
        o[3] = (int64_t)c[CNT_DRN_IN];
    } else if (kind == EMC_TALLY_EVENTS) {
        // one thread per (ensemble, valley x mechanism), summing the subcells
        if (i >= (int64_t)E * NV * NM) return;
        const int64_t e = i / (NV * NM), j = i - e * (NV * NM);
        const unsigned long long* ev = events + (size_t)e * C * NV * NM + j;
        unsigned long long sum = 0;
        for (int c = 0; c < C; ++c) sum += ev[(size_t)c * NV * NM];
        static_cast<unsigned long long*>(out)[i] = sum;
    } else if (kind == EMC_TALLY_CHARGE) {
        if (i >= (int64_t)E * C) return;
        static_cast<int64_t*>(out)[i] = nw ? (int64_t)charge[i] : (int64_t)alive[i / C];
    } else if (kind == EMC_TALLY_HEAT || kind == EMC_TALLY_HEAT_J) {
        if (i >= (int64_t)E * C) return;
        long long pop, iv;
        net_phonons(events + (size_t)i * NV * NM, &pop, &iv);
        if (kind == EMC_TALLY_HEAT) {
            static_cast<int64_t*>(out)[2 * i] = pop;
            static_cast<int64_t*>(out)[2 * i + 1] = iv;
        } else {
            const double* p = par + 6 * (i / C);
            static_cast<double*>(out)[i] = ((double)pop * p[0] + (double)iv * p[1]) * kQ * p[2];
        }
    } else if (kind == EMC_TALLY_PHI) {
        if (i >= (int64_t)E * C) return;
        static_cast<double*>(out)[i] = 0.0;
    } else if (kind == EMC_TALLY_FIELD) {
        if (i >= (int64_t)E * C * 3) return;
        static_cast<double*>(out)[i] = par[6 * (i / (3 * C)) + 3 + i % 3];
    }
}

bool finite_inputs(const double* charge_or_null, int n, const double* bc)
{
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(bc[i])) return false;
    if (charge_or_null)
        for (int i = 0; i < n; ++i)
            if (!std::isfinite(charge_or_null[i])) return false;
    return true;
}

emc_status check_err(emc_ctx* ctx)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h) {
        char buf[192];
        snprintf(buf, sizeof buf, "device error word 0x%x (1: flight loop bound, 2: non-finite particle energy, "
                                  "4: initial-energy draws, 8: index out of range (checked build))", h);
        return fail(ctx, EMC_EOVERFLOW, buf);
    }
    return EMC_OK;
}

template <typename Real>
emc_status init_impl(emc_ctx* ctx)
{
    emc_status s;
    if ((s = build_tables_and_phys<Real>(ctx)) != EMC_OK) return s;
    if ((s = alloc_particles<Real>(ctx)) != EMC_OK) return s;
    fill_params(ctx);
    {
        const size_t smem = flight_smem_bytes<Real>(ctx->P.nb_smem, ctx->n_tab <= 64 ? ctx->n_tab : 0);
        CK(flight_set_smem<Real>(smem));
        int dev = 0, nsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        ctx->grid_cap = nsm * flight_blocks_per_sm<Real>(ctx->geom == EMC_GEOM_NANOWIRE, ctx->block, smem);
    }
    launch_init<Real>(ctx->P, ctx->geom == EMC_GEOM_NANOWIRE, ctx->st);
    ctx->launches += 1;
    CK(cudaGetLastError());
    if (ctx->geom == EMC_GEOM_NANOWIRE) {
        if ((s = poisson_setup(ctx)) != EMC_OK) return s;
        // initial charge count and field
        CK(cudaMemsetAsync(ctx->charge, 0, sizeof(int) * (size_t)ctx->n_ens * ctx->ncell, ctx->st));
        launch_flight<Real>(ctx->P, true, 0, 1, ctx->block, ctx->grid_cap, ctx->st);
        ctx->launches += 1;
        if (ctx->sharded) ctx->shard_pending = 1;  // the wire's count first (emc_shard_tail)
        else if ((s = poisson_update<Real>(ctx)) != EMC_OK) return s;
    }
    CK(cudaGetLastError());
    return check_err(ctx);
}

// Contact refill, Poisson update and field after a chunk: captured once into
// a CUDA graph (fixed pointers and sizes) and replayed.
template <typename Real>
emc_status chunk_tail(emc_ctx* ctx)
{
    const int sweeps = std::is_same<Real, float>::value ? kPoissonSweepsStepF32 : kPoissonSweeps;
    if (!ctx->use_graph) {
        launch_inject<Real>(ctx->P, ctx->st);
        ctx->launches += 1;
        return poisson_update<Real>(ctx, sweeps);
    }
    if (!ctx->g_tail_exec) {
        const int64_t l0 = ctx->launches;
        CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
        launch_inject<Real>(ctx->P, ctx->st);
        ctx->launches += 1;
        emc_status s = poisson_update<Real>(ctx, sweeps);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
        if (s != EMC_OK) return s;
        CK(e);
        ctx->g_tail = g;
        CK(cudaGraphInstantiate(&ctx->g_tail_exec, g, 0));
        ctx->g_tail_launches = ctx->launches - l0;
        ctx->launches = l0;
    }
    CK(cudaGraphLaunch(ctx->g_tail_exec, ctx->st));
    ctx->launches += ctx->g_tail_launches;
    return EMC_OK;
}

emc_status prof_pair(emc_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b)
{
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    *a = ctx->ev_pool[ctx->ev_used];
    *b = ctx->ev_pool[ctx->ev_used + 1];
    ctx->ev_used += 2;
    return EMC_OK;
}

template <typename Real>
emc_status step_impl(emc_ctx* ctx, int32_t n)
{
    const bool nw = ctx->geom == EMC_GEOM_NANOWIRE;
    while (n > 0) {
        int chunk;
        bool boundary = false;
        if (nw) {
            const int into = int(ctx->steps_done % ctx->K);
            chunk = std::min(n, ctx->K - into);
            boundary = (into + chunk == ctx->K);
            if (ctx->sharded && (ctx->shard_pending || n > ctx->K - into))
                return fail(ctx, EMC_EINVAL, ctx->shard_pending ? "shards: exchange pending (emc_shard_tail)"
                                                                : "shards: emc_step may not cross the end of a Poisson period");
            if (boundary)
                CK(cudaMemsetAsync(ctx->charge, 0, sizeof(int) * (size_t)ctx->n_ens * ctx->ncell, ctx->st));
        } else {
            chunk = std::min(n, ctx->spl);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ctx->prof) {
            emc_status s = prof_pair(ctx, &e0, &e1);
            if (s != EMC_OK) return s;
            CK(cudaEventRecord(e0, ctx->st));
        }
        launch_flight<Real>(ctx->P, nw, chunk, boundary ? 1 : 0, ctx->block, ctx->grid_cap, ctx->st);
        ctx->launches += 1;
        if (ctx->prof) CK(cudaEventRecord(e1, ctx->st));
        if (boundary && ctx->sharded) {
            // refill and Poisson update wait for the wire's count
            ctx->shard_pending = 2;
            ctx->steps_done += chunk;
            if (ctx->sort_period > 0) ++ctx->flights_since_sort;
            CK(cudaGetLastError());
            return EMC_OK;
        }
        if (boundary) {
            emc_status s = chunk_tail<Real>(ctx);
            if (s != EMC_OK) return s;
        }
        CK(cudaGetLastError());
        ctx->steps_done += chunk;
        n -= chunk;
        if (ctx->sort_period > 0 && ++ctx->flights_since_sort >= ctx->sort_period && (!nw || boundary)) {
            emc_status s = sort_particles<Real>(ctx);
            if (s != EMC_OK) return s;
            ctx->flights_since_sort = 0;
        }
    }
    return EMC_OK;
}

// Two contexts advanced together: per chunk one flight launch over both
// contexts' particles (each on its own blocks), then each nanowire
// context's refill and Poisson update, each context's sort when due.  The
// chunk is the nanowire contexts' Poisson period (both in phase when both
// are nanowire), else the first context's steps per launch.
template <typename Real>
emc_status pair_step_impl(emc_ctx* a, emc_ctx* b, int32_t n)
{
    emc_ctx* ctx = a;  // errors are reported on the first context
    emc_ctx* c2[2] = {a, b};
    const bool nw[2] = {a->geom == EMC_GEOM_NANOWIRE, b->geom == EMC_GEOM_NANOWIRE};
    const int block = a->block;
    size_t smem = 0;
    int bps = 0;
    CK(pair_prepare<Real>(a->P, nw[0], b->P, nw[1], block, &smem, &bps));
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (a->n_slots + block - 1) / block + (b->n_slots + block - 1) / block;
    const int64_t cap = (int64_t)nsm * (bps > 0 ? bps : 1);
    const int grid = (int)(tiles < cap ? tiles : cap);
    while (n > 0) {
        int chunk = std::min(n, a->spl);
        for (int i = 0; i < 2; ++i)
            if (nw[i]) {
                const int into = int(c2[i]->steps_done % c2[i]->K);
                chunk = std::min(n, c2[i]->K - into);
            }
        bool boundary[2] = {false, false};
        for (int i = 0; i < 2; ++i)
            if (nw[i]) {
                boundary[i] = (c2[i]->steps_done % c2[i]->K) + chunk == c2[i]->K;
                if (boundary[i])
                    CK(cudaMemsetAsync(c2[i]->charge, 0, sizeof(int) * (size_t)c2[i]->n_ens * c2[i]->ncell, a->st));
            }
        launch_flight_pair<Real>(a->P, nw[0], chunk, boundary[0] ? 1 : 0, b->P, nw[1], chunk, boundary[1] ? 1 : 0,
                                 block, grid, smem, a->st);
        a->launches += 1;  // one launch for both contexts
        CK(cudaGetLastError());
        for (int i = 0; i < 2; ++i) {
            emc_ctx* c = c2[i];
            if (boundary[i]) {
                emc_status s = chunk_tail<Real>(c);
                if (s != EMC_OK) return s;
            }
            c->steps_done += chunk;
            if (c->sort_period > 0 && ++c->flights_since_sort >= c->sort_period && (!nw[i] || boundary[i])) {
                emc_status s = sort_particles<Real>(c);
                if (s != EMC_OK) return s;
                c->flights_since_sort = 0;
            }
        }
        CK(cudaGetLastError());
        n -= chunk;
    }
    return EMC_OK;
}

template <typename Real>
emc_status shard_tail_impl(emc_ctx* ctx)
{
    if (ctx->shard_pending == 1) {
        ctx->shard_pending = 0;
        return poisson_update<Real>(ctx);
    }
    ctx->shard_pending = 0;
    emc_status s = chunk_tail<Real>(ctx);
    if (s != EMC_OK) return s;
    if (ctx->sort_period > 0 && ctx->flights_since_sort >= ctx->sort_period) {
        if ((s = sort_particles<Real>(ctx)) != EMC_OK) return s;
        ctx->flights_since_sort = 0;
    }
    return EMC_OK;
}

}  // namespace

// =================================================================== ABI
extern "C" {

emc_status emc_batch_init(const emc_config* cfgs, int32_t n_ens, void* stream, emc_ctx** out)
{
    EMC_TRACE("emc_batch_init");
    if (!out) return EMC_EINVAL;
    *out = nullptr;
    emc_ctx* ctx = new (std::nothrow) emc_ctx();
    if (!ctx) return EMC_ENOMEM;
    emc_status s = validate(cfgs, n_ens, ctx);
    if (s != EMC_OK) {
        *out = ctx;  // keep the message readable through emc_last_error
        return s;
    }
    ctx->st = static_cast<cudaStream_t>(stream);
    ctx->use_graph = ctx->st != nullptr;  // the legacy default stream cannot be captured
    ctx->cfg.assign(cfgs, cfgs + n_ens);
    const emc_config& c0 = cfgs[0];
    ctx->n_ens = n_ens;
    ctx->prec = c0.precision;
    ctx->geom = c0.geometry;
    ctx->nb = c0.n_bins;
    ctx->dE = c0.dE_eV;
    ctx->dt_fs = c0.dt_s * 1e15;
    ctx->block = c0.block_size ? c0.block_size : 256;
    ctx->spl = c0.steps_per_launch > 0 ? c0.steps_per_launch : 50;
    ctx->K = c0.steps_per_poisson > 0 ? c0.steps_per_poisson : 10;
    ctx->sort_period = c0.sort_period;
    if (ctx->geom == EMC_GEOM_NANOWIRE) {
        ctx->nx = c0.nx; ctx->ny = c0.ny; ctx->nz = c0.nz;
        ctx->Lx = c0.Lx * 1e9; ctx->Ly = c0.Ly * 1e9; ctx->Lz = c0.Lz * 1e9;
        ctx->dx = ctx->Lx / c0.nx; ctx->dy = ctx->Ly / c0.ny; ctx->dz = ctx->Lz / c0.nz;
        ctx->gate_ix.resize(c0.nx);
        for (int i = 0; i < c0.nx; ++i) {
            const double xc = (i + 0.5) * c0.Lx / c0.nx;
            ctx->gate_ix[i] = (c0.gate_on && xc >= c0.gate_x0 && xc <= c0.gate_x1) ? 1 : 0;
        }
    }
    ctx->ncell = ctx->nx * ctx->ny * ctx->nz;
    // slots, table sets
    ctx->off.resize(n_ens);
    ctx->cap.resize(n_ens);
    ctx->n0.resize(n_ens);
    ctx->tabset.resize(n_ens);
    ctx->w.resize(n_ens);
    ctx->bias.resize((size_t)3 * n_ens);
    std::vector<int64_t> bits_off(n_ens);
    std::vector<uint32_t> seeds(n_ens);
    std::vector<int32_t> target(n_ens);
    std::vector<uint32_t> gid((size_t)2 * n_ens);
    ctx->sharded = cfgs[0].shard_n_global > 0;
    int64_t o = 0, bo = 0;
    for (int e = 0; e < n_ens; ++e) {
        const emc_config& c = cfgs[e];
        ctx->off[e] = o;
        ctx->cap[e] = std::max<int64_t>(c.capacity, c.n_particles);
        ctx->n0[e] = c.n_particles;
        o += ctx->cap[e];
        bits_off[e] = bo;
        bo += (ctx->cap[e] + 31) / 32;
        seeds[e] = c.seed;
        int ts = -1;
        for (int f = 0; f < e && ts < 0; ++f)
            if (same_table(cfgs[f], c)) ts = ctx->tabset[f];
        if (ts < 0) {
            ts = ctx->n_tab++;
            ctx->rc.push_back(make_rc(c));
        }
        ctx->tabset[e] = ts;
        const double V = c.Lx * c.Ly * c.Lz;
        // the wire's initial electrons (all shards) set the superparticle weight
        const int64_t n_wire = ctx->sharded ? c.shard_n_global : c.n_particles;
        gid[2 * e] = ctx->sharded ? uint32_t(c.shard_live_base) : 0u;
        gid[2 * e + 1] = ctx->sharded ? uint32_t(c.shard_spare_base) : uint32_t(c.n_particles);
        ctx->w[e] = (ctx->geom == EMC_GEOM_NANOWIRE && n_wire > 0) ? c.Nd_m3 * V / (double)n_wire : 1.0;
        const double Vcell = V / ctx->ncell;
        target[e] = (ctx->geom == EMC_GEOM_NANOWIRE) ? (int32_t)std::llround(c.Nd_m3 * Vcell / ctx->w[e]) : 0;
        ctx->bias[3 * e] = c.Vs;
        ctx->bias[3 * e + 1] = c.Vd;
        ctx->bias[3 * e + 2] = c.Vg;
    }
    ctx->n_slots = o;
    ctx->bits_words = bo;
    *out = ctx;
#define CKI(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(ctx, EMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    const size_t n = (size_t)ctx->n_slots;
    CKI(dalloc(ctx, &ctx->tag, n));
    CKI(dalloc(ctx, &ctx->id, n));
    CKI(dalloc(ctx, &ctx->slot_of_id, n));
    CKI(dalloc(ctx, &ctx->ctr, n));
    CKI(dalloc(ctx, &ctx->dead_bits, (size_t)bo));
    CKI(dalloc(ctx, &ctx->d_off, n_ens));
    CKI(dalloc(ctx, &ctx->d_cap, n_ens));
    CKI(dalloc(ctx, &ctx->d_n0, n_ens));
    CKI(dalloc(ctx, &ctx->d_bits_off, n_ens));
    CKI(dalloc(ctx, &ctx->d_seed, n_ens));
    CKI(dalloc(ctx, &ctx->d_tabset, n_ens));
    CKI(dalloc(ctx, &ctx->d_target, n_ens));
    CKI(dalloc(ctx, &ctx->d_gid, (size_t)2 * n_ens));
    if (ctx->sharded) {
        CKI(dalloc(ctx, &ctx->d_shard, (size_t)5 * n_ens));
        CKI(dalloc(ctx, &ctx->d_free, (size_t)2 * n_ens));
    }
    CKI(dalloc(ctx, &ctx->events, (size_t)n_ens * ctx->ncell * NV * NM));
    CKI(dalloc(ctx, &ctx->cnt, (size_t)n_ens * NCNT));
    CKI(dalloc(ctx, &ctx->sums, (size_t)n_ens * NSUM));
    CKI(dalloc(ctx, &ctx->charge, (size_t)n_ens * ctx->ncell));
    CKI(dalloc(ctx, &ctx->alive, n_ens));
    CKI(dalloc(ctx, &ctx->d_err, 1));
    auto up = [&](void* d, const void* h, size_t b) {
        return cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, ctx->st);
    };
    CKI(up(ctx->d_off, ctx->off.data(), 8 * n_ens));
    CKI(up(ctx->d_cap, ctx->cap.data(), 8 * n_ens));
    CKI(up(ctx->d_n0, ctx->n0.data(), 8 * n_ens));
    CKI(up(ctx->d_bits_off, bits_off.data(), 8 * n_ens));
    CKI(up(ctx->d_seed, seeds.data(), 4 * n_ens));
    CKI(up(ctx->d_tabset, ctx->tabset.data(), 4 * n_ens));
    CKI(up(ctx->d_target, target.data(), 4 * n_ens));
    CKI(up(ctx->d_gid, gid.data(), 8 * n_ens));
    CKI(up(ctx->alive, ctx->n0.data(), 8 * n_ens));
#undef CKI
    if (ctx->prec == EMC_FP64) return init_impl<double>(ctx);
    return init_impl<float>(ctx);
}

emc_status emc_init(const emc_config* cfg, void* stream, emc_ctx** out)
{
    return emc_batch_init(cfg, 1, stream, out);
}

emc_status emc_step(emc_ctx* ctx, int32_t n_steps)
{
    EMC_TRACE("emc_step");
    if (!ctx) return EMC_EINVAL;
    if (n_steps < 0) return fail(ctx, EMC_EINVAL, "n_steps < 0");
    if (n_steps == 0) return EMC_OK;
    emc_status s = ctx->prec == EMC_FP64 ? step_impl<double>(ctx, n_steps) : step_impl<float>(ctx, n_steps);
    if (s != EMC_OK) return s;
    return EMC_OK;
}

emc_status emc_tally(emc_ctx* ctx, int32_t kind, void* dst, size_t bytes, int32_t dst_is_device, int32_t reset)
{
    EMC_TRACE("emc_tally");
    if (!ctx || !dst) return EMC_EINVAL;
    const size_t need = tally_bytes(ctx->n_ens, ctx->ncell, kind);
    if (need == 0) return fail(ctx, EMC_EINVAL, "unknown tally kind");
    if (bytes < need) return fail(ctx, EMC_EINVAL, "destination too small");
    emc_status s = check_err(ctx);
    if (s != EMC_OK) return s;
    if ((s = emc_tally_async(ctx, kind, dst, bytes, dst_is_device, reset)) != EMC_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

emc_status emc_tally_async(emc_ctx* ctx, int32_t kind, void* dst, size_t bytes, int32_t dst_is_device, int32_t reset)
{
    EMC_TRACE("emc_tally_async");
    if (!ctx || !dst) return EMC_EINVAL;
    const int E = ctx->n_ens, C = ctx->ncell;
    const bool nw = ctx->geom == EMC_GEOM_NANOWIRE;
    const size_t need = tally_bytes(E, C, kind);
    if (need == 0) return fail(ctx, EMC_EINVAL, "unknown tally kind");
    if (bytes < need) return fail(ctx, EMC_EINVAL, "destination too small");
    const cudaMemcpyKind dir = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const void* direct = kind == EMC_TALLY_EVENTS_CELL ? (const void*)ctx->events
                       : (kind == EMC_TALLY_EVENTS && C == 1) ? (const void*)ctx->events
                       : (nw && kind == EMC_TALLY_PHI) ? (const void*)ctx->phi
                       : (nw && kind == EMC_TALLY_FIELD) ? (const void*)ctx->Efield : nullptr;
    if (direct) {
        CK(cudaMemcpyAsync(dst, direct, need, dir, ctx->st));
    } else {
        if (!ctx->tstage) {
            CK(dalloc(ctx, &ctx->tstage, stage_bytes(E, C)));
            CK(dalloc(ctx, &ctx->tpar, (size_t)6 * E));
            std::vector<double> par((size_t)6 * E);
            for (int e = 0; e < E; ++e) {
                const emc_config& c = ctx->cfg[e];
                double* q = &par[(size_t)6 * e];
                q[0] = c.hw_lo_eV; q[1] = c.hw_iv_eV; q[2] = ctx->w[e];
                q[3] = nw ? 0.0 : c.field_V_m[0]; q[4] = nw ? 0.0 : c.field_V_m[1]; q[5] = nw ? 0.0 : c.field_V_m[2];
            }
            CK(cudaMemcpyAsync(ctx->tpar, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice, ctx->st));
            // the parameters must be on the device before the host vector goes
            CK(cudaStreamSynchronize(ctx->st));
        }
        void* out = dst_is_device ? dst : (void*)ctx->tstage;
        const int64_t items = kind == EMC_TALLY_OBS || kind == EMC_TALLY_CROSSINGS ? E
                            : kind == EMC_TALLY_EVENTS ? (int64_t)E * NV * NM
                            : kind == EMC_TALLY_FIELD ? (int64_t)E * C * 3 : (int64_t)E * C;
        k_tally_pack<<<grid_for(items, 256), 256, 0, ctx->st>>>(kind, E, C, nw ? 1 : 0, ctx->cnt, ctx->sums, ctx->alive,
                                                                  ctx->charge, ctx->events, ctx->tpar, ctx->steps_done,
                                                                  out);
        ctx->launches += 1;
        if (!dst_is_device) CK(cudaMemcpyAsync(dst, ctx->tstage, need, cudaMemcpyDeviceToHost, ctx->st));
    }
    if (reset) {
        CK(cudaMemsetAsync(ctx->events, 0, 8ull * E * C * NV * NM, ctx->st));
        CK(cudaMemsetAsync(ctx->cnt, 0, 8ull * E * NCNT, ctx->st));
        CK(cudaMemsetAsync(ctx->sums, 0, 8ull * E * NSUM, ctx->st));
    }
    CK(cudaGetLastError());
    return EMC_OK;
}

emc_status poisson_solve(emc_ctx* ctx, const double* charge_or_null, const double* bc_volts, double* phi_out)
{
    EMC_TRACE("poisson_solve");
    if (!ctx || !bc_volts) return EMC_EINVAL;
    if (ctx->geom != EMC_GEOM_NANOWIRE) return fail(ctx, EMC_ESTATE, "poisson_solve needs the nanowire geometry");
    if (!finite_inputs(charge_or_null, ctx->ncell, bc_volts))
        return fail(ctx, EMC_EINVAL, "poisson_solve: charge density and voltages must be finite");
    const int n = ctx->ncell;
    double *rho = nullptr, *rhs = nullptr, *phi = nullptr, *bias = nullptr;
    float* r32 = nullptr;
    CK(cudaMallocAsync(&rho, 8 * n, ctx->st));
    CK(cudaMallocAsync(&rhs, 8 * n, ctx->st));
    CK(cudaMallocAsync(&phi, 8 * n, ctx->st));
    CK(cudaMallocAsync(&bias, 8 * 3, ctx->st));
    float* part = nullptr;
    CK(cudaMallocAsync(&r32, 4 * (size_t)n, ctx->st));
    CK(cudaMallocAsync(&part, 4 * (size_t)sweep_slices(n) * n, ctx->st));
    CK(cudaMemsetAsync(phi, 0, 8 * n, ctx->st));
    CK(cudaMemcpyAsync(bias, bc_volts, 24, cudaMemcpyHostToDevice, ctx->st));
    PoisGeo G = pgeo(ctx);
    const double Vcell = ctx->dx * ctx->dy * ctx->dz;
    if (charge_or_null) {
        CK(cudaMemcpyAsync(rho, charge_or_null, 8 * n, cudaMemcpyHostToDevice, ctx->st));
        k_rhs<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, nullptr, rho, ctx->d_w, ctx->d_Nd, Vcell,
                                                     kE2Eps0 / ctx->cfg[0].eps_s, bias, rhs);
    } else {
        k_rhs<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, ctx->charge, nullptr, ctx->d_w, ctx->d_Nd, Vcell,
                                                     kE2Eps0 / ctx->cfg[0].eps_s, bias, rhs);
    }
    for (int s = 0; s < kPoissonSweeps + 1; ++s) {
        k_resid<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, rhs, phi, r32);
        launch_sweep(ctx->G32, r32, part, phi, n, 1, ctx->st);
    }
    ctx->launches += 1 + 3 * (kPoissonSweeps + 1);
    CK(cudaGetLastError());
    if (phi_out) CK(cudaMemcpyAsync(phi_out, phi, 8 * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaFreeAsync(rho, ctx->st));
    CK(cudaFreeAsync(rhs, ctx->st));
    CK(cudaFreeAsync(phi, ctx->st));
    CK(cudaFreeAsync(bias, ctx->st));
    CK(cudaFreeAsync(r32, ctx->st));
    CK(cudaFreeAsync(part, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

}  // extern "C"

// accessors used by the thermal unit
namespace emc {
cudaStream_t ctx_stream(emc_ctx* ctx) { return ctx->st; }
int ctx_grid(emc_ctx* ctx, int* nx, int* ny, int* nz, double* Lx, double* Ly, double* Lz, int* n_ens)
{
    if (ctx->geom != EMC_GEOM_NANOWIRE) return 0;
    *nx = ctx->nx; *ny = ctx->ny; *nz = ctx->nz;
    *Lx = ctx->cfg[0].Lx; *Ly = ctx->cfg[0].Ly; *Lz = ctx->cfg[0].Lz;
    *n_ens = ctx->n_ens;
    return 1;
}
emc_status ctx_fail(emc_ctx* ctx, emc_status s, const char* msg) { return fail(ctx, s, msg); }
void ctx_count_launches(emc_ctx* ctx, int64_t n) { ctx->launches += n; }
}  // namespace emc

// ------------------------------------------- allocation-free Poisson solve
// Scratch of emc_poisson_solve_static: right-hand side, potential and charge
// density (double[kStaticCells] each), the three terminal voltages, and the
// float residual, in one file-scope device array that lives as long as the
// library is loaded on each device that uses it.
namespace {
constexpr int kStaticCells = 8192;
constexpr int kStaticSlices = (kStaticCells + 191) / 192;
constexpr size_t kStaticDoubles = 3 * (size_t)kStaticCells + 4 + kStaticCells / 2 +
                                  (size_t)kStaticSlices * kStaticCells / 2;
static __device__ __align__(256) double g_poisson_scratch[kStaticDoubles];

// Device address of the scratch array, looked up with cudaGetSymbolAddress
// once per CUDA context (the host-side symbol itself is not a device
// address).  The cache is keyed by the context's unique id, so a context
// created anew after a device reset (which reloads the module) gets its own
// lookup instead of a stale address.
typedef CUresult (*ctx_current_fn)(CUcontext*);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long*);
std::mutex g_scratch_mu;
std::map<unsigned long long, void*> g_scratch_addr;

emc_status static_scratch(emc_ctx* ctx, double** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        CK(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                            cudaEnableDefault, &q1));
        CK(cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000,
                                            cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            get_current = nullptr;
            get_id = nullptr;
            return fail(ctx, EMC_ECUDA, "static scratch: driver context queries unavailable");
        }
    }
    CUcontext cu = nullptr;
    unsigned long long id = 0;
    if (get_current(&cu) != CUDA_SUCCESS || !cu || get_id(cu, &id) != CUDA_SUCCESS)
        return fail(ctx, EMC_ESTATE, "static scratch: no current CUDA context on this thread");
    auto it = g_scratch_addr.find(id);
    if (it == g_scratch_addr.end()) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_poisson_scratch));
        it = g_scratch_addr.emplace(id, p).first;
    }
    *out = static_cast<double*>(it->second);
    return EMC_OK;
}
}  // namespace

extern "C" {

emc_status emc_poisson_solve_static(emc_ctx* ctx, const double* charge_or_null, const double* bc_volts,
                                    double* phi_out_or_null)
{
    EMC_TRACE("emc_poisson_solve_static");
    if (!ctx || !bc_volts) return EMC_EINVAL;
    if (ctx->geom != EMC_GEOM_NANOWIRE)
        return fail(ctx, EMC_ESTATE, "emc_poisson_solve_static needs the nanowire geometry");
    if (!finite_inputs(charge_or_null, ctx->ncell, bc_volts))
        return fail(ctx, EMC_EINVAL, "emc_poisson_solve_static: charge density and voltages must be finite");
    const int n = ctx->ncell;
    if (n > kStaticCells) {
        char buf[160];
        snprintf(buf, sizeof buf, "emc_poisson_solve_static: %d subcells exceed its static scratch limit of %d", n,
                 kStaticCells);
        return fail(ctx, EMC_EINVAL, buf);
    }
    double* base = nullptr;
    emc_status st = static_scratch(ctx, &base);
    if (st != EMC_OK) return st;
    double* rhs = base;
    double* phi = base + kStaticCells;
    double* rho = base + 2 * (size_t)kStaticCells;
    double* bias = base + 3 * (size_t)kStaticCells;
    float* r32 = reinterpret_cast<float*>(base + 3 * (size_t)kStaticCells + 4);
    float* part = r32 + kStaticCells;
    // the previous call's contents are still there: start the potential at zero
    CK(cudaMemsetAsync(phi, 0, 8 * (size_t)n, ctx->st));
    CK(cudaMemcpyAsync(bias, bc_volts, 24, cudaMemcpyHostToDevice, ctx->st));
    PoisGeo G = pgeo(ctx);
    const double Vcell = ctx->dx * ctx->dy * ctx->dz;
    if (charge_or_null) {
        CK(cudaMemcpyAsync(rho, charge_or_null, 8 * (size_t)n, cudaMemcpyHostToDevice, ctx->st));
        k_rhs<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, nullptr, rho, ctx->d_w, ctx->d_Nd, Vcell,
                                                     kE2Eps0 / ctx->cfg[0].eps_s, bias, rhs);
    } else {
        k_rhs<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, ctx->charge, nullptr, ctx->d_w, ctx->d_Nd, Vcell,
                                                     kE2Eps0 / ctx->cfg[0].eps_s, bias, rhs);
    }
    // the same sweeps as poisson_solve, so the two give the same potential
    for (int sw = 0; sw < kPoissonSweeps + 1; ++sw) {
        k_resid<<<grid_for(n, 256), 256, 0, ctx->st>>>(G, 1, rhs, phi, r32);
        launch_sweep(ctx->G32, r32, part, phi, n, 1, ctx->st);
    }
    ctx->launches += 1 + 3 * (kPoissonSweeps + 1);
    CK(cudaGetLastError());
    if (phi_out_or_null)
        CK(cudaMemcpyAsync(phi_out_or_null, phi, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

// ------------------------------------------------------- checkpoint/resume
// The blob: StateHeader, then the sections of state_sections() in order.
namespace {
constexpr uint64_t kStateMagic = 0x4554415453434d45ull;  // "EMCSTATE"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
    uint64_t magic;
    uint32_t version, precision, geometry, tmode;
    int32_t n_ens, ncell;
    int64_t n_slots, bits_words, steps_done, flights_since_sort;
    uint64_t cfg_hash;
};
static_assert(sizeof(StateHeader) == 72, "the state header layout is part of the ABI");

// FNV-1a over the configurations, launch-tuning fields zeroed: a state can
// only be restored into a context made from the same ensembles
uint64_t cfg_hash(const emc_ctx* ctx)
{
    uint64_t h = 1469598103934665603ull;
    // the fields up to the last one (trailing padding bytes are not hashed)
    const size_t used = offsetof(emc_config, table_smem_kb) + sizeof(int32_t);
    for (emc_config c : ctx->cfg) {
        c.sort_period = c.block_size = c.steps_per_launch = c.table_smem_kb = 0;
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&c);
        for (size_t i = 0; i < used; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
    return h;
}

struct Section {
    void* p;        // device buffer, or host memory when host = true
    size_t bytes;
    bool host;
};

std::vector<Section> state_sections(emc_ctx* ctx, bool tmode)
{
    const size_t n = (size_t)ctx->n_slots, E = ctx->n_ens, C = ctx->ncell;
    const size_t es = ctx->prec == EMC_FP64 ? 8 : 4;
    const bool nw = ctx->geom == EMC_GEOM_NANOWIRE;
    std::vector<Section> v = {{ctx->kx, es * n, false}, {ctx->ky, es * n, false}, {ctx->kz, es * n, false}};
    if (nw) v.insert(v.end(), {{ctx->x, es * n, false}, {ctx->y, es * n, false}, {ctx->z, es * n, false}});
    v.insert(v.end(), {{ctx->tr, es * n, false}, {ctx->tag, 4 * n, false}, {ctx->ctr, 8 * n, false},
                       {ctx->id, 4 * n, false}, {ctx->slot_of_id, 4 * n, false},
                       {ctx->dead_bits, 4 * (size_t)ctx->bits_words, false},
                       {ctx->events, 8 * E * C * NV * NM, false}, {ctx->cnt, 8 * E * NCNT, false},
                       {ctx->sums, 8 * E * NSUM, false}, {ctx->charge, 4 * E * C, false}, {ctx->alive, 8 * E, false},
                       {ctx->d_err, 4, false}, {ctx->bias.data(), 8 * 3 * E, true}});
    if (nw)
        v.insert(v.end(), {{ctx->d_bias, 8 * 3 * E, false}, {ctx->phi, 8 * E * C, false},
                           {ctx->Efield, 24 * E * C, false}, {ctx->acc_cell, 4 * es * E * C, false}});
    if (tmode)
        v.insert(v.end(), {{ctx->cell_bin, 4 * E * C, false}, {ctx->ens_g0, es * E * NV, false},
                           {ctx->ens_ig0, es * E * NV, false}, {ctx->ens_g0_host.data(), 8 * E * NV, true},
                           {ctx->cell_bin_host.data(), 4 * E * C, true}});
    return v;
}

size_t state_bytes(emc_ctx* ctx, bool tmode)
{
    size_t b = sizeof(StateHeader);
    for (const Section& s : state_sections(ctx, tmode)) b += s.bytes;
    return b;
}
}  // namespace

emc_status emc_state_size(emc_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return EMC_EINVAL;
    *bytes = state_bytes(ctx, ctx->cell_bin != nullptr);
    return EMC_OK;
}

emc_status emc_get_state(emc_ctx* ctx, void* dst, size_t bytes)
{
    EMC_TRACE("emc_get_state");
    if (!ctx || !dst) return EMC_EINVAL;
    if (ctx->shard_pending) return fail(ctx, EMC_EINVAL, "shards: exchange pending (emc_shard_tail)");
    const bool tmode = ctx->cell_bin != nullptr;
    if (bytes < state_bytes(ctx, tmode)) return fail(ctx, EMC_EINVAL, "emc_get_state: destination too small");
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.precision = (uint32_t)ctx->prec;
    h.geometry = (uint32_t)ctx->geom;
    h.tmode = tmode ? 1u : 0u;
    h.n_ens = ctx->n_ens;
    h.ncell = ctx->ncell;
    h.n_slots = ctx->n_slots;
    h.bits_words = ctx->bits_words;
    h.steps_done = ctx->steps_done;
    h.flights_since_sort = ctx->flights_since_sort;
    h.cfg_hash = cfg_hash(ctx);
    unsigned char* out = static_cast<unsigned char*>(dst);
    std::memcpy(out, &h, sizeof h);
    size_t off = sizeof h;
    for (const Section& s : state_sections(ctx, tmode)) {
        if (s.host) std::memcpy(out + off, s.p, s.bytes);
        else if (s.bytes) CK(cudaMemcpyAsync(out + off, s.p, s.bytes, cudaMemcpyDeviceToHost, ctx->st));
        off += s.bytes;
    }
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

emc_status emc_set_state(emc_ctx* ctx, const void* src, size_t bytes)
{
    EMC_TRACE("emc_set_state");
    if (!ctx || !src) return EMC_EINVAL;
    if (ctx->shard_pending) return fail(ctx, EMC_EINVAL, "shards: exchange pending (emc_shard_tail)");
    if (bytes < sizeof(StateHeader)) return fail(ctx, EMC_EINVAL, "emc_set_state: blob too small");
    StateHeader h;
    std::memcpy(&h, src, sizeof h);
    if (h.magic != kStateMagic || h.version != kStateVersion)
        return fail(ctx, EMC_EINVAL, "emc_set_state: not a state blob of this library version");
    if (h.precision != (uint32_t)ctx->prec || h.geometry != (uint32_t)ctx->geom || h.n_ens != ctx->n_ens ||
        h.ncell != ctx->ncell || h.n_slots != ctx->n_slots || h.bits_words != ctx->bits_words ||
        h.cfg_hash != cfg_hash(ctx))
        return fail(ctx, EMC_ESTATE, "emc_set_state: the blob belongs to a context of other ensembles");
    const bool tmode = h.tmode != 0;
    if (!tmode && ctx->cell_bin)
        return fail(ctx, EMC_ESTATE, "emc_set_state: this context has subcell temperatures, the blob has none");
    if (bytes < state_bytes(ctx, tmode)) return fail(ctx, EMC_EINVAL, "emc_set_state: blob too small");
    if (tmode && !ctx->cell_bin) {
        emc_status s = ctx->prec == EMC_FP64 ? build_bins<double>(ctx) : build_bins<float>(ctx);
        if (s != EMC_OK) return s;
        fill_params(ctx);
        if (ctx->g_tail_exec) {  // the captured tail holds the kernel parameters
            CK(cudaGraphExecDestroy(ctx->g_tail_exec));
            CK(cudaGraphDestroy(ctx->g_tail));
            ctx->g_tail_exec = nullptr;
            ctx->g_tail = nullptr;
        }
    }
    CK(cudaStreamSynchronize(ctx->st));
    const unsigned char* in = static_cast<const unsigned char*>(src);
    size_t off = sizeof h;
    for (const Section& s : state_sections(ctx, tmode)) {
        if (s.host) std::memcpy(s.p, in + off, s.bytes);
        else if (s.bytes) CK(cudaMemcpyAsync(s.p, in + off, s.bytes, cudaMemcpyHostToDevice, ctx->st));
        off += s.bytes;
    }
    ctx->steps_done = h.steps_done;
    ctx->flights_since_sort = h.flights_since_sort;
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

emc_status emc_set_bias(emc_ctx* ctx, int32_t ens, double Vs, double Vd, double Vg)
{
    EMC_TRACE("emc_set_bias");
    if (!ctx || ens < 0 || ens >= ctx->n_ens) return EMC_EINVAL;
    if (ctx->shard_pending) return fail(ctx, EMC_EINVAL, "shards: exchange pending (emc_shard_tail)");
    if (!std::isfinite(Vs) || !std::isfinite(Vd) || !std::isfinite(Vg))
        return fail(ctx, EMC_EINVAL, "emc_set_bias: terminal voltages must be finite");
    if (ctx->geom != EMC_GEOM_NANOWIRE) return fail(ctx, EMC_ESTATE, "emc_set_bias needs the nanowire geometry");
    const bool same = ctx->bias[3 * ens] == Vs && ctx->bias[3 * ens + 1] == Vd && ctx->bias[3 * ens + 2] == Vg;
    ctx->bias[3 * ens] = Vs;
    ctx->bias[3 * ens + 1] = Vd;
    ctx->bias[3 * ens + 2] = Vg;
    CK(cudaMemcpyAsync(ctx->d_bias + 3 * ens, &ctx->bias[3 * ens], 24, cudaMemcpyHostToDevice, ctx->st));
    // the field already belongs to these terminal voltages when none changed
    if (!same) {
        emc_status s = ctx->prec == EMC_FP64 ? poisson_update<double>(ctx) : poisson_update<float>(ctx);
        if (s != EMC_OK) return s;
    }
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

emc_status emc_set_bias_all(emc_ctx* ctx, const double* bias)
{
    EMC_TRACE("emc_set_bias_all");
    if (!ctx || !bias) return EMC_EINVAL;
    if (ctx->shard_pending) return fail(ctx, EMC_EINVAL, "shards: exchange pending (emc_shard_tail)");
    if (ctx->geom != EMC_GEOM_NANOWIRE) return fail(ctx, EMC_ESTATE, "emc_set_bias_all needs the nanowire geometry");
    for (int i = 0; i < 3 * ctx->n_ens; ++i)
        if (!std::isfinite(bias[i])) return fail(ctx, EMC_EINVAL, "emc_set_bias_all: terminal voltages must be finite");
    const bool same = std::memcmp(ctx->bias.data(), bias, sizeof(double) * 3 * ctx->n_ens) == 0;
    std::memcpy(ctx->bias.data(), bias, sizeof(double) * 3 * ctx->n_ens);
    CK(cudaMemcpyAsync(ctx->d_bias, bias, sizeof(double) * 3 * ctx->n_ens, cudaMemcpyHostToDevice, ctx->st));
    // the field already belongs to these terminal voltages when none changed
    if (same) return EMC_OK;
    return ctx->prec == EMC_FP64 ? poisson_update<double>(ctx) : poisson_update<float>(ctx);
}

emc_status emc_surrogate_train(emc_ctx* ctx, const emc_mlp_config* net, const float* X, const float* Y, int64_t n,
                               const emc_train_config* tc, float* loss_history)
{
    EMC_TRACE("emc_surrogate_train");
    if (!ctx || !net || !X || !Y || !tc) return EMC_EINVAL;
    if (ctx->sur) {
        emc_mlp_destroy(ctx->sur);
        ctx->sur = nullptr;
    }
    emc_mlp* m = nullptr;
    emc_status s = emc_mlp_create(net, ctx->st, &m);
    if (s == EMC_OK) s = emc_mlp_train(m, X, Y, n, tc, loss_history);
    if (s != EMC_OK) {
        const std::string msg = m ? emc_mlp_last_error(m) : "surrogate network";
        if (m) emc_mlp_destroy(m);
        return fail(ctx, s, "emc_surrogate_train: " + msg);
    }
    ctx->sur = m;
    return EMC_OK;
}

emc_status emc_surrogate_infer(emc_ctx* ctx, const float* X, float* Y, int64_t n)
{
    EMC_TRACE("emc_surrogate_infer");
    if (!ctx || n < 0 || (n > 0 && (!X || !Y))) return EMC_EINVAL;
    if (!ctx->sur) return fail(ctx, EMC_ESTATE, "emc_surrogate_infer: no surrogate trained on this context");
    const emc_status s = emc_mlp_infer(ctx->sur, X, Y, n);
    if (s != EMC_OK) return fail(ctx, s, std::string("emc_surrogate_infer: ") + emc_mlp_last_error(ctx->sur));
    return EMC_OK;
}

emc_status emc_surrogate_params(emc_ctx* ctx, float* dst, int64_t* count)
{
    if (!ctx || !count) return EMC_EINVAL;
    if (!ctx->sur) return fail(ctx, EMC_ESTATE, "emc_surrogate_params: no surrogate trained on this context");
    return emc_mlp_params(ctx->sur, dst, nullptr, count);
}

emc_status emc_profile(emc_ctx* ctx, int32_t enable)
{
    if (!ctx) return EMC_EINVAL;
    ctx->prof = enable != 0;
    if (enable) ctx->ev_used = 0;
    return EMC_OK;
}

emc_status emc_profile_read(emc_ctx* ctx, double* flight_ms, int64_t* flight_launches)
{
    if (!ctx) return EMC_EINVAL;
    CK(cudaStreamSynchronize(ctx->st));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
        tot += ms;
    }
    if (flight_ms) *flight_ms = tot;
    if (flight_launches) *flight_launches = (int64_t)(ctx->ev_used / 2);
    return EMC_OK;
}

emc_status emc_group_step(emc_ctx* const* ctxs, int32_t n_ctx, int32_t n_steps)
{
    EMC_TRACE("emc_group_step");
    if (!ctxs || n_ctx < 1 || n_ctx > 2) return EMC_EINVAL;
    for (int i = 0; i < n_ctx; ++i)
        if (!ctxs[i]) return EMC_EINVAL;
    if (n_ctx == 1) return emc_step(ctxs[0], n_steps);
    emc_ctx *a = ctxs[0], *b = ctxs[1];
    if (a == b) return fail(a, EMC_EINVAL, "emc_group_step: the same context twice");
    if (n_steps < 0) return fail(a, EMC_EINVAL, "n_steps < 0");
    if (n_steps == 0) return EMC_OK;
    if (a->st != b->st || a->prec != b->prec || a->block != b->block)
        return fail(a, EMC_EINVAL, "emc_group_step: the contexts need one stream, precision and block size");
    if (a->sharded || b->sharded) return fail(a, EMC_EINVAL, "emc_group_step: sharded contexts step alone");
    if (a->geom == EMC_GEOM_NANOWIRE && b->geom == EMC_GEOM_NANOWIRE &&
        (a->K != b->K || a->steps_done % a->K != b->steps_done % b->K))
        return fail(a, EMC_EINVAL, "emc_group_step: nanowire contexts need the same Poisson period and phase");
    if (a->prof || b->prof) return fail(a, EMC_EINVAL, "emc_group_step: flight profiling is per context");
    return a->prec == EMC_FP64 ? pair_step_impl<double>(a, b, n_steps) : pair_step_impl<float>(a, b, n_steps);
}

emc_status emc_shard_counts(emc_ctx* ctx, int32_t* charge_out, int64_t* free_out)
{
    EMC_TRACE("emc_shard_counts");
    if (!ctx || !charge_out || !free_out) return EMC_EINVAL;
    if (!ctx->sharded || !ctx->shard_pending)
        return fail(ctx, EMC_EINVAL, "emc_shard_counts: no exchange pending (or not a sharded context)");
    launch_free_counts<float>(ctx->P, ctx->d_free, ctx->st);
    ctx->launches += 1;
    CK(cudaGetLastError());
    const size_t nc = (size_t)ctx->n_ens * ctx->ncell;
    CK(cudaMemcpyAsync(charge_out, ctx->charge, sizeof(int) * nc, cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(free_out, ctx->d_free, sizeof(long long) * 2 * ctx->n_ens, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return check_err(ctx);
}

emc_status emc_shard_tail(emc_ctx* ctx, const int32_t* charge_global, const int64_t* free_prefix,
                          const int64_t* free_total, int32_t lead)
{
    EMC_TRACE("emc_shard_tail");
    if (!ctx || !charge_global || !free_prefix || !free_total) return EMC_EINVAL;
    if (!ctx->sharded || !ctx->shard_pending)
        return fail(ctx, EMC_EINVAL, "emc_shard_tail: no exchange pending (or not a sharded context)");
    const int E = ctx->n_ens;
    // host copies of the small per-ensemble inputs (they may be device memory)
    std::vector<long long> pre((size_t)2 * E), tot((size_t)2 * E), sh((size_t)5 * E);
    CK(cudaMemcpyAsync(pre.data(), free_prefix, sizeof(long long) * 2 * E, cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(tot.data(), free_total, sizeof(long long) * 2 * E, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int e = 0; e < E; ++e) {
        if (pre[2 * e] < 0 || pre[2 * e + 1] < 0 || tot[2 * e] < pre[2 * e] || tot[2 * e + 1] < pre[2 * e + 1])
            return fail(ctx, EMC_EINVAL, "emc_shard_tail: need 0 <= free_prefix <= free_total");
        sh[5 * e] = pre[2 * e];
        sh[5 * e + 1] = pre[2 * e + 1];
        sh[5 * e + 2] = tot[2 * e];
        sh[5 * e + 3] = tot[2 * e + 1];
        sh[5 * e + 4] = lead ? 1 : 0;
    }
    CK(cudaMemcpyAsync(ctx->d_shard, sh.data(), sizeof(long long) * 5 * E, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->charge, charge_global, sizeof(int) * (size_t)E * ctx->ncell, cudaMemcpyDefault,
                       ctx->st));
    emc_status s = ctx->prec == EMC_FP64 ? shard_tail_impl<double>(ctx) : shard_tail_impl<float>(ctx);
    if (s != EMC_OK) return s;
    CK(cudaStreamSynchronize(ctx->st));
    return check_err(ctx);
}

emc_status emc_set_temperature(emc_ctx* ctx, int32_t ens, const double* T_cells, int32_t n)
{
    EMC_TRACE("emc_set_temperature");
    if (!ctx || !T_cells || ens < 0 || ens >= ctx->n_ens) return EMC_EINVAL;
    if (ctx->geom != EMC_GEOM_NANOWIRE || ctx->n_tab != 1)
        return fail(ctx, EMC_ESTATE, "emc_set_temperature needs a nanowire context whose ensembles share one material/doping");
    if (n != 1 && n != ctx->ncell) return fail(ctx, EMC_EINVAL, "emc_set_temperature: n must be 1 or the subcell count");
    for (int i = 0; i < n; ++i)
        if (!(T_cells[i] > 0.0)) return fail(ctx, EMC_EINVAL, "emc_set_temperature: temperatures must be positive");
    return ctx->prec == EMC_FP64 ? set_temperature_impl<double>(ctx, ens, T_cells, n)
                                 : set_temperature_impl<float>(ctx, ens, T_cells, n);
}

emc_status emc_debug_philox(emc_ctx* ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out, int32_t n)
{
    if (!ctx || n < 0 || (n > 0 && (!ctr || !key || !out))) return EMC_EINVAL;
    if (n == 0) return EMC_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    CK(cudaMallocAsync(&dc, 16ull * n, ctx->st));
    CK(cudaMallocAsync(&dk, 8ull * n, ctx->st));
    CK(cudaMallocAsync(&dout, 16ull * n, ctx->st));
    CK(cudaMemcpyAsync(dc, ctr, 16ull * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(dk, key, 8ull * n, cudaMemcpyHostToDevice, ctx->st));
    k_debug_philox<<<grid_for(n, 128), 128, 0, ctx->st>>>(dc, dk, dout, n);
    ctx->launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dout, 16ull * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaFreeAsync(dc, ctx->st));
    CK(cudaFreeAsync(dk, ctx->st));
    CK(cudaFreeAsync(dout, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return EMC_OK;
}

emc_status emc_debug_particles(emc_ctx* ctx, double* k, double* r, double* tr, int32_t* valley, int32_t* ens,
                               uint32_t* idp, uint64_t* ctrp)
{
    if (!ctx) return EMC_EINVAL;
    const size_t n = (size_t)ctx->n_slots;
    const bool f64 = ctx->prec == EMC_FP64, nw = ctx->geom == EMC_GEOM_NANOWIRE;
    const size_t es = f64 ? 8 : 4;
    std::vector<unsigned char> b[7];
    void* src[7] = {ctx->kx, ctx->ky, ctx->kz, ctx->x, ctx->y, ctx->z, ctx->tr};
    for (int i = 0; i < 7; ++i) {
        b[i].assign(n * es, 0);
        if (src[i] && n) CK(cudaMemcpyAsync(b[i].data(), src[i], n * es, cudaMemcpyDeviceToHost, ctx->st));
    }
    std::vector<uint32_t> tg(n), idv(n);
    std::vector<uint64_t> cv(n);
    if (n) {
        CK(cudaMemcpyAsync(tg.data(), ctx->tag, 4 * n, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(idv.data(), ctx->id, 4 * n, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(cv.data(), ctx->ctr, 8 * n, cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    auto get = [&](int a, size_t i) -> double {
        return f64 ? reinterpret_cast<const double*>(b[a].data())[i] : (double)reinterpret_cast<const float*>(b[a].data())[i];
    };
    for (size_t i = 0; i < n; ++i) {
        if (k)
            for (int a = 0; a < 3; ++a) k[3 * i + a] = get(a, i) * 1e9;
        if (r)
            for (int a = 0; a < 3; ++a) r[3 * i + a] = nw ? get(3 + a, i) * 1e-9 : 0.0;
        if (tr) tr[i] = get(6, i) * 1e-15;
        if (valley) valley[i] = (tg[i] & 0xFFu) == DEAD ? -1 : (int32_t)(tg[i] & 0xFFu);
        if (ens) ens[i] = (int32_t)(tg[i] >> 8);
        if (idp) idp[i] = idv[i];
        if (ctrp) ctrp[i] = cv[i];
    }
    return EMC_OK;
}

emc_status emc_debug_tables(emc_ctx* ctx, int32_t ens, double* table, double* gamma0)
{
    if (!ctx || ens < 0 || ens >= ctx->n_ens) return EMC_EINVAL;
    const int ts = ctx->tabset[ens];
    const size_t per = (size_t)NV * ctx->nb * NM;
    if (table) CK(cudaMemcpyAsync(table, ctx->tab64 + ts * per, 8 * per, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (gamma0)
        for (int v = 0; v < NV; ++v) gamma0[v] = ctx->g0_host[(size_t)ts * NV + v] * 1e15;
    return EMC_OK;
}

emc_status emc_shape(const emc_ctx* ctx, int32_t* n_ens, int64_t* capacity, int32_t* n_cell)
{
    if (!ctx) return EMC_EINVAL;
    if (n_ens) *n_ens = ctx->n_ens;
    if (capacity) *capacity = ctx->n_slots;
    if (n_cell) *n_cell = ctx->ncell;
    return EMC_OK;
}

int64_t emc_launch_count(const emc_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* emc_last_error(const emc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void emc_destroy(emc_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    if (ctx->g_tail_exec) cudaGraphExecDestroy(ctx->g_tail_exec);
    if (ctx->g_tail) cudaGraphDestroy(ctx->g_tail);
    if (ctx->sur) emc_mlp_destroy(ctx->sur);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFree(p);
    delete ctx;
}

}  // extern "C"
