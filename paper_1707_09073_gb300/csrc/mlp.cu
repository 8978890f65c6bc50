// Surrogate MLP of libemc (include/emc.h, emc_mlp_*): local conditions
// (|E|, field angle, T, log10 N_d) -> Monte Carlo observables (drift
// velocity, mean energy, valley fractions, heat rate, current density),
// trained on data the Monte Carlo itself produces.
//
// Every matrix product runs on the tensor cores with BF16 operands and FP32
// accumulation (inline-PTX mma.sync m16n8k16); master weights, gradients and
// Adam moments are FP32.  Matrices are row-major; a layer holds
// W [out_p][in_p] and b [out_p] with dimensions padded to multiples of 16;
// the padding is zero and stays zero (its gradients are zero).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/emc.h"
#include "common.cuh"

namespace {

constexpr int kMaxLayers = 8;

struct Layer {
    int in = 0, out = 0, in_p = 0, out_p = 0;
    float *W = nullptr, *b = nullptr;
    float *gW = nullptr, *gb = nullptr;
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    __nv_bfloat16 *Wb = nullptr, *WTb = nullptr;  // W and W^T in BF16
};

}  // namespace

struct emc_mlp {
    cudaStream_t st = nullptr;
    emc_mlp_config cfg{};
    int n_layers = 0;
    Layer L[kMaxLayers];
    float* norm = nullptr;  // device [4][16]: x_shift, x_scale, y_shift, y_scale
    int64_t cap = 0;        // batch rows allocated (multiple of 16)
    __nv_bfloat16* act[kMaxLayers + 1] = {nullptr};
    float* z[kMaxLayers] = {nullptr};
    float *da = nullptr, *dzf = nullptr;
    __nv_bfloat16 *dzb = nullptr, *dzT = nullptr, *aT = nullptr;
    float *X = nullptr, *Y = nullptr, *loss = nullptr;
    float *Xall = nullptr, *Yall = nullptr;
    int64_t nall = 0;
    int64_t step = 0;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

emc_status mfail(emc_mlp* m, emc_status s, const std::string& msg)
{
    if (m) m->err = msg;
    return s;
}

#define MCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return mfail(m, EMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

template <typename T>
cudaError_t malloc0(emc_mlp* m, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaMemsetAsync(q, 0, std::max<size_t>(n, 1) * sizeof(T), m->st);
}

void mfree(emc_mlp* m, void* p)
{
    if (!p) return;
    auto it = std::find(m->allocs.begin(), m->allocs.end(), p);
    if (it != m->allocs.end()) m->allocs.erase(it);
    cudaFree(p);
}

int pad16(int x) { return (x + 15) / 16 * 16; }
unsigned gridn(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------- tensor core
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ float silu(float x) { return x / (1.f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x)
{
    const float s = 1.f / (1.f + __expf(-x));
    return s * (1.f + x * (1.f - s));
}

enum { EPI_BIAS = 1, EPI_SILU = 2, EPI_ACC = 4 };

// C[M][N] = A[M][K] . B[N][K]^T with bf16 row-major operands and fp32
// accumulation.  One warp owns a 16-row x 32-column tile (four m16n8k16
// tiles) and walks K in steps of 16; fragments are read straight from
// global memory (the matrices here are small).  M % 16 == 0, N % 8 == 0,
// K % 16 == 0.  Epilogue: + bias[n] (EPI_BIAS); z (fp32) receives the sum
// (or adds it, EPI_ACC); out (bf16) receives SiLU(sum) (EPI_SILU) or sum.
__global__ void k_gemm(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B, int M, int N, int K,
                       const float* __restrict__ bias, int epi, float* z, int ldz, __nv_bfloat16* out, int ldo)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int tiles_n = (N + 31) / 32;
    const int tm = warp / tiles_n, tn = warp % tiles_n;
    if (tm * 16 >= M) return;
    const int g = lane >> 2, t = lane & 3;
    const int r0 = tm * 16, n0 = tn * 32;
    float c[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        a[0] = ld2(A + (size_t)(r0 + g) * K + k0 + 2 * t);
        a[1] = ld2(A + (size_t)(r0 + g + 8) * K + k0 + 2 * t);
        a[2] = ld2(A + (size_t)(r0 + g) * K + k0 + 8 + 2 * t);
        a[3] = ld2(A + (size_t)(r0 + g + 8) * K + k0 + 8 + 2 * t);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + 8 * j;
            if (nn < N) {
                uint32_t b[2];
                b[0] = ld2(B + (size_t)(nn + g) * K + k0 + 2 * t);
                b[1] = ld2(B + (size_t)(nn + g) * K + k0 + 8 + 2 * t);
                mma_bf16(c[j], a, b);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int nn = n0 + 8 * j;
        if (nn >= N) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = r0 + g + 8 * h;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int col = nn + 2 * t + q;
                float v = c[j][2 * h + q];
                if (epi & EPI_BIAS) v += bias[col];
                if (z) {
                    float* zz = z + (size_t)row * ldz + col;
                    *zz = (epi & EPI_ACC) ? *zz + v : v;
                }
                if (out) out[(size_t)row * ldo + col] = __float2bfloat16_rn((epi & EPI_SILU) ? silu(v) : v);
            }
        }
    }
}

void gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, const float* bias, int epi, float* z,
          int ldz, __nv_bfloat16* out, int ldo, cudaStream_t st)
{
    const int64_t warps = (int64_t)(M / 16) * ((N + 31) / 32);
    k_gemm<<<gridn(warps * 32, 128), 128, 0, st>>>(A, B, M, N, K, bias, epi, z, ldz, out, ldo);
}

// ---------------------------------------------------------- elementwise
__global__ void k_input(const float* X, int64_t n, int n_in, int in_p, const float* norm, __nv_bfloat16* out,
                        int64_t rows)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * in_p) return;
    const int64_t r = i / in_p;
    const int c = int(i % in_p);
    float v = 0.f;
    if (r < n && c < n_in) v = (X[r * n_in + c] - norm[c]) / norm[16 + c];
    out[i] = __float2bfloat16_rn(v);
}

__global__ void k_output(const float* z, int ldz, int64_t n, int n_out, const float* norm, float* Y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n_out) return;
    const int64_t r = i / n_out;
    const int c = int(i % n_out);
    Y[i] = z[r * ldz + c] * norm[48 + c] + norm[32 + c];
}

// mean squared error of the normalised outputs, gradient w.r.t. z
__global__ void k_mse(const float* z, int ldz, const float* Y, int64_t n, int n_out, const float* norm, float* dz,
                      int64_t rows, float* loss)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ldz) return;
    const int64_t r = i / ldz;
    const int c = int(i % ldz);
    float g = 0.f;
    if (r < n && c < n_out) {
        const float d = z[i] - (Y[r * n_out + c] - norm[32 + c]) / norm[48 + c];
        const float inv = 1.f / float(n * n_out);
        g = 2.f * d * inv;
        atomicAdd(loss, d * d * inv);
    }
    dz[i] = g;
}

__global__ void k_transpose_f2b(const float* src, int rows, int cols, __nv_bfloat16* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = int(i / cols), c = int(i % cols);
    dst[(size_t)c * rows + r] = __float2bfloat16_rn(src[i]);
}
__global__ void k_transpose_b2b(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = int(i / cols), c = int(i % cols);
    dst[(size_t)c * rows + r] = src[i];
}
__global__ void k_f2b(const float* src, int64_t n, __nv_bfloat16* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// g[c] = sum over rows of dz[r][c]
__global__ void k_colsum(const float* dz, int64_t rows, int cols, float* g)
{
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += dz[r * cols + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[c] = red[0];
}

// dz = da * silu'(z) on the valid columns (padding stays 0)
__global__ void k_dsilu(const float* da, const float* z, int64_t n_elem, int cols, int valid, float* dz)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_elem) return;
    const int c = int(i % cols);
    dz[i] = c < valid ? da[i] * dsilu(z[i]) : 0.f;
}

// Adam with bias correction (Kingma & Ba, ICLR 2015)
__global__ void k_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// minibatch rows drawn with replacement from the dataset by a Philox stream
__global__ void k_gather(const float* Xall, const float* Yall, int64_t nall, int n_in, int n_out, uint32_t seed,
                         uint64_t step, int batch, float* X, float* Y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= batch) return;
    const emc::U4 r = emc::philox10(emc::U4{uint32_t(step), uint32_t(step >> 32), uint32_t(i), 0x5EEDu}, seed, 0x3779u);
    const int64_t src = (int64_t)(((uint64_t)r.a << 32 | r.b) % (uint64_t)nall);
    for (int c = 0; c < n_in; ++c) X[(int64_t)i * n_in + c] = Xall[src * n_in + c];
    for (int c = 0; c < n_out; ++c) Y[(int64_t)i * n_out + c] = Yall[src * n_out + c];
}

// ------------------------------------------------------------- passes
emc_status refresh_bf16(emc_mlp* m)
{
    for (int l = 0; l < m->n_layers; ++l) {
        Layer& y = m->L[l];
        const int64_t nw = (int64_t)y.out_p * y.in_p;
        k_f2b<<<gridn(nw, 256), 256, 0, m->st>>>(y.W, nw, y.Wb);
        k_transpose_f2b<<<gridn(nw, 256), 256, 0, m->st>>>(y.W, y.out_p, y.in_p, y.WTb);
    }
    MCK(cudaGetLastError());
    return EMC_OK;
}

emc_status ensure_batch(emc_mlp* m, int64_t n)
{
    const int64_t rows = (n + 15) / 16 * 16;
    if (rows <= m->cap) return EMC_OK;
    for (int l = 0; l <= m->n_layers; ++l) mfree(m, m->act[l]);
    for (int l = 0; l < m->n_layers; ++l) mfree(m, m->z[l]);
    mfree(m, m->da); mfree(m, m->dzf); mfree(m, m->dzb); mfree(m, m->dzT); mfree(m, m->aT);
    mfree(m, m->X); mfree(m, m->Y);
    int maxp = 16;
    for (int l = 0; l < m->n_layers; ++l) maxp = std::max(maxp, std::max(m->L[l].out_p, m->L[l].in_p));
    for (int l = 0; l <= m->n_layers; ++l)
        MCK(malloc0(m, &m->act[l], (size_t)rows * (l < m->n_layers ? m->L[l].in_p : m->L[l - 1].out_p)));
    for (int l = 0; l < m->n_layers; ++l) MCK(malloc0(m, &m->z[l], (size_t)rows * m->L[l].out_p));
    MCK(malloc0(m, &m->da, (size_t)rows * maxp));
    MCK(malloc0(m, &m->dzf, (size_t)rows * maxp));
    MCK(malloc0(m, &m->dzb, (size_t)rows * maxp));
    MCK(malloc0(m, &m->dzT, (size_t)rows * maxp));
    MCK(malloc0(m, &m->aT, (size_t)rows * maxp));
    MCK(malloc0(m, &m->X, (size_t)rows * m->cfg.n_in));
    MCK(malloc0(m, &m->Y, (size_t)rows * m->cfg.n_out));
    m->cap = rows;
    return EMC_OK;
}

// forward on the n rows in m->X; pre-activations and layer inputs kept
void forward(emc_mlp* m, int64_t n)
{
    const int64_t rows = (n + 15) / 16 * 16;
    k_input<<<gridn(rows * m->L[0].in_p, 256), 256, 0, m->st>>>(m->X, n, m->cfg.n_in, m->L[0].in_p, m->norm, m->act[0],
                                                                rows);
    for (int l = 0; l < m->n_layers; ++l) {
        const Layer& y = m->L[l];
        const bool last = l == m->n_layers - 1;
        gemm(m->act[l], y.Wb, (int)rows, y.out_p, y.in_p, y.b, EPI_BIAS | (last ? 0 : EPI_SILU), m->z[l], y.out_p,
             m->act[l + 1], y.out_p, m->st);
    }
}

// loss and parameter gradients for the rows in m->X / m->Y after forward()
void backward(emc_mlp* m, int64_t n)
{
    const int64_t rows = (n + 15) / 16 * 16;
    const int last = m->n_layers - 1;
    cudaMemsetAsync(m->loss, 0, sizeof(float), m->st);
    k_mse<<<gridn(rows * m->L[last].out_p, 256), 256, 0, m->st>>>(m->z[last], m->L[last].out_p, m->Y, n,
                                                                  m->cfg.n_out, m->norm, m->dzf, rows, m->loss);
    for (int l = last; l >= 0; --l) {
        const Layer& y = m->L[l];
        const int64_t nz = rows * y.out_p;
        // dW = dz^T a  (A operand dz^T [out_p][rows], B operand a^T [in_p][rows])
        k_transpose_f2b<<<gridn(nz, 256), 256, 0, m->st>>>(m->dzf, (int)rows, y.out_p, m->dzT);
        k_transpose_b2b<<<gridn(rows * y.in_p, 256), 256, 0, m->st>>>(m->act[l], (int)rows, y.in_p, m->aT);
        gemm(m->dzT, m->aT, y.out_p, y.in_p, (int)rows, nullptr, 0, y.gW, y.in_p, nullptr, 0, m->st);
        k_colsum<<<y.out_p, 256, 0, m->st>>>(m->dzf, rows, y.out_p, y.gb);
        if (l == 0) break;
        // da = dz W  (A operand dz [rows][out_p], B operand W^T [in_p][out_p])
        k_f2b<<<gridn(nz, 256), 256, 0, m->st>>>(m->dzf, nz, m->dzb);
        gemm(m->dzb, y.WTb, (int)rows, y.in_p, y.out_p, nullptr, 0, m->da, y.in_p, nullptr, 0, m->st);
        const Layer& p = m->L[l - 1];
        k_dsilu<<<gridn(rows * p.out_p, 256), 256, 0, m->st>>>(m->da, m->z[l - 1], rows * p.out_p, p.out_p, p.out,
                                                               m->dzf);
    }
}

// copy between the packed parameter vector (valid entries) and the padded
// layer arrays; dir 0: device layers -> vec, 1: vec -> device layers
emc_status pack(emc_mlp* m, std::vector<float>& vec, int dir, bool grads)
{
    size_t off = 0;
    for (int l = 0; l < m->n_layers; ++l) {
        const Layer& y = m->L[l];
        std::vector<float> W((size_t)y.out_p * y.in_p), b(y.out_p);
        float* dW = grads ? y.gW : y.W;
        float* db = grads ? y.gb : y.b;
        MCK(cudaMemcpyAsync(W.data(), dW, 4 * W.size(), cudaMemcpyDeviceToHost, m->st));
        MCK(cudaMemcpyAsync(b.data(), db, 4 * b.size(), cudaMemcpyDeviceToHost, m->st));
        MCK(cudaStreamSynchronize(m->st));
        for (int o = 0; o < y.out; ++o)
            for (int i = 0; i < y.in; ++i) {
                float& x = W[(size_t)o * y.in_p + i];
                if (dir == 0) vec[off + (size_t)o * y.in + i] = x;
                else x = vec[off + (size_t)o * y.in + i];
            }
        off += (size_t)y.out * y.in;
        for (int o = 0; o < y.out; ++o) {
            if (dir == 0) vec[off + o] = b[o];
            else b[o] = vec[off + o];
        }
        off += y.out;
        if (dir == 1) {
            MCK(cudaMemcpyAsync(dW, W.data(), 4 * W.size(), cudaMemcpyHostToDevice, m->st));
            MCK(cudaMemcpyAsync(db, b.data(), 4 * b.size(), cudaMemcpyHostToDevice, m->st));
            MCK(cudaStreamSynchronize(m->st));
        }
    }
    return EMC_OK;
}

int64_t n_params(const emc_mlp* m)
{
    int64_t n = 0;
    for (int l = 0; l < m->n_layers; ++l) n += (int64_t)m->L[l].out * m->L[l].in + m->L[l].out;
    return n;
}

}  // namespace

extern "C" {

emc_status emc_mlp_create(const emc_mlp_config* cfg, void* stream, emc_mlp** out)
{
    if (!cfg || !out) return EMC_EINVAL;
    *out = nullptr;
    emc_mlp* m = new (std::nothrow) emc_mlp();
    if (!m) return EMC_ENOMEM;
    *out = m;
    const emc_mlp_config& c = *cfg;
    if (c.n_in < 1 || c.n_in > 16 || c.n_out < 1 || c.n_out > 16 || c.n_hidden < 16 || c.n_hidden > 256 ||
        c.n_hidden % 16 || c.n_layers < 1 || c.n_layers > 6)
        return mfail(m, EMC_EINVAL, "mlp: n_in, n_out in 1..16; n_hidden multiple of 16 in 16..256; 1..6 layers");
    for (int i = 0; i < 16; ++i)
        if ((i < c.n_in && !(c.x_scale[i] != 0.f)) || (i < c.n_out && !(c.y_scale[i] != 0.f)))
            return mfail(m, EMC_EINVAL, "mlp: zero normalisation scale");
    m->st = static_cast<cudaStream_t>(stream);
    m->cfg = c;
    m->n_layers = c.n_layers + 1;
    std::mt19937_64 rng(c.seed);
    for (int l = 0; l < m->n_layers; ++l) {
        Layer& y = m->L[l];
        y.in = l == 0 ? c.n_in : c.n_hidden;
        y.out = l == m->n_layers - 1 ? c.n_out : c.n_hidden;
        y.in_p = pad16(y.in);
        y.out_p = pad16(y.out);
        const size_t nw = (size_t)y.out_p * y.in_p;
        MCK(malloc0(m, &y.W, nw)); MCK(malloc0(m, &y.b, y.out_p));
        MCK(malloc0(m, &y.gW, nw)); MCK(malloc0(m, &y.gb, y.out_p));
        MCK(malloc0(m, &y.mW, nw)); MCK(malloc0(m, &y.vW, nw));
        MCK(malloc0(m, &y.mb, y.out_p)); MCK(malloc0(m, &y.vb, y.out_p));
        MCK(malloc0(m, &y.Wb, nw)); MCK(malloc0(m, &y.WTb, nw));
        std::vector<float> W(nw, 0.f);
        const double lim = std::sqrt(6.0 / y.in);
        std::uniform_real_distribution<double> U(-lim, lim);
        for (int o = 0; o < y.out; ++o)
            for (int i = 0; i < y.in; ++i) W[(size_t)o * y.in_p + i] = (float)U(rng);
        MCK(cudaMemcpyAsync(y.W, W.data(), 4 * nw, cudaMemcpyHostToDevice, m->st));
        MCK(cudaStreamSynchronize(m->st));
    }
    MCK(malloc0(m, &m->norm, 64));
    float nh[64];
    std::memcpy(nh, c.x_shift, 64);
    std::memcpy(nh + 16, c.x_scale, 64);
    std::memcpy(nh + 32, c.y_shift, 64);
    std::memcpy(nh + 48, c.y_scale, 64);
    MCK(cudaMemcpyAsync(m->norm, nh, sizeof nh, cudaMemcpyHostToDevice, m->st));
    MCK(malloc0(m, &m->loss, 1));
    emc_status s = refresh_bf16(m);
    if (s != EMC_OK) return s;
    MCK(cudaStreamSynchronize(m->st));
    return EMC_OK;
}

emc_status emc_mlp_infer(emc_mlp* m, const float* X, float* Y, int64_t n)
{
    if (!m || (n > 0 && (!X || !Y)) || n < 0) return EMC_EINVAL;
    if (n == 0) return EMC_OK;
    const int64_t chunk = 1 << 16;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t nn = std::min(chunk, n - r0);
        emc_status s = ensure_batch(m, nn);
        if (s != EMC_OK) return s;
        MCK(cudaMemcpyAsync(m->X, X + r0 * m->cfg.n_in, 4 * nn * m->cfg.n_in, cudaMemcpyHostToDevice, m->st));
        forward(m, nn);
        const int last = m->n_layers - 1;
        k_output<<<gridn(nn * m->cfg.n_out, 256), 256, 0, m->st>>>(m->z[last], m->L[last].out_p, nn, m->cfg.n_out,
                                                                   m->norm, m->Y);
        MCK(cudaGetLastError());
        MCK(cudaMemcpyAsync(Y + r0 * m->cfg.n_out, m->Y, 4 * nn * m->cfg.n_out, cudaMemcpyDeviceToHost, m->st));
    }
    MCK(cudaStreamSynchronize(m->st));
    return EMC_OK;
}

emc_status emc_mlp_grad(emc_mlp* m, const float* X, const float* Y, int64_t n, float* grad, float* loss)
{
    if (!m || !X || !Y || n <= 0) return EMC_EINVAL;
    emc_status s = ensure_batch(m, n);
    if (s != EMC_OK) return s;
    MCK(cudaMemcpyAsync(m->X, X, 4 * n * m->cfg.n_in, cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->Y, Y, 4 * n * m->cfg.n_out, cudaMemcpyHostToDevice, m->st));
    forward(m, n);
    backward(m, n);
    MCK(cudaGetLastError());
    if (loss) MCK(cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    if (grad) {
        std::vector<float> v(n_params(m));
        s = pack(m, v, 0, true);
        if (s != EMC_OK) return s;
        std::memcpy(grad, v.data(), 4 * v.size());
    }
    return EMC_OK;
}

emc_status emc_mlp_train(emc_mlp* m, const float* X, const float* Y, int64_t n, const emc_train_config* tc,
                         float* loss_history)
{
    if (!m || !X || !Y || n <= 0 || !tc || tc->steps < 0 || tc->batch <= 0) return EMC_EINVAL;
    emc_status s = ensure_batch(m, tc->batch);
    if (s != EMC_OK) return s;
    if (m->nall < n) {
        mfree(m, m->Xall);
        mfree(m, m->Yall);
        MCK(malloc0(m, &m->Xall, (size_t)n * m->cfg.n_in));
        MCK(malloc0(m, &m->Yall, (size_t)n * m->cfg.n_out));
    }
    m->nall = n;
    MCK(cudaMemcpyAsync(m->Xall, X, 4 * n * m->cfg.n_in, cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->Yall, Y, 4 * n * m->cfg.n_out, cudaMemcpyHostToDevice, m->st));
    float* d_hist = nullptr;
    if (loss_history) MCK(cudaMallocAsync(&d_hist, 4 * std::max<int64_t>(tc->steps, 1), m->st));
    for (int64_t it = 0; it < tc->steps; ++it) {
        k_gather<<<gridn(tc->batch, 256), 256, 0, m->st>>>(m->Xall, m->Yall, n, m->cfg.n_in, m->cfg.n_out, tc->seed,
                                                           (uint64_t)(m->step), tc->batch, m->X, m->Y);
        forward(m, tc->batch);
        backward(m, tc->batch);
        ++m->step;
        const float c1 = 1.f - std::pow(tc->beta1, (float)m->step), c2 = 1.f - std::pow(tc->beta2, (float)m->step);
        for (int l = 0; l < m->n_layers; ++l) {
            Layer& y = m->L[l];
            const int64_t nw = (int64_t)y.out_p * y.in_p;
            k_adam<<<gridn(nw, 256), 256, 0, m->st>>>(y.W, y.gW, y.mW, y.vW, nw, tc->lr, tc->beta1, tc->beta2, tc->eps,
                                                      c1, c2);
            k_adam<<<gridn(y.out_p, 256), 256, 0, m->st>>>(y.b, y.gb, y.mb, y.vb, y.out_p, tc->lr, tc->beta1,
                                                           tc->beta2, tc->eps, c1, c2);
        }
        s = refresh_bf16(m);
        if (s != EMC_OK) return s;
        if (d_hist) MCK(cudaMemcpyAsync(d_hist + it, m->loss, 4, cudaMemcpyDeviceToDevice, m->st));
    }
    MCK(cudaGetLastError());
    if (d_hist) {
        MCK(cudaMemcpyAsync(loss_history, d_hist, 4 * tc->steps, cudaMemcpyDeviceToHost, m->st));
        MCK(cudaFreeAsync(d_hist, m->st));
    }
    MCK(cudaStreamSynchronize(m->st));
    return EMC_OK;
}

emc_status emc_mlp_params(emc_mlp* m, float* dst, const float* src, int64_t* count)
{
    if (!m) return EMC_EINVAL;
    const int64_t np = n_params(m);
    if (count) *count = np;
    std::vector<float> v(np);
    if (dst) {
        emc_status s = pack(m, v, 0, false);
        if (s != EMC_OK) return s;
        std::memcpy(dst, v.data(), 4 * np);
    }
    if (src) {
        std::memcpy(v.data(), src, 4 * np);
        emc_status s = pack(m, v, 1, false);
        if (s != EMC_OK) return s;
        s = refresh_bf16(m);
        if (s != EMC_OK) return s;
        MCK(cudaStreamSynchronize(m->st));
    }
    return EMC_OK;
}

const char* emc_mlp_last_error(const emc_mlp* m) { return m ? m->err.c_str() : "null mlp"; }

void emc_mlp_destroy(emc_mlp* m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}

}  // extern "C"
