// Surrogate MLP of libemc (include/emc.h, emc_mlp_*): local conditions
// (|E|, field angle, T, log10 N_d) -> Monte Carlo observables (drift
// velocity, mean energy, valley fractions, heat rate, current density),
// trained on data the Monte Carlo itself produces.
//
// Every matrix product runs on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands staged in shared memory, FP32 accumulator in tensor memory);
// master weights, gradients and Adam moments are FP32.  Matrices are row-major; a layer holds
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
#include "trace.h"
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
    int* d_err = nullptr;  // set by a tensor-core wait that expired
    float *Xall = nullptr, *Yall = nullptr;
    int64_t nall = 0;
    bool fused = true;                     // inference in one fused launch when the network fits
    float *fX = nullptr, *fY = nullptr;    // its input and output rows
    int64_t fcap = 0;
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
// x sigmoid(x) with the hardware exponential and the approximate division
// (for x below about -88 the denominator is infinite and the result 0)
__device__ __forceinline__ float silu(float x) { return __fdividef(x, 1.f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x)
{
    const float s = 1.f / (1.f + __expf(-x));
    return s * (1.f + x * (1.f - s));
}

enum { EPI_BIAS = 1, EPI_SILU = 2, EPI_ACC = 4 };

// 5th-generation tensor cores (tcgen05): one CTA of four warps computes a
// 128-row x BN-column tile of C = A . B^T (A [M][K], B [N][K], both BF16
// row-major, i.e. K-major operands) over a range of K, with the FP32
// accumulator in tensor memory.  K is walked in blocks of 64 through two
// shared-memory stages: the warps stage block i + 1 (canonical K-major
// layout without swizzle: 8-row x 16-byte core matrices, 128 B apart along
// K, 8-row groups 1024 B apart) while the tensor core works on block i; one
// thread issues the 128 x BN x 16 MMAs and commits each block to the
// mbarrier of its stage, which the warps wait on before refilling it.  The
// epilogue reads the accumulator with tcgen05.ld (warp w owns rows 32w ..
// 32w + 31), adds the bias, applies SiLU and writes FP32 and/or BF16; with
// K split over several CTAs (gridDim.z > 1) the partial sums are added
// atomically into z, which the caller has zeroed.  Every wait is bounded:
// on expiry the error word is set, the MMAs in flight are waited for
// (bounded again), tensor memory is freed and the CTA exits.
constexpr int kTcBM = 128, kTcBK = 64;
constexpr size_t kTcStageA = (size_t)kTcBM * kTcBK * 2;
constexpr long long kTcWaitCycles = 2000000000ll;  // ~1 s at the GB300 clock

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

// stage the K block [k0, k0 + kb) of rows [r0, r0 + rows) of X (row length
// K) in the core-matrix layout with 16-byte asynchronous copies (all in
// flight at once; the caller commits and waits); rows at or beyond rmax are
// zero-filled by the copy itself (source size 0)
__device__ __forceinline__ void tc_stage(unsigned char* dst, const __nv_bfloat16* __restrict__ X, int r0, int rows,
                                         int rmax, int K, int k0, int kb)
{
    const int nch = kb >> 3;
    for (int i = threadIdx.x; i < rows * nch; i += blockDim.x) {
        const int r = i / nch, c = i - (i / nch) * nch;
        const bool in = r0 + r < rmax;
        const __nv_bfloat16* src = X + (size_t)(in ? r0 + r : 0) * K + k0 + 8 * c;
        const uint32_t d = smem_u32(dst + (r >> 3) * 1024 + c * 128 + (r & 7) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
}

__global__ void __launch_bounds__(128) k_gemm_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                                                 int M, int N, int K, int BN, int k_per_cta,
                                                 const float* __restrict__ bias, int epi, float* z, int ldz,
                                                 __nv_bfloat16* out, int ldo, int* err)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_slot;
    const size_t stage = kTcStageA + (size_t)BN * kTcBK * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * k_per_cta, kend = min(K, kbeg + k_per_cta);
    const bool split = gridDim.z > 1;
    const uint32_t ncols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    const uint32_t bar0 = smem_u32(&bars[0]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc(kTcBM, BN);
    uint32_t phase[2] = {0u, 0u};
    int pending[2] = {0, 0};  // commits of a stage not yet waited for
    bool ok = true;
    int it = 0;
    const int nblk = (kend - kbeg + kTcBK - 1) / kTcBK;
    // block 0 in flight before the loop; block i + 1 is copied while the
    // tensor core works on block i
    if (nblk > 0) {
        const int kb = min(kTcBK, kend - kbeg);
        tc_stage(tc_smem, A, m0, kTcBM, M, K, kbeg, kb);
        tc_stage(tc_smem + kTcStageA, B, n0, BN, N, K, kbeg, kb);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (; it < nblk && ok; ++it) {
        const int sidx = it & 1;
        const int k0 = kbeg + it * kTcBK;
        const int kb = min(kTcBK, kend - k0);
        if (it + 1 < nblk) {
            const int nx = sidx ^ 1;
            if (pending[nx]) {
                // the MMAs that read the next stage (block it - 1) must be
                // done before it is refilled (on expiry the commit stays
                // pending and the drain below waits again)
                ok = __syncthreads_and(mbar_wait(bar0 + 8u * nx, phase[nx])) != 0;
                if (!ok) break;
                phase[nx] ^= 1u;
                pending[nx] = 0;
            }
            const int k1 = k0 + kTcBK;
            const int kb1 = min(kTcBK, kend - k1);
            unsigned char* nA = tc_smem + nx * stage;
            tc_stage(nA, A, m0, kTcBM, M, K, k1, kb1);
            tc_stage(nA + kTcStageA, B, n0, BN, N, K, k1, kb1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        unsigned char* sA = tc_smem + sidx * stage;
        unsigned char* sB = sA + kTcStageA;
        // the copies must be visible to the tensor core's (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int s = 0; s < (kb >> 4); ++s) {
                const uint64_t da = tc_sdesc(smem_u32(sA) + 256u * s, 128u, 1024u);
                const uint64_t db = tc_sdesc(smem_u32(sB) + 256u * s, 128u, 1024u);
                const uint32_t acc = (it > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar0 + 8u * sidx)
                         : "memory");
        }
        pending[sidx] = 1;
    }
    // no copy may still be landing in shared memory when the CTA moves on
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // drain: every outstanding commit (the MMAs complete in issue order)
    for (int q = 0; q < 2; ++q) {
        const int sidx = (it + q) & 1;  // oldest first
        if (pending[sidx]) {
            const bool w = __syncthreads_and(mbar_wait(bar0 + 8u * sidx, phase[sidx])) != 0;
            ok = ok && w;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else if (kend > kbeg) {
        // the stages are free now: each warp transposes its 32 rows x 16
        // columns through 2 KB of them, then writes 64-byte row segments
        float* tb = reinterpret_cast<float*>(tc_smem) + warp * (32 * 17);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) tb[lane * 17 + j] = __uint_as_float(r[j]);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = q * 8 + (lane >> 2), cc = (lane & 3) * 4;
                const int row = m0 + warp * 32 + rr, col = n0 + c0 + cc;
                if (row < M && col < N) {
                    float v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = tb[rr * 17 + cc + i];
                    if (split) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) atomicAdd(z + (size_t)row * ldz + col + i, v[i]);
                    } else {
                        if (epi & EPI_BIAS) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) v[i] += bias[col + i];
                        }
                        if (z) {
                            float4* zz = reinterpret_cast<float4*>(z + (size_t)row * ldz + col);
                            if (epi & EPI_ACC) {
                                const float4 o = *zz;
                                *zz = make_float4(o.x + v[0], o.y + v[1], o.z + v[2], o.w + v[3]);
                            } else {
                                *zz = make_float4(v[0], v[1], v[2], v[3]);
                            }
                        }
                        if (out) {
                            if (epi & EPI_SILU) {
#pragma unroll
                                for (int i = 0; i < 4; ++i) v[i] = silu(v[i]);
                            }
                            const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
                            const __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
                            uint2 pk;
                            pk.x = *reinterpret_cast<const uint32_t*>(&h0);
                            pk.y = *reinterpret_cast<const uint32_t*>(&h1);
                            *reinterpret_cast<uint2*>(out + (size_t)row * ldo + col) = pk;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

constexpr size_t kTcMaxSmem = 2 * (kTcStageA + (size_t)256 * kTcBK * 2);

// ------------------------------------------------------------ fused
// Inference of the whole network in one launch: a persistent CTA of
// 4 x kFzGroups warps stages every layer's BF16 weights once in shared memory (the
// canonical K-major layout without swizzle of k_gemm_tc, here over a
// layer's whole K: 8-row groups K * 16 bytes apart), then walks 128-row
// tiles of the input.  Per tile and layer: the activations sit in shared
// memory, one thread issues the K/16 MMAs into the tensor-memory
// accumulator and commits them to an mbarrier; after the wait warp w reads
// rows 32 (w % 4) .. + 31 (the tensor-memory lanes its quarter may access)
// of every kFzGroups-th 16-column chunk, from chunk w / 4 on, back
// (tcgen05.ld), adds the bias, applies SiLU (hidden layers) and writes the
// next layer's BF16 activations over the ones the finished MMAs read; the
// last layer's outputs are de-normalised into Y.
// Only the inputs are read and the outputs written.  The arithmetic is the
// layer-by-layer path's (same normalisation, the same MMAs in the same
// order, bias and SiLU in FP32, BF16 rounding of the activations).
struct FusedNet {
    const __nv_bfloat16* W[kMaxLayers];  // [out_p][in_p], BF16
    const float* b[kMaxLayers];          // [out_p]
    uint32_t w_off[kMaxLayers];          // byte offset of layer l's weights in shared memory
    int in_p[kMaxLayers], out_p[kMaxLayers];
    int n_layers, n_in, n_out;
    uint32_t a_off;                      // byte offset of the activation tile
    uint32_t ncols;                      // tensor-memory columns (power of two >= every out_p, >= 32)
};

__device__ __forceinline__ uint4 pack_bf16x8(const float* v)
{
    uint4 pk;
    uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return pk;
}

constexpr int kFzGroups = 4;  // column groups: 128 x kFzGroups threads per CTA

__global__ void __launch_bounds__(128 * kFzGroups) k_mlp_fused(const FusedNet N, const float* __restrict__ X, int64_t n,
                                                   const float* __restrict__ norm, float* __restrict__ Y, int* err)
{
    extern __shared__ __align__(1024) unsigned char fz_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int rt = tid & 127, grp = tid >> 7;  // row within the tile, column group
    const uint32_t bar0 = smem_u32(&bar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(N.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // every layer's weights, 16-byte chunks into the core-matrix layout
    for (int l = 0; l < N.n_layers; ++l) {
        const int K = N.in_p[l], nch = K >> 3, total = N.out_p[l] * nch;
        unsigned char* dst = fz_smem + N.w_off[l];
        const uint4* src = reinterpret_cast<const uint4*>(N.W[l]);
        for (int i = tid; i < total; i += blockDim.x) {
            const int r = i / nch, c = i - r * nch;
            *reinterpret_cast<uint4*>(dst + (r >> 3) * (K * 16) + c * 128 + (r & 7) * 16) = src[i];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    unsigned char* act = fz_smem + N.a_off;
    uint32_t phase = 0u;
    bool ok = true;
    const int64_t tiles = (n + 127) / 128;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int64_t row = t * 128 + rt;  // this thread's row = its tensor-memory lane
        if (grp == 0) {
            // the row's inputs, normalised, as BF16 (K = in_p of layer 0)
            const int K = N.in_p[0];
            for (int c0 = 0; c0 < K; c0 += 8) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + j;
                    v[j] = (row < n && c < N.n_in) ? (X[row * N.n_in + c] - norm[c]) / norm[16 + c] : 0.f;
                }
                *reinterpret_cast<uint4*>(act + (rt >> 3) * (K * 16) + (c0 >> 3) * 128 + (rt & 7) * 16) =
                    pack_bf16x8(v);
            }
        }
        for (int l = 0; l < N.n_layers; ++l) {
            const int K = N.in_p[l], Nn = N.out_p[l];
            const bool last = l == N.n_layers - 1;
            // the activations written by the threads must be visible to the
            // tensor core's (async proxy) reads, and every warp done reading
            // the accumulator of the previous layer
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t idesc = tc_idesc(128, Nn);
                const uint32_t a0 = smem_u32(act), b0 = smem_u32(fz_smem + N.w_off[l]);
                const uint32_t sbo = (uint32_t)K * 16u;
                for (int s = 0; s < (K >> 4); ++s) {
                    const uint64_t da = tc_sdesc(a0 + 256u * s, 128u, sbo);
                    const uint64_t db = tc_sdesc(b0 + 256u * s, 128u, sbo);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar0)
                             : "memory");
            }
            ok = __syncthreads_and(mbar_wait(bar0, phase)) != 0;
            if (!ok) break;  // block-uniform
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const float* bias = N.b[l];
            for (int c0 = 16 * grp; c0 < Nn; c0 += 16 * kFzGroups) {
                uint32_t r[16];
                const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(ta)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) + bias[c0 + j];
                if (!last) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = silu(v[j]);
                    // the next layer's K is this layer's out_p
                    unsigned char* d = act + (rt >> 3) * (Nn * 16) + (c0 >> 3) * 128 + (rt & 7) * 16;
                    *reinterpret_cast<uint4*>(d) = pack_bf16x8(v);
                    *reinterpret_cast<uint4*>(d + 128) = pack_bf16x8(v + 8);
                } else if (row < n) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = c0 + j;
                        if (c < N.n_out) Y[row * N.n_out + c] = v[j] * norm[48 + c] + norm[32 + c];
                    }
                }
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // the MMAs of the expired wait may still be running: wait again
        // (bounded) before the tensor memory is given back
        (void)__syncthreads_and(mbar_wait(bar0, phase));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(N.ncols) : "memory");
    }
}

// shared memory above which the fused kernel is not used (one CTA per SM)
constexpr size_t kFusedMaxSmem = 200 * 1024;

// C[M][N] = A[M][K] . B[N][K]^T; M % 16 == 0, 16 <= N <= 256 with N % 16 == 0,
// K % 16 == 0.  Tiles of 128 rows x BN columns; narrower column tiles and a
// split of K (partial sums added atomically into z) when there are too few
// tiles to occupy the GPU.
void gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, const float* bias, int epi, float* z,
          int ldz, __nv_bfloat16* out, int ldo, int* err, cudaStream_t st)
{
    const int mt = (M + kTcBM - 1) / kTcBM;
    int BN = N;
    while (BN > 32 && (int64_t)mt * (N / BN) < 128 && (BN / 2) % 16 == 0 && N % (BN / 2) == 0) BN /= 2;
    int splits = 1;
    const bool can_split = out == nullptr && epi == 0 && z != nullptr;
    if (can_split) {
        while ((int64_t)mt * (N / BN) * splits < 128 && K / (splits * 2) >= 2 * kTcBK) splits *= 2;
    }
    const int kpc = splits > 1 ? ((K / splits + kTcBK - 1) / kTcBK) * kTcBK : K;
    if (splits > 1) cudaMemsetAsync(z, 0, sizeof(float) * (size_t)M * ldz, st);
    const size_t smem = 2 * (kTcStageA + (size_t)BN * kTcBK * 2);
    dim3 grid((unsigned)mt, (unsigned)(N / BN), (unsigned)((K + kpc - 1) / kpc));
    k_gemm_tc<<<grid, 128, smem, st>>>(A, B, M, N, K, BN, kpc, bias, epi, z, ldz, out, ldo, err);
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

// forward on the n rows in m->X; layer inputs kept, pre-activations kept
// for every layer when keep_z (training) and for the last layer always
void forward(emc_mlp* m, int64_t n, bool keep_z = true)
{
    const int64_t rows = (n + 15) / 16 * 16;
    k_input<<<gridn(rows * m->L[0].in_p, 256), 256, 0, m->st>>>(m->X, n, m->cfg.n_in, m->L[0].in_p, m->norm, m->act[0],
                                                                rows);
    for (int l = 0; l < m->n_layers; ++l) {
        const Layer& y = m->L[l];
        const bool last = l == m->n_layers - 1;
        gemm(m->act[l], y.Wb, (int)rows, y.out_p, y.in_p, y.b, EPI_BIAS | (last ? 0 : EPI_SILU),
             (keep_z || last) ? m->z[l] : nullptr, y.out_p, m->act[l + 1], y.out_p, m->d_err, m->st);
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
        gemm(m->dzT, m->aT, y.out_p, y.in_p, (int)rows, nullptr, 0, y.gW, y.in_p, nullptr, 0, m->d_err, m->st);
        k_colsum<<<y.out_p, 256, 0, m->st>>>(m->dzf, rows, y.out_p, y.gb);
        if (l == 0) break;
        // da = dz W  (A operand dz [rows][out_p], B operand W^T [in_p][out_p])
        k_f2b<<<gridn(nz, 256), 256, 0, m->st>>>(m->dzf, nz, m->dzb);
        gemm(m->dzb, y.WTb, (int)rows, y.in_p, y.out_p, nullptr, 0, m->da, y.in_p, nullptr, 0, m->d_err, m->st);
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

// the tensor-core kernels set the error word when a wait expired
emc_status check_device(emc_mlp* m)
{
    int e = 0;
    MCK(cudaMemcpyAsync(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    if (e) {
        MCK(cudaMemsetAsync(m->d_err, 0, sizeof(int), m->st));
        return mfail(m, EMC_ETIMEOUT, "tensor-core GEMM: wait for the MMAs expired");
    }
    return EMC_OK;
}

// The fused inference plan: every layer's weights (128-byte aligned) and one
// 128-row activation tile in shared memory.  False when they do not fit
// (the layer-by-layer path runs instead).
bool fused_plan(const emc_mlp* m, FusedNet& f, size_t& smem)
{
    size_t off = 0;
    int maxk = 16, maxn = 16;
    f.n_layers = m->n_layers;
    f.n_in = m->cfg.n_in;
    f.n_out = m->cfg.n_out;
    for (int l = 0; l < m->n_layers; ++l) {
        const Layer& y = m->L[l];
        f.W[l] = y.Wb;
        f.b[l] = y.b;
        f.in_p[l] = y.in_p;
        f.out_p[l] = y.out_p;
        f.w_off[l] = (uint32_t)off;
        off = (off + (size_t)y.out_p * y.in_p * 2 + 127) & ~size_t(127);
        maxk = std::max(maxk, std::max(y.in_p, y.out_p));
        maxn = std::max(maxn, y.out_p);
    }
    f.a_off = (uint32_t)off;
    off += (size_t)128 * maxk * 2;
    uint32_t nc = 32;
    while (nc < (uint32_t)maxn) nc <<= 1;
    f.ncols = nc;
    // no more CTAs may share an SM than its 512 tensor-memory columns hold:
    // each asks for at least 448 bytes of shared memory per column
    smem = std::max(off, (size_t)nc * 448);
    return maxn <= 256 && smem <= kFusedMaxSmem;
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
    MCK(malloc0(m, &m->d_err, 1));
    MCK(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcMaxSmem));
    MCK(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedMaxSmem));
    MCK(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared));
    emc_status s = refresh_bf16(m);
    if (s != EMC_OK) return s;
    MCK(cudaStreamSynchronize(m->st));
    return EMC_OK;
}

emc_status emc_mlp_debug_set_error(emc_mlp* m)
{
    if (!m) return EMC_EINVAL;
    const int one = 1;
    MCK(cudaMemcpyAsync(m->d_err, &one, sizeof(int), cudaMemcpyHostToDevice, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return EMC_OK;
}

emc_status emc_mlp_set_fused(emc_mlp* m, int32_t enable)
{
    if (!m) return EMC_EINVAL;
    m->fused = enable != 0;
    return EMC_OK;
}

emc_status emc_mlp_infer(emc_mlp* m, const float* X, float* Y, int64_t n)
{
    EMC_TRACE("emc_mlp_infer");
    if (!m || (n > 0 && (!X || !Y)) || n < 0) return EMC_EINVAL;
    if (n == 0) return EMC_OK;
    FusedNet f{};
    size_t fsm = 0;
    if (m->fused && fused_plan(m, f, fsm)) {
        const int64_t chunk = 1 << 20;
        const int64_t want = std::min(n, chunk);
        if (want > m->fcap) {
            mfree(m, m->fX);
            mfree(m, m->fY);
            m->fcap = 0;
            MCK(malloc0(m, &m->fX, (size_t)want * m->cfg.n_in));
            MCK(malloc0(m, &m->fY, (size_t)want * m->cfg.n_out));
            m->fcap = want;
        }
        int dev = 0, sms = 0;
        MCK(cudaGetDevice(&dev));
        MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        // two CTAs per SM where they fit (one's epilogue overlaps the other's
        // MMAs); CTAs beyond what is resident wait for a free slot, and the
        // shared-memory request keeps the resident ones within the SM's
        // tensor memory
        const int per_sm = 2;
        for (int64_t r0 = 0; r0 < n; r0 += chunk) {
            const int64_t nn = std::min(chunk, n - r0);
            MCK(cudaMemcpyAsync(m->fX, X + r0 * m->cfg.n_in, 4 * nn * m->cfg.n_in, cudaMemcpyHostToDevice, m->st));
            const int64_t tiles = (nn + 127) / 128;
            const int grid = (int)std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * sms);
            k_mlp_fused<<<grid, 128 * kFzGroups, fsm, m->st>>>(f, m->fX, nn, m->norm, m->fY, m->d_err);
            MCK(cudaGetLastError());
            MCK(cudaMemcpyAsync(Y + r0 * m->cfg.n_out, m->fY, 4 * nn * m->cfg.n_out, cudaMemcpyDeviceToHost, m->st));
        }
        MCK(cudaStreamSynchronize(m->st));
        return check_device(m);
    }
    const int64_t chunk = 1 << 16;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t nn = std::min(chunk, n - r0);
        emc_status s = ensure_batch(m, nn);
        if (s != EMC_OK) return s;
        MCK(cudaMemcpyAsync(m->X, X + r0 * m->cfg.n_in, 4 * nn * m->cfg.n_in, cudaMemcpyHostToDevice, m->st));
        forward(m, nn, false);
        const int last = m->n_layers - 1;
        k_output<<<gridn(nn * m->cfg.n_out, 256), 256, 0, m->st>>>(m->z[last], m->L[last].out_p, nn, m->cfg.n_out,
                                                                   m->norm, m->Y);
        MCK(cudaGetLastError());
        MCK(cudaMemcpyAsync(Y + r0 * m->cfg.n_out, m->Y, 4 * nn * m->cfg.n_out, cudaMemcpyDeviceToHost, m->st));
    }
    MCK(cudaStreamSynchronize(m->st));
    return check_device(m);
}

emc_status emc_mlp_grad(emc_mlp* m, const float* X, const float* Y, int64_t n, float* grad, float* loss)
{
    EMC_TRACE("emc_mlp_grad");
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
    s = check_device(m);
    if (s != EMC_OK) return s;
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
    EMC_TRACE("emc_mlp_train");
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
    return check_device(m);
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
