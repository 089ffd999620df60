// Learned warm start: a 5 -> 4 x 512 (GELU) -> 2000 MLP whose softmax output
// starts the power iteration, trained on GPU by the library's own forward
// and backward kernels.
//
// The network predicts, in a frame rolled so that the pulse bin
// c = floor(tau / Delta) sits at index 0, a log-correction z to the flux
// prior: the start vector is pi0_j ~ exp(z_{(j - c) mod N} + log lambda_j)
// (the batch kernel forms it).  Inputs: the sub-bin pulse position
// tau / Delta - c, sigma, log S, log B and x_d / t_r, scaled to about [-1, 1].
//
// All GEMMs are tcgen05 BF16 x BF16 -> FP32 kernels: TMA loads 128-byte
// swizzled 128x64 tiles into a 3-stage shared-memory ring, one thread
// issues 128x128x16 MMAs into a TMEM accumulator, and the epilogue reads
// TMEM with tcgen05.ld and fuses bias, GELU, GELU' and the layout changes
// the backward pass needs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "spl.h"
#include "spl_host_pool.h"
#include "spl_kernels.h"
#include "spl_umma.cuh"

using namespace spl;

namespace spl {
namespace mlp {

constexpr int kIn = 5;          // real input features
constexpr int kInPad = 64;      // padded K of the first layer
constexpr int kHid = 512;
constexpr int kLayers = 5;      // 4 hidden + output
constexpr int kOut = 2000;      // bins of the learned frame
constexpr int kOutPad = 2048;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr uint32_t kTileBytesA = BM * BK * 2;         // 16 KB
constexpr uint32_t kTileBytesB = BN * BK * 2;         // 32 KB
constexpr uint32_t kStageBytes = kTileBytesA + kTileBytesB;
constexpr uint32_t kTmemCols = 2 * BN;                // two accumulators: the epilogue of one tile
                                                      // overlaps the MMAs of the next
constexpr size_t kGemmSmem = (size_t)STAGES * kStageBytes + 1024;
// 12 warps, persistent (one CTA per SM, tiles strided over the grid):
// warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the MMAs, warp 2 owns the
// TMEM allocation, and warps 4..11 run the epilogue: warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (the lane quadrant a warp may access) and accumulator
// columns 128 ((w - 4) / 4) .. + 127.
constexpr int kGemmThreads = 384;
constexpr int kEpiWarp0 = 4, kEpiWarps = 8;
constexpr uint32_t kWaitLimit = 1u << 26;

enum : int { EPI_GELU = 0, EPI_LOGITS = 1, EPI_DGELU = 2, EPI_F32 = 3 };

struct GemmArgs {
    int M, N, K;                       // M % 128 == 0, K % 64 == 0, N % 32 == 0 (N tiles of 256)
    const float *bias;                 // [N]
    __nv_bfloat16 *out_bf16;           // [M][ld] row-major
    __nv_bfloat16 *out_bf16_t;         // [N][M] transposed, may be NULL
    __nv_bfloat16 *out_pre;            // [M][ld] pre-activation, may be NULL
    const __nv_bfloat16 *pre_in;       // [M][ld] pre-activation (GELU')
    float *out_f32;                    // [M][ld]
    int ld;
    int *err_flag;
};

// GELU in its tanh form, GELU(x) = x/2 (1 + tanh(k (x + 0.044715 x^3))),
// k = sqrt(2/pi) (Hendrycks and Gimpel, 2016); the hardware tanh (MUFU,
// relative error about 2^-11, far below the BF16 rounding of the stored
// activations) keeps the epilogue short.
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kGeluK = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float gelu_f(float x) {
    const float t = tanh_hw(kGeluK * fmaf(kGeluA * x, x * x, x));
    return 0.5f * x * (1.f + t);
}

// d/dx GELU = (1 + t)/2 + x/2 (1 - t^2) k (1 + 3 a x^2)
__device__ __forceinline__ float gelu_grad_f(float x) {
    const float x2 = x * x;
    const float t = tanh_hw(kGeluK * fmaf(kGeluA * x, x2, x));
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluK * fmaf(3.f * kGeluA, x2, 1.f);
}

// D[M x N] = A[M x K] * B[N x K]^T, both operands K-major BF16.
template <int MODE>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta,
                                                                   const __grid_constant__ CUtensorMap tb, GemmArgs g) {
    extern __shared__ uint8_t gemm_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];
    __shared__ __align__(8) uint64_t tempty_bar[2];
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KB = g.K / BK;
    // tiles in row-major order of (M tile, N tile): the CTAs running at one
    // time share A tiles (one 128-row slice of the activations) through L2
    const int n_tiles = (g.N + BN - 1) / BN;
    const int total = (g.M / BM) * n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            umma::mbar_init(&full_bar[s], 1);
            umma::mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&tfull_bar[b], 1);
            umma::mbar_init(&tempty_bar[b], kEpiWarps);
        }
        umma::fence_barrier_init();
        umma::prefetch_tmap(&ta);
        umma::prefetch_tmap(&tb);
    }
    if (warp == 2) {
        umma::tmem_alloc(&tmem_base, kTmemCols);
        umma::tmem_relinquish();
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = tmem_base;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // TMA producer: a ring of STAGES (A, B) k-blocks across all tiles
        uint32_t it = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
            for (int kb = 0; kb < KB; ++kb, ++it) {
                const uint32_t s = it % STAGES;
                if (it >= STAGES && !umma::mbar_wait(&empty_bar[s], ((it / STAGES) - 1) & 1, kWaitLimit)) {
                    ok = false;
                    break;
                }
                uint8_t *st = smem + (size_t)s * kStageBytes;
                umma::mbar_arrive_expect_tx(&full_bar[s], kStageBytes);
                umma::tma_load_2d(st, &ta, &full_bar[s], kb * BK, m0);
                umma::tma_load_2d(st + kTileBytesA, &tb, &full_bar[s], kb * BK, n0);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tile i accumulates into TMEM buffer i % 2 once the
        // epilogue has emptied it
        const uint32_t idesc = umma::idesc_bf16_f32(BM, BN);
        uint32_t it = 0, i = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
            const uint32_t buf = i & 1;
            if (i >= 2 && !umma::mbar_wait(&tempty_bar[buf], ((i >> 1) - 1) & 1, kWaitLimit)) {
                ok = false;
                break;
            }
            umma::tc_fence_after();
            const uint32_t acc = tmem + buf * BN;
            for (int kb = 0; kb < KB; ++kb, ++it) {
                const uint32_t s = it % STAGES;
                if (!umma::mbar_wait(&full_bar[s], (it / STAGES) & 1, kWaitLimit)) {
                    ok = false;
                    break;
                }
                umma::tc_fence_after();
                const uint32_t a_addr = umma::smem_addr(smem + (size_t)s * kStageBytes);
                const uint32_t b_addr = a_addr + kTileBytesA;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    // advance 16 bf16 (32 bytes) along K inside the 128-byte swizzle atom
                    umma::mma_bf16(acc, umma::sdesc_kmajor_sw128(a_addr + kk * 32),
                                   umma::sdesc_kmajor_sw128(b_addr + kk * 32), idesc, (kb | kk) ? 1u : 0u);
                }
                umma::mma_commit(&empty_bar[s]);
            }
            umma::mma_commit(&tfull_bar[buf]);
        }
    } else if (warp >= kEpiWarp0) {
        // Epilogue: warp w owns accumulator rows 32 (w % 4) .. + 31 (TMEM
        // lanes) and columns 128 ((w - 4) / 4) .. + 127 of each tile.
        const int quad = warp & 3, half = (warp - kEpiWarp0) >> 2;
        uint32_t i = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
            const uint32_t buf = i & 1;
            if (!umma::mbar_wait(&tfull_bar[buf], (i >> 1) & 1, kWaitLimit)) {
                ok = false;
                break;
            }
            umma::tc_fence_after();
            const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
            const int row = m0 + quad * 32 + lane;
#pragma unroll 1
            for (int c0 = 128 * half; c0 < 128 * half + 128; c0 += 32) {
                uint32_t r[32];
                umma::tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + buf * BN + (uint32_t)c0, r);
                umma::tmem_ld_wait();
                const int nb = n0 + c0;
                if (nb >= g.N) continue;
                float v[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
                if (MODE == EPI_GELU || MODE == EPI_LOGITS) {
                    const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + nb);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 bb = __ldg(b4 + q);
                        v[4 * q] += bb.x;
                        v[4 * q + 1] += bb.y;
                        v[4 * q + 2] += bb.z;
                        v[4 * q + 3] += bb.w;
                    }
                }
                if (MODE == EPI_GELU) {
                    if (g.out_pre) {
                        uint4 *dst = reinterpret_cast<uint4 *>(g.out_pre + (size_t)row * g.ld + nb);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            __nv_bfloat162 h[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                h[e] = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
                            dst[q] = *reinterpret_cast<uint4 *>(h);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = gelu_f(v[c]);
                }
                if (MODE == EPI_DGELU) {
                    const __nv_bfloat16 *pre = g.pre_in + (size_t)row * g.ld + nb;
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] *= gelu_grad_f(__bfloat162float(pre[c]));
                }
                if (MODE == EPI_GELU || MODE == EPI_DGELU) {
                    uint4 *dst = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld + nb);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        __nv_bfloat162 h[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            h[e] = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
                        dst[q] = *reinterpret_cast<uint4 *>(h);
                    }
                    if (g.out_bf16_t) {
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (nb + c < g.N) g.out_bf16_t[(size_t)(nb + c) * g.M + row] = __float2bfloat16_rn(v[c]);
                    }
                } else {
                    float4 *dst = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld + nb);
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            // this warp is done with the buffer
            umma::tc_fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tempty_bar[buf]);
        }
    }
    if (!ok && g.err_flag) atomicExch(g.err_flag, 1);
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        umma::tc_fence_after();
        umma::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------- auxiliary kernels

// Input features (bf16, padded to 64 columns) and their transpose.
__global__ void features_kernel(const spl_pixel_t *__restrict__ px, int n, int M, __nv_bfloat16 *__restrict__ X,
                                __nv_bfloat16 *__restrict__ Xt) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float f[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (m < n) {
        const spl_pixel_t p = px[m];
        const int c = mlp_frame_shift(p.t_r, p.tau, p.n_bins);
        const double pos = p.tau * (double)p.n_bins / p.t_r;
        f[0] = (float)(2.0 * (pos - (double)c) - 1.0);
        f[1] = (float)((p.sigma - 0.6) / 0.4);
        f[2] = (float)((log(fmax(p.S, 1e-30)) + 1.5) / 3.1);
        f[3] = (float)((log(fmax(p.B, 1e-30)) + 1.5) / 3.1);
        f[4] = (float)(2.0 * fmod(p.t_d, p.t_r) / p.t_r - 1.0);
    }
    for (int k = 0; k < kInPad; ++k) {
        const __nv_bfloat16 v = __float2bfloat16_rn(k < kIn ? f[k] : 0.f);
        X[(size_t)m * kInPad + k] = v;
        if (Xt) Xt[(size_t)k * M + m] = v;
    }
}

// Cross-entropy of the start vector against the target pmf and its gradient
// with respect to the network output (learned frame).  One block per pixel:
//   e_j = z_{(j - c) mod N} + log lambda_j,  q = softmax(e),
//   loss = -sum_j t_j log q_j,  dz_{(j - c) mod N} = (q_j - t_j) * scale.
template <int NT>
__global__ void __launch_bounds__(NT) softmax_loss_kernel(const spl_pixel_t *__restrict__ px, int n, int M,
                                                           const float *__restrict__ logits,
                                                           const float *__restrict__ target, float scale,
                                                           __nv_bfloat16 *__restrict__ dz,
                                                           __nv_bfloat16 *__restrict__ dzt, float *__restrict__ loss) {
    __shared__ float e[kOut];
    __shared__ float red[NT / 32 + 2];
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    if (m >= n) {   // padded rows: zero gradient
        for (int i = tid; i < kOutPad; i += NT) {
            dz[(size_t)m * kOutPad + i] = __float2bfloat16_rn(0.f);
            dzt[(size_t)i * M + m] = __float2bfloat16_rn(0.f);
        }
        return;
    }
    const spl_pixel_t p = px[m];
    const int N = kOut;
    const int c = mlp_frame_shift(p.t_r, p.tau, N);
    const float *z = logits + (size_t)m * kOutPad;
    float mx = -INFINITY;
    for (int j = tid; j < N; j += NT) {
        const double s = ((double)j + 0.5) * p.t_r / N;
        const double zz = (s - p.tau) / p.sigma;
        const double lam = p.S * exp(-0.5 * zz * zz) * 0.39894228040143267794 / p.sigma + p.B / p.t_r;
        int i = j - c;
        i += (i < 0) ? N : 0;
        const float v = z[i] + logf((float)lam);
        e[j] = v;
        mx = fmaxf(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        float v = red[0];
        for (int w = 1; w < NT / 32; ++w) v = fmaxf(v, red[w]);
        red[NT / 32] = v;
    }
    __syncthreads();
    mx = red[NT / 32];
    __syncthreads();
    float sum = 0.f;
    for (int j = tid; j < N; j += NT) sum += __expf(e[j] - mx);
    const float S = block_sum<NT>(sum, red);
    const float lse = mx + logf(S);
    float ls = 0.f;
    for (int j = tid; j < N; j += NT) {
        const float t = target[(size_t)m * N + j];
        const float q = __expf(e[j] - lse);
        ls -= t * (e[j] - lse);
        int i = j - c;
        i += (i < 0) ? N : 0;
        const __nv_bfloat16 gv = __float2bfloat16_rn((q - t) * scale);
        dz[(size_t)m * kOutPad + i] = gv;
        dzt[(size_t)i * M + m] = gv;
    }
    for (int i = N + tid; i < kOutPad; i += NT) {
        dz[(size_t)m * kOutPad + i] = __float2bfloat16_rn(0.f);
        dzt[(size_t)i * M + m] = __float2bfloat16_rn(0.f);
    }
    const float L = block_sum<NT>(ls, red);
    if (tid == 0) loss[m] = L;
}

// db_n = sum_m dA[m][n], from the transposed gradient (one warp per n).
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ dAt, int Nn, int M, float *__restrict__ db) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= Nn) return;
    float s = 0.f;
    for (int m = lane; m < M; m += 32) s += __bfloat162float(dAt[(size_t)n * M + m]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[n] = s;
}

// AdamW on FP32 master parameters; refreshes the BF16 weight and its
// transpose.  Padding (rows >= Nreal, columns >= Kreal) stays zero.
__global__ void adamw_kernel(float *__restrict__ w, float *__restrict__ mom, float *__restrict__ vel,
                             const float *__restrict__ grad, int64_t count, int rows, int cols, int Kreal,
                             int Nreal, int apply, float lr, float b1, float b2, float c1, float c2, float eps,
                             float wd, __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wbt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) {
        const int r = cols > 0 ? (int)(i / cols) : 0;
        const int k = cols > 0 ? (int)(i - (int64_t)r * cols) : (int)i;
        const bool real = cols > 0 ? (r < Nreal && k < Kreal) : (i < Nreal);
        float x = w[i];
        if (real && apply) {
            const float gr = grad[i];
            const float m = b1 * mom[i] + (1.f - b1) * gr;
            const float v = b2 * vel[i] + (1.f - b2) * gr * gr;
            mom[i] = m;
            vel[i] = v;
            const float mh = m / c1, vh = v / c2;
            x -= lr * (mh / (sqrtf(vh) + eps) + wd * x);
            w[i] = x;
        }
        if (wb) {
            const __nv_bfloat16 b = __float2bfloat16_rn(real ? x : 0.f);
            wb[i] = b;
            if (wbt) wbt[(size_t)k * rows + r] = b;
        }
    }
}

}  // namespace mlp
}  // namespace spl

// ======================================================================
// Host side
// ======================================================================

using namespace spl::mlp;

namespace {

spl_status_t mfail(cudaError_t e, const char *where) { return note_cuda_error(e, where); }

#define MCU(expr)                                          \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return mfail(e_, #expr);    \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows][cols] with box_rows x 64 boxes
// and 128-byte swizzle (cols * 2 must be a multiple of 16).
bool tmap_bf16(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t launch_gemm_mode(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &g, cudaStream_t s) {
    auto k = gemm_bf16_kernel<MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int tiles = (g.M / BM) * ((g.N + BN - 1) / BN);
    k<<<tiles < sms ? tiles : sms, kGemmThreads, kGemmSmem, s>>>(ta, tb, g);
    return cudaGetLastError();
}

// D = A[M][K] * B[N][K]^T with A, B row-major bf16 device matrices.
spl_status_t gemm(int mode, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int Nrows_b,
                  GemmArgs g, cudaStream_t s) {
    if (M % BM || K % BK) return SPL_EINVAL;
    CUtensorMap ta, tb;
    if (!tmap_bf16(&ta, A, M, K, BM) || !tmap_bf16(&tb, B, Nrows_b, K, BN)) return mfail(cudaErrorInvalidValue, "tmap");
    g.M = M;
    g.N = N;
    g.K = K;
    cudaError_t e;
    switch (mode) {
        case EPI_GELU: e = launch_gemm_mode<EPI_GELU>(ta, tb, g, s); break;
        case EPI_LOGITS: e = launch_gemm_mode<EPI_LOGITS>(ta, tb, g, s); break;
        case EPI_DGELU: e = launch_gemm_mode<EPI_DGELU>(ta, tb, g, s); break;
        default: e = launch_gemm_mode<EPI_F32>(ta, tb, g, s); break;
    }
    return e == cudaSuccess ? SPL_OK : mfail(e, "gemm launch");
}

// Layer l: W [rows_l][cols_l] (padded), real [nreal_l][kreal_l].
const int kRows[kLayers] = {kHid, kHid, kHid, kHid, kOutPad};
const int kCols[kLayers] = {kInPad, kHid, kHid, kHid, kHid};
const int kNreal[kLayers] = {kHid, kHid, kHid, kHid, kOut};
const int kKreal[kLayers] = {kIn, kHid, kHid, kHid, kHid};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
}

}  // namespace

struct spl_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0;      // padded to a multiple of 128
    // parameters (FP32 master, Adam moments, BF16 copies)
    float *W[kLayers] = {}, *b[kLayers] = {};
    float *mW[kLayers] = {}, *vW[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
    float *gW[kLayers] = {}, *gb[kLayers] = {};
    __nv_bfloat16 *Wb[kLayers] = {}, *Wbt[kLayers] = {};
    // activations [M][512], transposes [512][M], pre-activations
    __nv_bfloat16 *X = nullptr, *Xt = nullptr;
    __nv_bfloat16 *H[4] = {}, *Ht[4] = {}, *A[4] = {};
    __nv_bfloat16 *dA[4] = {}, *dAt[4] = {};
    __nv_bfloat16 *dZ = nullptr, *dZt = nullptr;
    float *logits = nullptr;   // [M][2048]
    float *warm = nullptr;     // [warm_cap][2048] logits of a whole learned batch
    size_t warm_cap = 0;
    float *loss = nullptr;     // [M]
    spl_pixel_t *d_px = nullptr;
    spl_pixel_t *h_stage = nullptr;   // pinned staging of the pixels to upload [max_batch]
    cudaEvent_t ev_stage = nullptr;   // the last copy out of h_stage
    int *err = nullptr;
    int step = 0;
};

namespace {

void mlp_release(spl_mlp *m) {
    if (!m) return;
    for (int l = 0; l < kLayers; ++l) {
        void *p[] = {m->W[l], m->b[l], m->mW[l], m->vW[l], m->mb[l], m->vb[l], m->gW[l], m->gb[l], m->Wb[l], m->Wbt[l]};
        for (void *q : p)
            if (q) cudaFree(q);
    }
    for (int l = 0; l < 4; ++l) {
        void *p[] = {m->H[l], m->Ht[l], m->A[l], m->dA[l], m->dAt[l]};
        for (void *q : p)
            if (q) cudaFree(q);
    }
    void *p[] = {m->X, m->Xt, m->dZ, m->dZt, m->logits, m->loss, m->d_px, m->err, m->warm};
    for (void *q : p)
        if (q) cudaFree(q);
    if (m->ev_stage) cudaEventSynchronize(m->ev_stage);
    if (m->h_stage) cudaFreeHost(m->h_stage);
    if (m->ev_stage) cudaEventDestroy(m->ev_stage);
    delete m;
}

spl_status_t refresh_bf16(spl_mlp *m) {
    for (int l = 0; l < kLayers; ++l) {
        const int64_t cnt = (int64_t)kRows[l] * kCols[l];
        const int blocks = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
        // zero learning rate: only re-derives the BF16 copies
        adamw_kernel<<<blocks, 256, 0, m->stream>>>(m->W[l], m->mW[l], m->vW[l], m->gW[l], cnt, kRows[l], kCols[l],
                                                    kKreal[l], kNreal[l], 0, 0.f, 0.9f, 0.999f, 1.f, 1.f, 1e-8f,
                                                    0.f, m->Wb[l], m->Wbt[l]);
        MCU(cudaGetLastError());
    }
    return SPL_OK;
}

spl_status_t check_batch(spl_mlp *m, const spl_pixel_t *h_px, int n) {
    if (!m || !h_px || n < 1 || n > m->max_batch) return SPL_EINVAL;
    for (int k = 0; k < n; ++k) {
        const spl_pixel_t &p = h_px[k];
        if (p.n_bins != kOut || !(p.t_r > 0) || !(p.sigma > 0) || p.tau < 0 || p.tau >= p.t_r || p.S < 0 ||
            p.B <= 0 || !std::isfinite(p.S + p.B + p.t_d + p.tau + p.sigma + p.t_r))
            return SPL_EINVAL;
    }
    return SPL_OK;
}

int padM(int n) { return (n + BM - 1) / BM * BM; }

// Forward pass for n pixels already on the device; train=1 keeps the
// transposes and pre-activations the backward pass needs.
spl_status_t forward(spl_mlp *m, int n, bool train, float *logits_out = nullptr) {
    cudaStream_t s = m->stream;
    const int M = padM(n);
    features_kernel<<<(M + 127) / 128, 128, 0, s>>>(m->d_px, n, M, m->X, train ? m->Xt : nullptr);
    MCU(cudaGetLastError());
    const __nv_bfloat16 *in = m->X;
    int K = kInPad;
    for (int l = 0; l < 4; ++l) {
        GemmArgs g{};
        g.bias = m->b[l];
        g.out_bf16 = m->H[l];
        g.out_bf16_t = train ? m->Ht[l] : nullptr;
        g.out_pre = train ? m->A[l] : nullptr;
        g.ld = kHid;
        g.err_flag = m->err;
        spl_status_t st = gemm(EPI_GELU, in, m->Wb[l], M, kHid, K, kRows[l], g, s);
        if (st != SPL_OK) return st;
        in = m->H[l];
        K = kHid;
    }
    GemmArgs g{};
    g.bias = m->b[4];
    g.out_f32 = logits_out ? logits_out : m->logits;
    g.ld = kOutPad;
    g.err_flag = m->err;
    return gemm(EPI_LOGITS, in, m->Wb[4], M, kOutPad, kHid, kRows[4], g, s);
}

// Loss and gradients for n pixels with targets d_target [n][2000].
spl_status_t backward(spl_mlp *m, int n, const float *d_target) {
    cudaStream_t s = m->stream;
    const int M = padM(n);
    softmax_loss_kernel<256><<<M, 256, 0, s>>>(m->d_px, n, M, m->logits, d_target, 1.f / (float)n, m->dZ, m->dZt,
                                               m->loss);
    MCU(cudaGetLastError());
    // output layer
    {
        GemmArgs g{};
        g.out_f32 = m->gW[4];
        g.ld = kHid;
        g.err_flag = m->err;
        spl_status_t st = gemm(EPI_F32, m->dZt, m->Ht[3], kOutPad, kHid, M, kHid, g, s);
        if (st != SPL_OK) return st;
        bias_grad_kernel<<<(kOutPad + 7) / 8, 256, 0, s>>>(m->dZt, kOutPad, M, m->gb[4]);
        MCU(cudaGetLastError());
        GemmArgs h{};
        h.out_bf16 = m->dA[3];
        h.out_bf16_t = m->dAt[3];
        h.pre_in = m->A[3];
        h.ld = kHid;
        h.err_flag = m->err;
        st = gemm(EPI_DGELU, m->dZ, m->Wbt[4], M, kHid, kOutPad, kHid, h, s);
        if (st != SPL_OK) return st;
    }
    for (int l = 3; l >= 0; --l) {
        // dW_l = dA_l^T * H_{l-1}  (H_{-1} = X)
        const __nv_bfloat16 *Hin_t = l > 0 ? m->Ht[l - 1] : m->Xt;
        const int Kin = l > 0 ? kHid : kInPad;
        GemmArgs g{};
        g.out_f32 = m->gW[l];
        g.ld = Kin;
        g.err_flag = m->err;
        spl_status_t st = gemm(EPI_F32, m->dAt[l], Hin_t, kHid, Kin, M, Kin, g, s);
        if (st != SPL_OK) return st;
        bias_grad_kernel<<<(kHid + 7) / 8, 256, 0, s>>>(m->dAt[l], kHid, M, m->gb[l]);
        MCU(cudaGetLastError());
        if (l > 0) {
            GemmArgs h{};
            h.out_bf16 = m->dA[l - 1];
            h.out_bf16_t = m->dAt[l - 1];
            h.pre_in = m->A[l - 1];
            h.ld = kHid;
            h.err_flag = m->err;
            st = gemm(EPI_DGELU, m->dA[l], m->Wbt[l], M, kHid, kHid, kHid, h, s);
            if (st != SPL_OK) return st;
        }
    }
    return SPL_OK;
}

// The caller's pixels (pageable memory) are copied into the pinned staging
// buffer on the host pool, then sent with one asynchronous copy: a direct
// copy from pageable memory would hold the host for the driver's own staging
// while the GPU waits.  The staging buffer is refilled only after its last
// copy has run.
spl_status_t upload_pixels(spl_mlp *m, const spl_pixel_t *h_px, int n) {
    MCU(cudaEventSynchronize(m->ev_stage));
    spl_pixel_t *dst = m->h_stage;
    spl::host_parallel_for(n, 4096, [&](int64_t lo, int64_t hi) {
        std::memcpy(dst + lo, h_px + lo, sizeof(spl_pixel_t) * (size_t)(hi - lo));
    });
    MCU(cudaMemcpyAsync(m->d_px, dst, sizeof(spl_pixel_t) * n, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaEventRecord(m->ev_stage, m->stream));
    return SPL_OK;
}

spl_status_t read_err(spl_mlp *m) {
    int h = 0;
    MCU(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    return h ? SPL_ETIMEOUT : SPL_OK;
}

// Canonical packed parameter order: for each layer W (real rows x real
// cols, row-major) then b (real rows).
int64_t packed_count() {
    int64_t c = 0;
    for (int l = 0; l < kLayers; ++l) c += (int64_t)kNreal[l] * kKreal[l] + kNreal[l];
    return c;
}

}  // namespace

extern "C" int64_t spl_mlp_param_count(void) { return packed_count(); }

extern "C" spl_status_t spl_mlp_create(int32_t max_batch, uint64_t seed, void *stream, spl_mlp_t **out) {
    if (!out || max_batch < 1 || max_batch > (1 << 22)) return SPL_EINVAL;
    *out = nullptr;
    spl_mlp *m = new (std::nothrow) spl_mlp();
    if (!m) return SPL_ENOMEM;
    m->stream = static_cast<cudaStream_t>(stream);
    m->max_batch = padM(max_batch);
    const int M = m->max_batch;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    for (int l = 0; l < kLayers; ++l) {
        const size_t cnt = (size_t)kRows[l] * kCols[l];
        chk(dalloc(&m->W[l], cnt)); chk(dalloc(&m->mW[l], cnt)); chk(dalloc(&m->vW[l], cnt)); chk(dalloc(&m->gW[l], cnt));
        chk(dalloc(&m->b[l], kRows[l])); chk(dalloc(&m->mb[l], kRows[l])); chk(dalloc(&m->vb[l], kRows[l]));
        chk(dalloc(&m->gb[l], kRows[l]));
        chk(dalloc(&m->Wb[l], cnt)); chk(dalloc(&m->Wbt[l], cnt));
    }
    chk(dalloc(&m->X, (size_t)M * kInPad));
    chk(dalloc(&m->Xt, (size_t)M * kInPad));
    for (int l = 0; l < 4; ++l) {
        chk(dalloc(&m->H[l], (size_t)M * kHid)); chk(dalloc(&m->Ht[l], (size_t)M * kHid));
        chk(dalloc(&m->A[l], (size_t)M * kHid)); chk(dalloc(&m->dA[l], (size_t)M * kHid));
        chk(dalloc(&m->dAt[l], (size_t)M * kHid));
    }
    chk(dalloc(&m->dZ, (size_t)M * kOutPad));
    chk(dalloc(&m->dZt, (size_t)M * kOutPad));
    chk(dalloc(&m->logits, (size_t)M * kOutPad));
    chk(dalloc(&m->loss, (size_t)M));
    chk(dalloc(&m->d_px, (size_t)M));
    chk(cudaHostAlloc(reinterpret_cast<void **>(&m->h_stage), sizeof(spl_pixel_t) * (size_t)M, cudaHostAllocDefault));
    chk(cudaEventCreateWithFlags(&m->ev_stage, cudaEventDisableTiming));
    chk(dalloc(&m->err, 1));
    if (e != cudaSuccess) { mlp_release(m); return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : mfail(e, "alloc"); }
    // Initialisation on the host (uniform fan-in scaling, seeded), zero padding.
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto urand = [&]() {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return (double)(st >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < kLayers; ++l) {
        std::vector<float> w((size_t)kRows[l] * kCols[l], 0.f), b(kRows[l], 0.f);
        const double a = std::sqrt(3.0 / kKreal[l]);
        for (int r = 0; r < kNreal[l]; ++r)
            for (int k = 0; k < kKreal[l]; ++k) w[(size_t)r * kCols[l] + k] = (float)((2.0 * urand() - 1.0) * a);
        chk(cudaMemcpy(m->W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(m->b[l], b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice));
        chk(cudaMemset(m->mW[l], 0, sizeof(float) * w.size())); chk(cudaMemset(m->vW[l], 0, sizeof(float) * w.size()));
        chk(cudaMemset(m->gW[l], 0, sizeof(float) * w.size()));
        chk(cudaMemset(m->mb[l], 0, sizeof(float) * b.size())); chk(cudaMemset(m->vb[l], 0, sizeof(float) * b.size()));
        chk(cudaMemset(m->gb[l], 0, sizeof(float) * b.size()));
    }
    chk(cudaMemset(m->err, 0, sizeof(int)));
    if (e != cudaSuccess) { mlp_release(m); return mfail(e, "init"); }
    spl_status_t s2 = refresh_bf16(m);
    if (s2 != SPL_OK) { mlp_release(m); return s2; }
    *out = m;
    return SPL_OK;
}

extern "C" void spl_mlp_free(spl_mlp_t *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_release(m);
}

extern "C" spl_status_t spl_mlp_set_params(spl_mlp_t *m, const float *h, int64_t count) {
    if (!m || !h || count != packed_count()) return SPL_EINVAL;
    MCU(cudaStreamSynchronize(m->stream));
    const float *p = h;
    for (int l = 0; l < kLayers; ++l) {
        std::vector<float> w((size_t)kRows[l] * kCols[l], 0.f), b(kRows[l], 0.f);
        for (int r = 0; r < kNreal[l]; ++r)
            for (int k = 0; k < kKreal[l]; ++k) w[(size_t)r * kCols[l] + k] = *p++;
        for (int r = 0; r < kNreal[l]; ++r) b[r] = *p++;
        MCU(cudaMemcpy(m->W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
        MCU(cudaMemcpy(m->b[l], b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice));
    }
    return refresh_bf16(m);
}

static spl_status_t get_packed(spl_mlp_t *m, float *const *W, float *const *b, float *h) {
    MCU(cudaStreamSynchronize(m->stream));
    float *p = h;
    for (int l = 0; l < kLayers; ++l) {
        std::vector<float> w((size_t)kRows[l] * kCols[l]), bb(kRows[l]);
        MCU(cudaMemcpy(w.data(), W[l], sizeof(float) * w.size(), cudaMemcpyDeviceToHost));
        MCU(cudaMemcpy(bb.data(), b[l], sizeof(float) * bb.size(), cudaMemcpyDeviceToHost));
        for (int r = 0; r < kNreal[l]; ++r)
            for (int k = 0; k < kKreal[l]; ++k) *p++ = w[(size_t)r * kCols[l] + k];
        for (int r = 0; r < kNreal[l]; ++r) *p++ = bb[r];
    }
    return SPL_OK;
}

extern "C" spl_status_t spl_mlp_get_params(spl_mlp_t *m, float *h, int64_t count) {
    if (!m || !h || count != packed_count()) return SPL_EINVAL;
    return get_packed(m, m->W, m->b, h);
}

static spl_status_t set_packed(spl_mlp_t *m, float *const *W, float *const *b, const float *h) {
    MCU(cudaStreamSynchronize(m->stream));
    const float *p = h;
    for (int l = 0; l < kLayers; ++l) {
        std::vector<float> w((size_t)kRows[l] * kCols[l], 0.f), bb(kRows[l], 0.f);
        for (int r = 0; r < kNreal[l]; ++r)
            for (int k = 0; k < kKreal[l]; ++k) w[(size_t)r * kCols[l] + k] = *p++;
        for (int r = 0; r < kNreal[l]; ++r) bb[r] = *p++;
        MCU(cudaMemcpy(W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
        MCU(cudaMemcpy(b[l], bb.data(), sizeof(float) * bb.size(), cudaMemcpyHostToDevice));
    }
    return SPL_OK;
}

// AdamW state: first moments then second moments, each packed like the
// parameters (padding entries stay zero: their gradients are zero), and the
// step count used for bias correction.
extern "C" spl_status_t spl_mlp_get_state(spl_mlp_t *m, float *h, int64_t count, int32_t *step) {
    const int64_t pc = packed_count();
    if (!m || !h || !step || count != 2 * pc) return SPL_EINVAL;
    spl_status_t st = get_packed(m, m->mW, m->mb, h);
    if (st == SPL_OK) st = get_packed(m, m->vW, m->vb, h + pc);
    if (st == SPL_OK) *step = m->step;
    return st;
}

extern "C" spl_status_t spl_mlp_set_state(spl_mlp_t *m, const float *h, int64_t count, int32_t step) {
    const int64_t pc = packed_count();
    if (!m || !h || count != 2 * pc || step < 0) return SPL_EINVAL;
    spl_status_t st = set_packed(m, m->mW, m->mb, h);
    if (st == SPL_OK) st = set_packed(m, m->vW, m->vb, h + pc);
    if (st == SPL_OK) m->step = step;
    return st;
}

extern "C" spl_status_t spl_mlp_forward(spl_mlp_t *m, const spl_pixel_t *h_px, int32_t n, float *d_logits) {
    spl_status_t st = check_batch(m, h_px, n);
    if (st != SPL_OK) return st;
    MCU(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    if ((st = upload_pixels(m, h_px, n)) != SPL_OK) return st;
    if ((st = forward(m, n, false)) != SPL_OK) return st;
    if (d_logits)
        MCU(cudaMemcpyAsync(d_logits, m->logits, sizeof(float) * (size_t)n * kOutPad, cudaMemcpyDeviceToDevice,
                            m->stream));
    return read_err(m);
}

extern "C" spl_status_t spl_mlp_time_forward(spl_mlp_t *m, const spl_pixel_t *h_px, int32_t n, int32_t reps,
                                             float *ms_per_forward) {
    if (!ms_per_forward || reps < 1) return SPL_EINVAL;
    spl_status_t st = check_batch(m, h_px, n);
    if (st != SPL_OK) return st;
    MCU(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    if ((st = upload_pixels(m, h_px, n)) != SPL_OK) return st;
    if ((st = forward(m, n, false)) != SPL_OK) return st;   // warm-up
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MCU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, m->stream);
    for (int32_t r = 0; r < reps && e == cudaSuccess && st == SPL_OK; ++r) st = forward(m, n, false);
    if (e == cudaSuccess && st == SPL_OK) e = cudaEventRecord(e1, m->stream);
    if (e == cudaSuccess && st == SPL_OK) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess && st == SPL_OK) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != SPL_OK) return st;
    if (e != cudaSuccess) return mfail(e, "time forward");
    *ms_per_forward = ms / (float)reps;
    return read_err(m);
}

extern "C" spl_status_t spl_mlp_loss_grad(spl_mlp_t *m, const spl_pixel_t *h_px, int32_t n, const float *d_target,
                                          float *h_loss, float *h_grads) {
    spl_status_t st = check_batch(m, h_px, n);
    if (st != SPL_OK || !d_target) return st != SPL_OK ? st : SPL_EINVAL;
    MCU(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    if ((st = upload_pixels(m, h_px, n)) != SPL_OK) return st;
    if ((st = forward(m, n, true)) != SPL_OK) return st;
    if ((st = backward(m, n, d_target)) != SPL_OK) return st;
    if ((st = read_err(m)) != SPL_OK) return st;
    if (h_loss) {
        std::vector<float> l((size_t)n);
        MCU(cudaMemcpy(l.data(), m->loss, sizeof(float) * n, cudaMemcpyDeviceToHost));
        double s = 0;
        for (float x : l) s += x;
        *h_loss = (float)(s / n);
    }
    if (h_grads) return get_packed(m, m->gW, m->gb, h_grads);
    return SPL_OK;
}

extern "C" spl_status_t spl_mlp_train_step(spl_mlp_t *m, const spl_pixel_t *h_px, int32_t n, const float *d_target,
                                           float lr, float weight_decay, float *h_loss) {
    spl_status_t st = check_batch(m, h_px, n);
    if (st != SPL_OK || !d_target || !(lr >= 0.f)) return st != SPL_OK ? st : SPL_EINVAL;
    if ((st = upload_pixels(m, h_px, n)) != SPL_OK) return st;
    if ((st = forward(m, n, true)) != SPL_OK) return st;
    if ((st = backward(m, n, d_target)) != SPL_OK) return st;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    for (int l = 0; l < kLayers; ++l) {
        const int64_t cnt = (int64_t)kRows[l] * kCols[l];
        const int blocks = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
        adamw_kernel<<<blocks, 256, 0, m->stream>>>(m->W[l], m->mW[l], m->vW[l], m->gW[l], cnt, kRows[l], kCols[l],
                                                    kKreal[l], kNreal[l], 1, lr, b1, b2, c1, c2, 1e-8f,
                                                    weight_decay, m->Wb[l], m->Wbt[l]);
        MCU(cudaGetLastError());
        adamw_kernel<<<(kRows[l] + 255) / 256, 256, 0, m->stream>>>(m->b[l], m->mb[l], m->vb[l], m->gb[l], kRows[l],
                                                                  0, 0, 0, kNreal[l], 1, lr, b1, b2, c1, c2,
                                                                  1e-8f, 0.f, nullptr, nullptr);
        MCU(cudaGetLastError());
    }
    if (h_loss) {
        std::vector<float> l((size_t)n);
        MCU(cudaMemcpyAsync(l.data(), m->loss, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
        MCU(cudaStreamSynchronize(m->stream));
        double s = 0;
        for (float x : l) s += x;
        *h_loss = (float)(s / n);
    }
    return SPL_OK;
}

// Raw GEMM for tests: D[M][N] = A[M][K] * B[N][K]^T (bf16 in, fp32 out).
extern "C" spl_status_t spl_gemm_bf16(const void *d_A, const void *d_B, int32_t M, int32_t N, int32_t K, float *d_D,
                                      void *stream) {
    if (!d_A || !d_B || !d_D || M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64 || N % 32) return SPL_EINVAL;
    int *err = nullptr;
    MCU(cudaMalloc(&err, sizeof(int)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MCU(cudaMemsetAsync(err, 0, sizeof(int), s));
    GemmArgs g{};
    g.out_f32 = d_D;
    g.ld = N;
    g.err_flag = err;
    spl_status_t st = gemm(EPI_F32, static_cast<const __nv_bfloat16 *>(d_A), static_cast<const __nv_bfloat16 *>(d_B),
                           M, N, K, N, g, s);
    int h = 0;
    if (st == SPL_OK) {
        MCU(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        MCU(cudaStreamSynchronize(s));
    }
    cudaFree(err);
    if (st != SPL_OK) return st;
    return h ? SPL_ETIMEOUT : SPL_OK;
}

// The logits buffer of the last spl_mlp_forward, [n][2048] (device, owned by m).
extern "C" const float *spl_mlp_logits(spl_mlp_t *m) { return m ? m->logits : nullptr; }

// Logits of the whole batch into m->warm, chunk by chunk (max_batch rows at a time).
static spl_status_t learned_logits(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n) {
    const size_t rows = (size_t)padM(n);
    if (m->warm_cap < rows) {
        if (m->warm) cudaFree(m->warm);
        m->warm = nullptr;
        m->warm_cap = 0;
        cudaError_t e = dalloc(&m->warm, rows * kOutPad);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : mfail(e, "warm logits");
        m->warm_cap = rows;
    }
    MCU(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    for (int32_t k0 = 0; k0 < n; k0 += m->max_batch) {
        const int32_t c = std::min<int32_t>(m->max_batch, n - k0);
        spl_status_t st = check_batch(m, h_pixels + k0, c);
        if (st != SPL_OK) return st;
        if ((st = upload_pixels(m, h_pixels + k0, c)) != SPL_OK) return st;
        if ((st = forward(m, c, false, m->warm + (size_t)k0 * kOutPad)) != SPL_OK) return st;
    }
    return SPL_OK;
}

extern "C" spl_status_t spl_batch_stationary_learned_host(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n,
                                                          double tol, int32_t max_iter, float *h_out,
                                                          spl_report_t *h_reports, void *stream,
                                                          const spl_batch_opts_t *opts) {
    if (!m || n < 1 || !h_pixels || !h_out) return SPL_EINVAL;
    if (stream != static_cast<void *>(m->stream)) return SPL_EINVAL;
    spl_status_t st = learned_logits(m, h_pixels, n);
    if (st != SPL_OK) return st;
    st = batch_host_run(h_pixels, n, tol, max_iter, m->warm, nullptr, SPL_WARM_LEARNED, kOutPad, h_out, h_reports,
                        m->stream, opts);
    if (st == SPL_OK || st == SPL_ENOCONV) {
        int h = 0;
        MCU(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
        MCU(cudaStreamSynchronize(m->stream));
        if (h) return SPL_ETIMEOUT;
    }
    return st;
}

extern "C" spl_status_t spl_batch_stationary_learned(spl_mlp_t *m, const spl_pixel_t *h_pixels, int32_t n, double tol,
                                                     int32_t max_iter, float *d_out, const int64_t *d_offsets,
                                                     spl_report_t *h_reports, void *stream,
                                                     const spl_batch_opts_t *opts) {
    if (!m || n < 1 || !h_pixels) return SPL_EINVAL;
    if (stream != static_cast<void *>(m->stream)) return SPL_EINVAL;
    spl_status_t lst = learned_logits(m, h_pixels, n);
    if (lst != SPL_OK) return lst;
    spl_batch_opts_t o{};
    if (opts) o = *opts;
    o.warm_kind = SPL_WARM_LEARNED;
    o.warm_ld = kOutPad;
    if (o.min_iter < 1) o.min_iter = 1;
    o.time_kernel = 1;   // spl_batch_kernel_ms then reports this call's batch kernel
    spl_status_t st = spl_batch_stationary_ex(h_pixels, n, tol, max_iter, m->warm, d_out, d_offsets, h_reports,
                                              stream, &o);
    if (st == SPL_OK || st == SPL_ENOCONV) {
        int h = 0;
        MCU(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
        MCU(cudaStreamSynchronize(m->stream));
        if (h) return SPL_ETIMEOUT;
    }
    return st;
}
