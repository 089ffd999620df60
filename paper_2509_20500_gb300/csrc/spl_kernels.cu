// libspl kernels for sm_103a: cumulative flux (K1), materialised build (K2),
// TMA-staged GEMV power step (K3), matrix-free power step (K4), the
// persistent batch driver (K5) and the per-step finish kernel.
//
// All power steps compute y_j = sum_i pi_i P~_ij with P~ = row-normalised P
// (Sec. 2.3).  Using the factorisation of Eq. 6 (see spl_device.cuh),
//   P~_ij = (u_p / r_i) * w_j * mu(p, j),  p = (i + l) mod N,
// so in "p-space" (k = p_i, i = (k - l) mod N) the step reads
//   y_j = sum_k h_k * w_j * mu(k, j),   h_k = pi_{(k - l) mod N} * u_k / r'_k,
// where r'_k = u_k sum_j w_j mu(k, j) is the row sum of row (k - l) mod N.
// The roll J_l of Sec. 3.4 is therefore only an index rotation when h is
// formed; no permuted copy of anything is made.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spl_device.cuh"
#include "spl_kernels.h"

namespace spl {

// ======================================================================
// Dense triangle passes (the regenerated-matrix inner loops, K4)
// ======================================================================
//
// A thread owns C consecutive outputs a0..a0+C-1 inside a warp span
// [base, base + 32 C).  Over the input index b the triangle weight is
// uniform outside the span, so the loop splits into a "below" region
// b < base, the 32C-wide band and an "above" region b >= base + 32C; only
// the band needs a per-entry select.  Every entry costs one FFMA:
// acc_c += v_b * m_c(b) with the regenerated factor m_c(b).  Sums are
// blocked: four interleaved FFMA chains over a kChain-row chunk, whose sum
// is added into a compensated outer accumulator.

// Tuning knobs of the dense passes (compile-time): chunk length of the
// compensated sums, FFMA chains per output, outputs per thread in the batch
// kernel and its target blocks per SM.
// 64-row chunks: within a chunk every FMA rounds a chain's running sum, so
// the terms that follow a large one (the tails of a concentrated h after the
// pulse rows) each cost half an ulp of that large sum.  Restarting the chains
// every 64 rows keeps the FP32 fixed point of bright narrow pulses within
// about 1e-7 L1 of the exact pmf (the 24 brightest array pixels: 1.7e-7 with
// 64 rows, 4.7e-7 with 128, up to 1.1e-6 with 256).
#ifndef SPL_KCHAIN
#define SPL_KCHAIN 64
#endif
#ifndef SPL_NCH
#define SPL_NCH 4
#endif
#ifndef SPL_BATCH_C
#define SPL_BATCH_C 8
#endif
#ifndef SPL_BATCH_MINB
#define SPL_BATCH_MINB 2
#endif
// 1: issue the four FFMA chains of a column as two packed FP32x2 FMAs
// (fma.rn.f32x2, sm_100+), same per-lane rounding, half the instructions.
#ifndef SPL_FFMA2
#define SPL_FFMA2 1
#endif
// Unroll depth of the uniform-weight loop (float4 steps); deeper hides more
// shared-memory latency, shallower keeps the hot code small.  Measured on the
// 65536-pixel array (plain start, batch kernel): 1: 82.0, 2: 77.8, 3: 72.8,
// 4: 69.8, 6: 74.6, 8: 72.2, 16: 71.8 ms.
#ifndef SPL_TRI_UNROLL
#define SPL_TRI_UNROLL 4
#endif
constexpr int kTriUnroll = SPL_TRI_UNROLL;
// The same for the single- and multi-chain kernels, whose pass pieces are
// inlined one after the other (kOneCopy false) with 64-row chunks (12-chain
// N = 10000 sweep: 4: 0.547, 8: 0.537, 16: 0.605 ms).
#ifndef SPL_TRI_UNROLL_CHAIN
#define SPL_TRI_UNROLL_CHAIN 8
#endif
constexpr int kTriUnrollChain = SPL_TRI_UNROLL_CHAIN;
constexpr int kChain = SPL_KCHAIN;
// Chunk length where the summed vector is spread out (the row pass, and
// column passes whose iterate has sum_j pi_j^2 <= kFineIpr): there 256-row
// chunks stay at the accuracy of 64-row ones (measured on 4096 array pixels:
// FP32 fixed point within 2.1e-7 L1 below the threshold, up to 1.0e-6 above
// it), at a quarter of the flushes.
constexpr int kChainCoarse = 256;
constexpr float kFineIpr = 0.01f;
constexpr int kNch = SPL_NCH;

// Compensated accumulation of a chunk sum x into (acc, comp) by Dekker's
// Fast2Sum: the rounding error of acc + x is x - (s - acc), exact while
// |acc| >= |x| (the usual case once a few chunks are in; otherwise a close
// estimate), three operations instead of TwoSum's six.
__device__ __forceinline__ void fast_two_sum_acc(float &acc, float &comp, float x) {
    const float s = acc + x;
    comp += x - (s - acc);
    acc = s;
}

// Compensated accumulation of a positive chunk sum x into (acc, comp):
// TwoSum gives the exact rounding error of acc + x, which is carried in comp.
__device__ __forceinline__ void two_sum_acc(float &acc, float &comp, float x) {
    const float s = acc + x;
    const float bb = s - acc;
    const float e = (acc - (s - bb)) + (x - bb);
    acc = s;
    comp += e;
}

template <int C>
__device__ __forceinline__ void chains_zero(float (&in)[kNch][C]) {
#pragma unroll
    for (int h = 0; h < kNch; ++h)
#pragma unroll
        for (int c = 0; c < C; ++c) in[h][c] = 0.f;
}

template <int C>
__device__ __forceinline__ void chains_flush(float (&in)[kNch][C], float (&acc)[C], float (&comp)[C]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float t;
        if (kNch == 4) t = (in[0][c] + in[1][c]) + (in[2][c] + in[3][c]);
        else if (kNch == 2) t = in[0][c] + in[1][c];
        else t = in[0][c];
        fast_two_sum_acc(acc[c], comp[c], t);
    }
}

// Uniform-weight run over b in [lo, hi) (multiples of 4).  Each chunk of kc
// rows (the template default KC, or a runtime value so that one copy of the
// code serves several chunk lengths) is summed in kNch interleaved FFMA
// chains (float4 lane e feeds chain e % kNch), which are then added into the
// compensated outer accumulator: relative rounding error per output about
// one FP32 unit roundoff instead of ~15 for one sequential 2000-term chain.
template <int C, int KC = kChain, int UNR = kTriUnroll>
__device__ __forceinline__ void tri_run(const float *__restrict__ v, int lo, int hi, const float (&m)[C],
                                        float (&acc)[C], float (&comp)[C], int kc = KC) {
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
#if SPL_FFMA2
    static_assert(kNch == 4, "packed form keeps four chains per output");
    float2 mm[C];
#pragma unroll
    for (int c = 0; c < C; ++c) mm[c] = make_float2(m[c], m[c]);
    for (int b0 = lo; b0 < hi; b0 += kc) {
        const int q1 = (min(hi, b0 + kc) - b0) >> 2;
        float2 in01[C], in23[C];
#pragma unroll
        for (int c = 0; c < C; ++c) { in01[c] = make_float2(0.f, 0.f); in23[c] = make_float2(0.f, 0.f); }
#pragma unroll UNR
        for (int q = 0; q < q1; ++q) {
            const float4 x = v4[(b0 >> 2) + q];
            const float2 xa = make_float2(x.x, x.y), xb = make_float2(x.z, x.w);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                in01[c] = __ffma2_rn(xa, mm[c], in01[c]);
                in23[c] = __ffma2_rn(xb, mm[c], in23[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c)
            fast_two_sum_acc(acc[c], comp[c], (in01[c].x + in01[c].y) + (in23[c].x + in23[c].y));
    }
#else
    for (int b0 = lo; b0 < hi; b0 += kc) {
        const int q1 = (min(hi, b0 + kc) - b0) >> 2;
        float in[kNch][C];
        chains_zero<C>(in);
#pragma unroll UNR
        for (int q = 0; q < q1; ++q) {
            const float4 x = v4[(b0 >> 2) + q];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                in[0 % kNch][c] = fmaf(x.x, m[c], in[0 % kNch][c]);
                in[1 % kNch][c] = fmaf(x.y, m[c], in[1 % kNch][c]);
                in[2 % kNch][c] = fmaf(x.z, m[c], in[2 % kNch][c]);
                in[3 % kNch][c] = fmaf(x.w, m[c], in[3 % kNch][c]);
            }
        }
        chains_flush<C>(in, acc, comp);
    }
#endif
}

// Column pass: out_c = sum_b v_b * (b <= a_c ? mlo_c : mhi_c)
//   (power step: v = h, mlo = w_j, mhi = w_j eL).
// Row pass:    out_c = sum_b v_b * (b >= a_c ? mlo_c : mhi_c)
//   (row sums:  v = w, mlo = u_k, mhi = u_k eL).
// The thread owns outputs a_c = base + 32 c + lane (c < C): lane-interleaved
// inside the warp span [base, base + 32 C), so stores and factor loads are
// coalesced and, inside the span, 32-entry block cb is "near" for columns
// c > cb, "far" for c < cb, and needs a per-entry select only for c == cb.
// b runs over [b_lo, b_hi); v is indexed by b (callers offset the pointer
// for a chunk).  All bounds are multiples of 4; the span either starts at or
// after b_lo, or lies fully below it (with kLoCut: b_lo may also fall inside
// the span at a 32-entry block boundary); a span reaching past b_hi is cut at
// a 32-entry block boundary (b_hi a multiple of 32 then).  kc is the chunk
// length (see tri_run).  kOneCopy runs the pieces below, inside and above the
// span as one loop, each one copy of code (the batch kernel, where hot-code
// size matters); otherwise they are inlined one after the other (the
// single-chain kernels, whose warps each see only a few row blocks).
template <int C, bool kRowPass, int KC = kChain, bool kLoCut = false, bool kOneCopy = true>
__device__ __forceinline__ void tri_pass(const float *__restrict__ v, int b_lo, int b_hi, int base, int lane,
                                         const float (&mlo)[C], const float (&mhi)[C], float (&out)[C],
                                         int kc = KC) {
    float acc[C], comp[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { acc[c] = 0.f; comp[c] = 0.f; }
    const int span_end = base + 32 * C;
    // below the span (part 0: b < a for every owned a), the span itself
    // (part 1), above the span (part 2: b > a); one copy of each piece of
    // code, in this order
    auto piece = [&](int part) {
        if (part != 1) {
            const bool below = part == 0;
            float m[C];
#pragma unroll
            for (int c = 0; c < C; ++c) m[c] = (below != kRowPass) ? mlo[c] : mhi[c];
            tri_run<C, KC, kOneCopy ? kTriUnroll : kTriUnrollChain>(v, below ? b_lo : max(b_lo, span_end),
                                                                   below ? min(b_hi, base) : b_hi, m, acc, comp, kc);
            return;
        }
        // the span itself (32 C entries, added as chunks of at most kChain)
        if ((kLoCut ? base + 32 * C > b_lo : base >= b_lo) && base < b_hi) {
            const float4 *v4 = reinterpret_cast<const float4 *>(v);
            float in[kNch][C];
            chains_zero<C>(in);
#pragma unroll
            for (int cb = 0; cb < C; ++cb) {
                // weights of the columns that are uniform over this block
                float m[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const bool near = kRowPass ? (c < cb) : (c > cb);
                    m[c] = near ? mlo[c] : mhi[c];
                }
                // blocks outside [b_lo, b_hi) (only where the span is cut) add nothing
                const bool in_range = base + 32 * cb < b_hi && (!kLoCut || base + 32 * cb >= b_lo);
                // unrolled 2 deep (array, plain start: 1: 70.4, 2: 69.9, 4: 74.0, 8: 80.0 ms)
#pragma unroll 2
                for (int q = 0; q < (in_range ? 8 : 0); ++q) {
                    const float4 x = v4[((base + 32 * cb) >> 2) + q];
                    const int t = 4 * q;   // offset of x.x inside the block
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (c == cb) {
                            // per-entry triangle weight of the owned column
                            const bool n0 = kRowPass ? (t + 0 >= lane) : (t + 0 <= lane);
                            const bool n1 = kRowPass ? (t + 1 >= lane) : (t + 1 <= lane);
                            const bool n2 = kRowPass ? (t + 2 >= lane) : (t + 2 <= lane);
                            const bool n3 = kRowPass ? (t + 3 >= lane) : (t + 3 <= lane);
                            in[0 % kNch][c] = fmaf(x.x, n0 ? mlo[c] : mhi[c], in[0 % kNch][c]);
                            in[1 % kNch][c] = fmaf(x.y, n1 ? mlo[c] : mhi[c], in[1 % kNch][c]);
                            in[2 % kNch][c] = fmaf(x.z, n2 ? mlo[c] : mhi[c], in[2 % kNch][c]);
                            in[3 % kNch][c] = fmaf(x.w, n3 ? mlo[c] : mhi[c], in[3 % kNch][c]);
                        } else {
                            in[0 % kNch][c] = fmaf(x.x, m[c], in[0 % kNch][c]);
                            in[1 % kNch][c] = fmaf(x.y, m[c], in[1 % kNch][c]);
                            in[2 % kNch][c] = fmaf(x.z, m[c], in[2 % kNch][c]);
                            in[3 % kNch][c] = fmaf(x.w, m[c], in[3 % kNch][c]);
                        }
                    }
                }
                if (((cb + 1) * 32) % kc == 0 || cb == C - 1) {
                    chains_flush<C>(in, acc, comp);
                    chains_zero<C>(in);
                }
            }
        }
    };
    if constexpr (kOneCopy) {
#pragma unroll 1
        for (int part = 0; part < 3; ++part) piece(part);
    } else {
        piece(0);
        piece(1);
        piece(2);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) out[c] = acc[c] + comp[c];
}

// Rounds n up to a multiple of the pass chain (and of 32C for the spans).
__host__ __device__ __forceinline__ int pad_len(int n, int C) {
    const int q = 32 * C > kChain ? 32 * C : kChain;
    return (n + q - 1) / q * q;
}

// ======================================================================
// Block-wide scans for the structured (O(N)) power step
// ======================================================================
//
// Inclusive scan of v[0..n) into out[0..n) in tiles of NT*8 consecutive
// elements (thread t holds 8 consecutive ones), carrying the running sum
// between tiles; rev = true scans from the end (suffix sums).  Returns the
// total.  red needs 2 * (NT/32) + 2 floats.
template <int NT>
__device__ float block_scan(const float *v, float *out, int n, bool rev, float *red) {
    constexpr int IT = 8, NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float carry = 0.f;
    for (int t0 = 0; t0 < n; t0 += NT * IT) {
        float x[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = t0 + tid * IT + i;
            x[i] = (e < n) ? v[rev ? n - 1 - e : e] : 0.f;
        }
#pragma unroll
        for (int i = 1; i < IT; ++i) x[i] += x[i - 1];
        float sc = x[IT - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += y;
        }
        float lane_ex = __shfl_up_sync(0xffffffffu, sc, 1);
        if (lane == 0) lane_ex = 0.f;
        if (lane == 31) red[wid] = sc;
        __syncthreads();
        if (wid == 0) {
            float ws = (lane < NW) ? red[lane] : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            float wex = __shfl_up_sync(0xffffffffu, ws, 1);
            if (lane == 0) wex = 0.f;
            if (lane < NW) red[NW + 2 + lane] = wex;
            if (lane == NW - 1) red[NW] = ws;
        }
        __syncthreads();
        const float off = carry + red[NW + 2 + wid] + lane_ex;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int e = t0 + tid * IT + i;
            if (e < n) out[rev ? n - 1 - e : e] = x[i] + off;
        }
        carry += red[NW];
        __syncthreads();
    }
    return carry;
}

// rho_k = 1 / (S_k + eL P_k) for k < n <= 8 NT, from one pass over w: S_k =
// sum_{j >= k} w_j (inclusive suffix) and P_k = sum_{j < k} w_j (exclusive
// prefix), both accumulated outward from their own end (no subtraction from
// the total, which would cancel where the suffix is small).  Thread t holds
// w[8t .. 8t+8); the two thread-level scans run as warp shuffles in opposite
// directions and the warp totals cross one barrier.  red needs 2 NT/32 floats.
template <int NT>
__device__ __forceinline__ void row_rho_scan(const float *w, float *rho, int n, float eL, float *red) {
    constexpr int IT = 8, NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int e0 = tid * IT;
    float x[IT], pe[IT], si[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) x[i] = (e0 + i < n) ? w[e0 + i] : 0.f;
    pe[0] = 0.f;
#pragma unroll
    for (int i = 1; i < IT; ++i) pe[i] = pe[i - 1] + x[i - 1];
    si[IT - 1] = x[IT - 1];
#pragma unroll
    for (int i = IT - 2; i >= 0; --i) si[i] = si[i + 1] + x[i];
    float a = pe[IT - 1] + x[IT - 1], b = si[0];   // the thread's total, summed from each end
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ya = __shfl_up_sync(0xffffffffu, a, o);
        const float yb = __shfl_down_sync(0xffffffffu, b, o);
        if (lane >= o) a += ya;
        if (lane + o < 32) b += yb;
    }
    float ax = __shfl_up_sync(0xffffffffu, a, 1);     // exclusive: lanes before this one
    float bx = __shfl_down_sync(0xffffffffu, b, 1);   // exclusive: lanes after this one
    if (lane == 0) ax = 0.f;
    if (lane == 31) bx = 0.f;
    if (lane == 31) red[wid] = a;
    if (lane == 0) red[NW + wid] = b;
    __syncthreads();
    float wa = 0.f, wb = 0.f;
    for (int q = 0; q < wid; ++q) wa += red[q];
    for (int q = NW - 1; q > wid; --q) wb += red[NW + q];
    const float offa = wa + ax, offb = wb + bx;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int k = e0 + i;
        if (k < n) rho[k] = 1.f / ((si[i] + offb) + eL * (pe[i] + offa));
    }
}

// ======================================================================
// K5: persistent batch driver with the per-CTA matrix-free step
// ======================================================================
//
// One CTA processes one pixel at a time, taking pixels from an atomic work
// queue (the host orders them by decreasing N); several CTAs share an SM so
// that one pixel's FP64 flux phase and barriers overlap another pixel's
// dense passes.  Per pixel:
//   K1    w_j, u_j (FP64 flux -> FP32 factors), eL, Lambda
//   rows  r'_k by the dense row pass, stored as rho_k = u_k / r'_k
//   start pi = uniform, or normalised warm weights, or softmax of logits
//   loop  h_k = pi_{(k-l) mod N} rho_k;  y = dense column pass;
//         pi' = y / sum(y); step statistics; stop rule
// Shared memory: v (the broadcast vector), pi, rho, and when they fit also
// w, u, y, d1, d2; otherwise those five live in per-CTA global scratch.

// K1 of the batch path.  exp(Lambda/2 - F_j) splits into
//   exp(Lambda/2 - S G_j) * exp(-B (j + 1/2) / N),  G_j = Phi(z_j) - Phi(z_0),
// where the second factor is a geometric sequence taken from two FP64
// tables (64 j-steps and 64-j blocks), so outside the pulse (|z| > 9, where
// G_j is one of two constants) a bin costs two FP64 products instead of an
// FP64 exp; inside the pulse G_j needs an FP64 erfc and the two exponentials
// come from exp_series.  The per-pixel constants (PixelConst) come from
// pixel_const_kernel.

// One thread per pixel: the constants of the work list's pixels.
__global__ void __launch_bounds__(128) pixel_const_kernel(const PixelDev *__restrict__ px, int n,
                                                          PixelConst *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    PixelConst c;
    pixel_const(px[k], c);
    out[k] = c;
}

// Fills the geometric tables of one pixel: t_lo[b] = exp(-beta (b + 1/2)),
// t_hi[a] = exp(-64 beta a), by FP64 products from the pixel's constants.
template <int NT>
__device__ __forceinline__ void fill_geo_tables(const PixelConst &c, double *t_lo, double *t_hi, int nblk) {
    for (int b = threadIdx.x; b < 64; b += NT) t_lo[b] = c.g0 * pow_uint(c.q1, b);
    for (int a = threadIdx.x; a < nblk; a += NT) t_hi[a] = pow_uint(c.q64, a);
}

// Phi(b) - Phi(a) for a <= b, from the side of the distribution where both
// tails are small, so a narrow interval far out keeps its relative accuracy.
__device__ __forceinline__ double cdf_diff(double a, double b) {
    constexpr double k = 0.70710678118654752440;
    if (a >= 0.0) return 0.5 * (erfc(a * k) - erfc(b * k));
    if (b <= 0.0) return 0.5 * (erfc(-b * k) - erfc(-a * k));
    return 1.0 - 0.5 * (erfc(b * k) + erfc(-a * k));
}


// Factors of bin j: two FP64 products outside the pulse; inside it an FP64
// erfc for G_j and two exponentials by exp_series.
__device__ __forceinline__ void batch_flux_bin(const PixelDev &p, const PixelConst &f, const double *t_lo,
                                               const double *t_hi, int j, float &w, float &u, float &lam_f) {
    const double g = t_hi[j >> 6] * t_lo[j & 63];                // exp(-B (j + 1/2) / N)
    if (j < f.j_lo || j > f.j_hi) {
        const double wd = (j < f.j_lo ? f.bgK_lo : f.bgK_hi) * g;
        w = (float)wd;
        lam_f = f.bg_f;
        if (!(f.bg > 0.0)) {
            // no background: lambda_j = w_j = 0 here, and u_j = exp(F_j - Lambda/2)
            // is the side's constant (g = 1 when B = 0)
            u = j < f.j_lo ? f.uK_lo : f.uK_hi;
            return;
        }
        // Row factor u_j = exp(F_j - Lambda/2) = lambda_j / w_j.  It cancels
        // exactly in the row-normalised matrix, so FP32 accuracy is enough.
        u = lam_f / w;
    } else {
        const double s = ((double)j + 0.5) * f.delta;
        const double z = (s - p.tau) * f.inv_sigma;
        const double G = std_cdf(z) - f.Phi0;
        const double lam = p.S * exp_series(-0.5 * z * z) * f.gnorm + f.bg;
        const double wd = lam * exp_series(0.5 * f.Lambda - p.S * G) * g;
        w = (float)wd;
        lam_f = (float)lam;
        u = lam_f / w;
    }
}

// SPL_FLUX_BININT: replaces the point column factors w_j (in w and its copy
// v) by the exact integral of the detection density over bin j instead of
// its midpoint value.  With e_j = exp(Lambda/2 - F_j) = 1 / u_j:
//   pulse bins  w_j = e_j exp(F_j - F_lo) (1 - exp(-m_j)) / Delta,
//               F_j - F_lo the mass of the lower half bin, m_j the bin's mass;
//   tail bins   w_j = w_j(point) 2 sinh(beta/2) / beta  (background only).
// Each thread rewrites the bins it wrote in the flux loop.
template <int NT>
__device__ __forceinline__ void binint_pass(const PixelDev &p, const PixelConst &f, const float *u, float *w,
                                            float *v, int N) {
    for (int j = threadIdx.x; j < N; j += NT) {
        float x;
        if (j < f.j_lo || j > f.j_hi) {
            x = (float)((double)w[j] * f.tail_ratio);
        } else {
            const double z = (((double)j + 0.5) * f.delta - p.tau) * f.inv_sigma;
            const double zl = z - f.half_z;
            const double h_lo = p.S * cdf_diff(zl, z) + 0.5 * f.beta;
            const double m = p.S * cdf_diff(zl, z + f.half_z) + f.beta;
            x = (float)(exp(h_lo) * -expm1(-m) / (f.delta * (double)u[j]));
        }
        w[j] = x;
        v[j] = x;
    }
}

// Blocks per SM of the structured instantiation (no dense loops, few
// registers; array, plain start: 4: 10.2, 5: 9.2, 6: 8.69, 8: 8.72 ms).
#ifndef SPL_STRUCT_MINB
#define SPL_STRUCT_MINB 6
#endif
constexpr int kStructMinBlocks = SPL_STRUCT_MINB;

template <int NT, int C, int LEVEL, bool STRUCT>
__global__ void __launch_bounds__(NT, STRUCT ? kStructMinBlocks : (NT <= 256 ? SPL_BATCH_MINB : 1))
    batch_fused_kernel(BatchArgs a) {
    extern __shared__ float4 smem4[];
    __shared__ float red[8 * (NT / 32) + 8];
    __shared__ int s_item;
    __shared__ float s_scal[4];
    __shared__ double s_tlo[64];

    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // Per-pixel vectors: the broadcast vector v always lives in shared memory;
    // level 2 keeps all eight vectors there, level 1 keeps v, pi, rho, level 0
    // only v (the rest go to this block's slot of global scratch).  Addresses
    // are formed where they are used (index 0 v, 1 pi, 2 rho, 3 w, 4 u, 5 y,
    // 6 d1, 7 d2).
    const int np = a.npad_max;
    constexpr int level = LEVEL;
    float *const smem_f = reinterpret_cast<float *>(smem4);
    float *const gslot = LEVEL == 2 ? nullptr : a.scratch + (size_t)blockIdx.x * (LEVEL == 0 ? 7 : 5) * np;
    auto vec = [&](int idx) -> float * {
        if (LEVEL == 2 || idx == 0 || (LEVEL == 1 && idx <= 2)) return smem_f + (size_t)idx * np;
        if (idx <= 2) return gslot + (size_t)(idx + 4) * np;
        return gslot + (size_t)(idx - 3) * np;
    };
    float *sv = smem_f;
#define spi (vec(1))
#define srho (vec(2))
#define gw (vec(3))
#define gu (vec(4))
#define gy (vec(5))
#define gd1 (vec(6))
#define gd2 (vec(7))
    double *s_thi = reinterpret_cast<double *>(smem_f + (level == 2 ? 8 : (level == 1 ? 3 : 1)) * (size_t)np);

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n) break;
        const PixelDev p = a.px[item];
        const int N = p.N, l = p.l;
        const int64_t off = a.offsets ? a.offsets[p.index] : p.out_off;
        const int npad = pad_len(N, C);
        const int nrow = (N + 31) & ~31;         // rows a pass reads (v is zero in [N, npad))
        const int span = NT * C;                 // outputs per group
        const int ngroups = (N + span - 1) / span;

        // ---- K1: factors (FP64 inside), Lambda, eL
        const PixelConst bf = a.pconst[item];
        fill_geo_tables<NT>(bf, s_tlo, s_thi, (N + 63) >> 6);
        const float eL = bf.eL;
        __syncthreads();
        const bool learned = a.warm != nullptr && a.warm_kind == 2;
        for (int j = tid; j < npad; j += NT) {
            float w = 0.f, u = 0.f, lam = 0.f;
            if (j < N) batch_flux_bin(p, bf, s_tlo, s_thi, j, w, u, lam);
            sv[j] = w;      // broadcast vector of the row pass
            gw[j] = w;
            gu[j] = u;
            if (learned && j < N) spi[j] = logf(lam);   // flux prior of the learned start
        }
        if (a.flux_kind) binint_pass<NT>(p, bf, gu, gw, sv, N);
        __syncthreads();

        // ---- row sums r'_k, rho_k = u_k / r'_k
        if ((STRUCT || a.row_scan) && N <= 8 * NT) {
            // r'_k / u_k = sum_{j >= k} w_j + eL sum_{j < k} w_j in one pass
            row_rho_scan<NT>(gw, srho, N, eL, red);
        } else if (STRUCT || a.row_scan) {
            // the same from an inclusive suffix scan and an inclusive prefix
            // scan of w over several tiles (prefix - w_k is the exclusive
            // prefix, whose rounding is damped by eL)
            block_scan<NT>(gw, gy, N, false, red);      // gy = prefix
            block_scan<NT>(gw, sv, N, true, red);       // sv = suffix
            for (int k = tid; k < N; k += NT) srho[k] = 1.f / (sv[k] + eL * (gy[k] - gw[k]));
            __syncthreads();
        } else {
        for (int g = 0; g < ngroups; ++g) {
            const int base = (g * NW + wid) * 32 * C;
            if (base < N) {
                float mlo[C], mhi[C], r[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int k = base + 32 * c + lane;
                    const float u = (k < N) ? gu[k] : 0.f;
                    mlo[c] = u;
                    mhi[c] = u * eL;
                }
                tri_pass<C, true, kChainCoarse>(sv, 0, nrow, base, lane, mlo, mhi, r);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int k = base + 32 * c + lane;
                    if (k < N) srho[k] = mlo[c] / r[c];
                }
            }
        }
        }

        // ---- a priori bound on |lambda_2|: Dobrushin's ergodicity coefficient
        // tau(P~) <= 1 - sum_j min_k P~_kj.  In p-space row k of P~ is
        // w_j mu(k, j) / R_k, and R_k = 1 / rho_k = sum_{j >= k} w_j +
        // e^-Lambda sum_{j < k} w_j never increases with k, so the column
        // minimum is w_j min(rho_0, e^-Lambda rho_{j+1}) (rho_0 for the last
        // column).  The roll J_l only permutes rows and leaves it unchanged.
        __syncthreads();
        float cmin = 0.f;
        {
            const float r0 = srho[0];
            for (int j = tid; j < N; j += NT) cmin += gw[j] * (j + 1 < N ? fminf(r0, eL * srho[j + 1]) : r0);
        }
        // 1e-6 covers the FP32 rounding of the sum
        const float tau = fminf(1.f, fmaxf(0.f, 1.f - block_sum<NT>(cmin, red)) + 1e-6f);
        __syncthreads();   // every thread has read red[0] before it is reused

        // ---- start vector: uniform, normalised weights, softmax of logits,
        // or the learned start exp(z_{(j - c) mod N} + log lambda_j) / sum.
        float lsum = 0.f;
        if (a.warm == nullptr) {
            for (int j = tid; j < N; j += NT) spi[j] = 1.f / (float)N;
        } else if (a.warm_kind == 0) {
            for (int j = tid; j < N; j += NT) {
                const float x = fmaxf(a.warm[off + j], 0.f);
                spi[j] = x;
                lsum += x;
            }
        } else {
            float mx = -INFINITY;
            if (a.warm_kind == 1) {
                for (int j = tid; j < N; j += NT) {
                    const float e = a.warm[off + j];
                    spi[j] = e;
                    mx = fmaxf(mx, e);
                }
            } else {
                const float *z = a.warm + (size_t)p.index * a.warm_ld;
                const int c = mlp_frame_shift(p.t_r, p.tau, N);
                for (int j = tid; j < N; j += NT) {
                    int i = j - c;
                    i += (i < 0) ? N : 0;
                    const float e = z[i] + spi[j];
                    spi[j] = e;
                    mx = fmaxf(mx, e);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) red[wid] = mx;
            __syncthreads();
            if (tid == 0) {
                float m = red[0];
                for (int w2 = 1; w2 < NW; ++w2) m = fmaxf(m, red[w2]);
                s_scal[0] = m;
            }
            __syncthreads();
            mx = s_scal[0];
            for (int j = tid; j < N; j += NT) {
                const float x = __expf(spi[j] - mx);
                spi[j] = x;
                lsum += x;
            }
        }
        // sum_j pi_j^2 of the start picks the first column pass's chunk length
        bool fine = 1.f / (float)N > kFineIpr;
        if (a.warm != nullptr) {
            const float tot = block_sum<NT>(lsum, red);
            const bool ok = tot > 0.f && isfinite(tot);
            const float inv = ok ? 1.f / tot : 0.f;
            float q2 = 0.f;
            for (int j = tid; j < N; j += NT) {
                const float x = ok ? spi[j] * inv : 1.f / (float)N;
                spi[j] = x;
                q2 = fmaf(x, x, q2);
            }
            fine = block_sum<NT>(q2, red) > kFineIpr;
        }
        for (int j = tid; j < N; j += NT) { gd1[j] = 0.f; gd2[j] = 0.f; }
        __syncthreads();

        // ---- power iteration
        StopState st;
        stop_init(st, tau, a.warm != nullptr ? kWarmRhoFloor : 0.f);
        int status = ST_ENOCONV;
        // h_k = pi_{(k - l) mod N} * rho_k (J_l folded into the index) for the
        // first step; later steps get h from the statistics loop.
        for (int k = tid; k < npad; k += NT) {
            float h = 0.f;
            if (k < N) {
                int i = k - l;
                i += (i < 0) ? N : 0;
                h = spi[i] * srho[k];
            }
            sv[k] = h;
        }
        __syncthreads();
        // reduction scratch: [0, NW) step sums, [NW, 6 NW) step statistics,
        // [6 NW, 8 NW + 2) the structured step's scan; disjoint, so no buffer is
        // rewritten before every thread has read it
        float *redA = red;
        float *redS = red + NW;
        float *redC = red + 6 * NW;
        for (int it = 0; it < a.max_iter; ++it) {
            float ysum = 0.f;
            if constexpr (STRUCT) {
                // y_j = w_j (P_j + eL (T - P_j)), P = inclusive prefix of h, T = sum h
                const float T = block_scan<NT>(sv, gy, N, false, redC);
                for (int j = tid; j < N; j += NT) {
                    const float P = gy[j];
                    const float y = gw[j] * fmaf(eL, T - P, P);
                    gy[j] = y;
                    ysum += y;
                }
            } else {
            for (int g = 0; g < ngroups; ++g) {
                const int base = (g * NW + wid) * 32 * C;
                if (base < N) {
                    float mlo[C], mhi[C], y[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const int j = base + 32 * c + lane;
                        const float w = (j < N) ? gw[j] : 0.f;
                        mlo[c] = w;
                        mhi[c] = w * eL;
                    }
                    // one code path for both chunk lengths (only the outer step differs);
                    // h is zero from N on, so a warp whose columns end below N stops at
                    // N rounded up to 4 (the same sums bit for bit); the warp whose span
                    // holds column N runs to the 32-row block boundary its span needs
                    const int bhi = base + 32 * C <= N ? ((N + 3) & ~3) : nrow;
                    tri_pass<C, false>(sv, 0, bhi, base, lane, mlo, mhi, y, fine ? kChain : kChainCoarse);
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const int j = base + 32 * c + lane;
                        if (j < N) { gy[j] = y[c]; ysum += y[c]; }
                    }
                }
            }
            }
            // one barrier: orders the y writes and ends every read of h
            const float s = block_sum_1bar<NT>(ysum, redA);
            const float inv = 1.f / s;
            float stats[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (int j = tid; j < N; j += NT) {
                const float pn = gy[j] * inv;
                const float d = pn - spi[j];
                const float e1 = gd1[j], e2 = gd2[j];
                stats[0] += fabsf(d);
                stats[1] = fmaf(d, d, stats[1]);
                stats[2] = fmaf(d, e1, stats[2]);
                stats[3] = fmaf(d, e2, stats[3]);
                stats[4] = fmaf(pn, pn, stats[4]);
                gd2[j] = e1;
                gd1[j] = d;
                spi[j] = pn;
                // next step's broadcast vector: h at k = (j + l) mod N
                int k = j + l;
                k -= (k >= N) ? N : 0;
                sv[k] = pn * srho[k];
            }
            // one barrier: orders pi, d and h before the next step
            block_sum_k_1bar<NT, 5>(stats, redS);
            fine = stats[4] > kFineIpr;
            const int su = stop_update(st, stats[0], stats[1], stats[2], stats[3], a.tol_err, a.min_iter);
            if (su != STOP_CONTINUE) {
                status = su == STOP_CONVERGED ? ST_OK : ST_ENOCONV;
                break;
            }
        }
        __syncthreads();
        // ---- output
        for (int j = tid; j < N; j += NT) a.out[off + j] = spi[j];
        if (tid == 0 && a.reports) {
            ReportDev r;
            r.iters = st.k;
            r.status = status;
            r.last_step_l1 = st.delta[(st.k + 7) & 7];
            r.err_bound = st.err;
            r.lambda2_abs = st.rho;
            r.lambda2_phase = st.theta;
            a.reports[p.index] = r;
        }
        __syncthreads();
        // host-buffer calls: the pixel's range gains one finished pixel, after
        // every thread's output write (the host copies a range once its count
        // is full)
        if (a.range_done != nullptr && tid == 0) {
            __threadfence();
            atomicAdd(a.range_done + (int)(((long long)(p.index + 1) * a.nranges - 1) / a.range_n), 1);
        }
    }
}

#undef spi
#undef srho
#undef gw
#undef gu
#undef gy
#undef gd1
#undef gd2


// ======================================================================
// K8: spectral analysis (|lambda_2| and its phase, Sec. 4)
// ======================================================================
//
// One block per pixel.  After the flux factors and row sums (structured
// form), pi is found by power iteration, then the subdominant eigenvalues
// of P~ by orthogonal iteration on two vectors deflated against pi:
//   Y = X P~ - (X P~ 1) pi      (P~ 1 = 1, pi 1 = 1: removes the lambda = 1 part)
//   H_ab = <y_a, x_b>           (2 x 2 projection; its eigenvalues tend to the
//                                two largest-modulus eigenvalues below 1,
//                                a complex pair or two real ones)
//   X = orthonormalise(Y)
// Every product x P~ uses the O(N) structured form of Eq. 6.  Results:
// out[2k] = |lambda_2|, out[2k+1] = |arg lambda_2| of pixel k.

// y = x P~ in the structured form (x indexed by row i, y by column j).
template <int NT>
__device__ __forceinline__ float apply_structured(const float *x, const float *rho, const float *w, float eL, int N,
                                                  int l, float *hbuf, float *y, float *red) {
    for (int k = threadIdx.x; k < N; k += NT) {
        int i = k - l;
        i += (i < 0) ? N : 0;
        hbuf[k] = x[i] * rho[k];
    }
    __syncthreads();
    const float T = block_scan<NT>(hbuf, y, N, false, red);
    float sy = 0.f;
    for (int j = threadIdx.x; j < N; j += NT) {
        const float P = y[j];
        const float v = w[j] * fmaf(eL, T - P, P);
        y[j] = v;
        sy += v;
    }
    return sy;   // per-thread partial sum of y
}

template <int NT>
__global__ void __launch_bounds__(NT) spectral_kernel(SpectralArgs a) {
    extern __shared__ float4 smem4[];
    constexpr int NW = NT / 32;
    // reduction scratch: two alternating buffers of 4 NW (one-barrier
    // reductions never reuse the buffer of the reduction just before), and
    // the scan's own region
    __shared__ float red[10 * NW + 8];
    __shared__ double s_tlo[64];
    const int np = a.npad_max;
    float *base = reinterpret_cast<float *>(smem4);
    float *w = base, *rho = base + np, *pi = base + 2 * np, *x = base + 3 * np, *z = base + 4 * np;
    float *y1 = base + 5 * np, *y2 = base + 6 * np, *hb = base + 7 * np;
    double *s_thi = reinterpret_cast<double *>(base + 8 * (size_t)np);
    float *redC = red + 8 * NW;
    bool flip = false;
    auto buf = [&]() -> float * { flip = !flip; return flip ? red : red + 4 * NW; };
    const int tid = threadIdx.x;

    for (int item = blockIdx.x; item < a.n; item += gridDim.x) {
        const PixelDev p = a.px[item];
        const int N = p.N, l = p.l;
        const PixelConst bf = a.pconst[item];
        fill_geo_tables<NT>(bf, s_tlo, s_thi, (N + 63) >> 6);
        const float eL = bf.eL;
        __syncthreads();
        for (int j = tid; j < N; j += NT) {
            float wj, uj, lam;
            batch_flux_bin(p, bf, s_tlo, s_thi, j, wj, uj, lam);
            w[j] = wj;
        }
        __syncthreads();
        block_scan<NT>(w, y1, N, false, redC);       // prefix
        block_scan<NT>(w, y2, N, true, redC);        // suffix
        for (int k = tid; k < N; k += NT) rho[k] = 1.f / (y2[k] + eL * (y1[k] - w[k]));
        for (int j = tid; j < N; j += NT) pi[j] = 1.f / (float)N;
        __syncthreads();
        // pi by power iteration (structured step) to a small step
        for (int it = 0; it < a.pi_iters; ++it) {
            const float sy = block_sum_1bar<NT>(apply_structured<NT>(pi, rho, w, eL, N, l, hb, y1, redC), buf());
            float dl = 0.f;
            for (int j = tid; j < N; j += NT) {
                const float pn = y1[j] / sy;
                dl += fabsf(pn - pi[j]);
                pi[j] = pn;
            }
            const float delta = block_sum_1bar<NT>(dl, buf());
            if (delta < 1e-7f) break;
        }
        // deterministic start vectors (hashed from bin and pixel index)
        for (int j = tid; j < N; j += NT) {
            uint32_t hx = (uint32_t)j * 2654435761u ^ (uint32_t)(p.index + 1) * 2246822519u;
            hx ^= hx >> 15;
            hx *= 2246822519u;
            hx ^= hx >> 13;
            uint32_t hz = hx * 3266489917u + 374761393u;
            hz ^= hz >> 16;
            x[j] = (float)(hx & 0xFFFFFF) / 16777216.f - 0.5f;
            z[j] = (float)(hz & 0xFFFFFF) / 16777216.f - 0.5f;
        }
        __syncthreads();
        float H[4] = {0.f, 0.f, 0.f, 0.f};
        for (int m = 0; m <= a.subspace_iters; ++m) {
            // (1) deflate against pi and orthonormalise x, z (Gram-Schmidt)
            float sxz[2] = {0.f, 0.f};
            for (int j = tid; j < N; j += NT) { sxz[0] += x[j]; sxz[1] += z[j]; }
            block_sum_k_1bar<NT, 2>(sxz, buf());
            float nx = 0.f;
            for (int j = tid; j < N; j += NT) {
                const float v = x[j] - sxz[0] * pi[j];
                x[j] = v;
                z[j] = z[j] - sxz[1] * pi[j];
                nx = fmaf(v, v, nx);
            }
            nx = block_sum_1bar<NT>(nx, buf());
            const float ix = nx > 0.f ? rsqrtf(nx) : 0.f;
            float dxz = 0.f;
            for (int j = tid; j < N; j += NT) {
                x[j] *= ix;
                dxz = fmaf(x[j], z[j], dxz);
            }
            dxz = block_sum_1bar<NT>(dxz, buf());
            float nz = 0.f;
            for (int j = tid; j < N; j += NT) {
                const float v = z[j] - dxz * x[j];
                z[j] = v;
                nz = fmaf(v, v, nz);
            }
            nz = block_sum_1bar<NT>(nz, buf());
            const float iz = nz > 0.f ? rsqrtf(nz) : 0.f;
            for (int j = tid; j < N; j += NT) z[j] *= iz;
            __syncthreads();
            if (m == a.subspace_iters) break;
            // (2) Y = X P~ deflated, (3) projection H_ab = <y_a, x_b>
            const float s1 = block_sum_1bar<NT>(apply_structured<NT>(x, rho, w, eL, N, l, hb, y1, redC), buf());
            const float s2 = block_sum_1bar<NT>(apply_structured<NT>(z, rho, w, eL, N, l, hb, y2, redC), buf());
            float hh[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j = tid; j < N; j += NT) {
                const float a1 = y1[j] - s1 * pi[j], a2 = y2[j] - s2 * pi[j];
                hh[0] = fmaf(a1, x[j], hh[0]);
                hh[1] = fmaf(a1, z[j], hh[1]);
                hh[2] = fmaf(a2, x[j], hh[2]);
                hh[3] = fmaf(a2, z[j], hh[3]);
                x[j] = a1;
                z[j] = a2;
            }
            block_sum_k_1bar<NT, 4>(hh, buf());
#pragma unroll
            for (int q = 0; q < 4; ++q) H[q] = hh[q];
        }
        if (tid == 0) {
            // eigenvalues of the projection (x -> H0 x + H1 z, z -> H2 x + H3 z)
            const double tr = (double)H[0] + H[3];
            const double det = (double)H[0] * H[3] - (double)H[1] * H[2];
            const double disc = tr * tr - 4.0 * det;
            double mod, ph;
            if (disc < 0.0) {
                mod = sqrt(fmax(det, 0.0));
                ph = atan2(sqrt(-disc), tr);
            } else {
                const double r1 = 0.5 * (tr + sqrt(disc)), r2 = 0.5 * (tr - sqrt(disc));
                const double r = fabs(r1) >= fabs(r2) ? r1 : r2;
                mod = fabs(r);
                ph = r >= 0.0 ? 0.0 : 3.14159265358979323846;
            }
            a.out[2 * (size_t)p.index] = (float)mod;
            a.out[2 * (size_t)p.index + 1] = (float)ph;
        }
        __syncthreads();
    }
}

size_t spectral_smem_bytes(int npad) { return (size_t)8 * npad * sizeof(float) + (size_t)(npad / 64 + 2) * 8; }

cudaError_t launch_spectral(const SpectralArgs &a, int grid, cudaStream_t s) {
    auto k = spectral_kernel<256>;
    const size_t smem = spectral_smem_bytes(a.npad_max);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = launch_pixel_const(a.px, a.n, a.pconst, s)) != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

// ======================================================================
// K1 for a single chain: per-bin vectors
// ======================================================================

__global__ void chain_flux_kernel(PixelDev p, float *__restrict__ w, float *__restrict__ u,
                                  float *__restrict__ lam_out, double *__restrict__ F_out,
                                  double *__restrict__ scal /* [0]=Lambda [1]=eL */, int npad) {
    const FluxConst fc = flux_const(p);
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < npad; j += stride) {
        if (j < p.N) {
            double F, lam;
            flux_bin(p, fc, j, F, lam);
            const double e = exp(0.5 * fc.Lambda - F);
            w[j] = (float)(lam * e);
            u[j] = (float)(1.0 / e);
            if (lam_out) lam_out[j] = (float)lam;
            if (F_out) F_out[j] = F;
        } else {
            w[j] = 0.f;
            u[j] = 0.f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[0] = fc.Lambda;
        scal[1] = exp(-fc.Lambda);
    }
}

// ======================================================================
// K2: materialised build with the roll in the row address
// ======================================================================
//
// One warp per row i (grid-stride).  p = (i + l) mod N selects the row
// factor u_p: row i of E = J_l E_base is row p of E_base, read in place.
// P_ij = u_p * w_j * (p > j ? eL : 1) with 16-byte stores; the row sum is
// accumulated in 128-term chains and warp-reduced.

__global__ void __launch_bounds__(256) build_matrix_kernel(int N, int l, int ld, const float *__restrict__ w,
                                                           const float *__restrict__ u,
                                                           const double *__restrict__ scal,
                                                           float *__restrict__ P, float *__restrict__ rowsum) {
    const float eL = (float)scal[1];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const bool vec = (N & 3) == 0;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += warps) {
        int p = i + l;
        p -= (p >= N) ? N : 0;
        const float up = u[p];
        const float upe = up * eL;
        float *row = P + (size_t)i * ld;
        float acc = 0.f, comp = 0.f, in = 0.f;
        int cnt = 0;
        if (vec) {
            const float4 *w4 = reinterpret_cast<const float4 *>(w);
            float4 *r4 = reinterpret_cast<float4 *>(row);
            for (int q = lane; q < (N >> 2); q += 32) {
                const float4 x = w4[q];
                const int j = q << 2;
                float4 o;
                o.x = x.x * ((p > j) ? upe : up);
                o.y = x.y * ((p > j + 1) ? upe : up);
                o.z = x.z * ((p > j + 2) ? upe : up);
                o.w = x.w * ((p > j + 3) ? upe : up);
                __stcs(r4 + q, o);
                in += (o.x + o.y) + (o.z + o.w);
                if (++cnt == kChain / 4) { two_sum_acc(acc, comp, in); in = 0.f; cnt = 0; }
            }
        } else {
            for (int j = lane; j < N; j += 32) {
                const float o = w[j] * ((p > j) ? upe : up);
                __stcs(row + j, o);
                in += o;
                if (++cnt == kChain) { two_sum_acc(acc, comp, in); in = 0.f; cnt = 0; }
            }
        }
        two_sum_acc(acc, comp, in);
        acc += comp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) rowsum[i] = acc;
    }
}

// ======================================================================
// K3: TMA-staged GEMV over the materialised P (HBM-bound)
// ======================================================================
//
// Work unit = one 32-row x 128-column tile (16 KB).  Tiles are numbered
// slab-major (slab = 128 columns) and each CTA takes one contiguous range of
// tiles, so every CTA streams the same number of bytes.  A single thread
// issues cp.async.bulk.tensor.2d loads into a ring of STAGES shared-memory
// buffers, each guarded by an mbarrier with an expected transaction count;
// the 128 threads of the CTA each own one column of the slab and accumulate
// c_i * P_ij down the rows (c_i = pi_i / r_i), in 32-term chains per tile.
// A CTA's range spans at most two slabs; the partial column sums of each are
// written to part[cta][slot][128] and reduced in fixed order by the finish
// kernel (deterministic, no atomics).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

#ifndef SPL_GEMV_COLS
#define SPL_GEMV_COLS 256
#endif
#ifndef SPL_GEMV_STAGES
#define SPL_GEMV_STAGES 4
#endif
constexpr int kGemvCols = SPL_GEMV_COLS;     // slab width (columns per TMA box)
constexpr int kGemvRows = 32;
constexpr int kGemvTileBytes = kGemvCols * kGemvRows * 4;
constexpr int kGemvThreads = 256;
constexpr int kGemvCG = kGemvCols / 4;       // column groups of 4 (one float4)
constexpr int kGemvRG = kGemvThreads / kGemvCG;
constexpr int kGemvRowsPerThread = kGemvRows / kGemvRG;
constexpr int kGemvMaxSmemC = 16384;   // row coefficients staged in shared memory up to this N

// 256 threads per CTA: thread (rg, cg) owns columns 4cg..4cg+3 of the slab and
// rows rg*R .. rg*R+R-1 of every 32-row tile (R = rows per thread), so each
// tile is read from shared memory with 16-byte loads.  The row coefficients
// c_i are staged in shared memory once (when N <= 16384).  Per-thread partial
// sums use TwoSum compensation across tiles; the row groups are combined in
// shared memory when the slab changes and at the end.
template <int STAGES, bool kSmemC>
__global__ void __launch_bounds__(kGemvThreads) gemv_tma_kernel(const __grid_constant__ CUtensorMap tmap, GemvArgs a) {
    extern __shared__ __align__(1024) uint8_t gsm[];
    uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
    float *cs = reinterpret_cast<float *>(tiles + (size_t)STAGES * kGemvTileBytes);
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ float red[kGemvRG][kGemvCols];
    if (a.state && a.state->done) return;

    const int tid = threadIdx.x;
    const int cg = tid % kGemvCG, rg = tid / kGemvCG;
    const int per = a.tiles_per_cta;
    const int t0 = blockIdx.x * per;
    const int t1 = min(a.total_tiles, t0 + per);
    const int ntiles = t1 - t0;
    if (ntiles <= 0) return;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int it) {
        const int t = t0 + it;
        const int slab = t / a.tiles_per_slab;
        const int rt = t - slab * a.tiles_per_slab;
        const int s = it % STAGES;
        mbar_expect_tx(&full[s], kGemvTileBytes);
        tma_load_2d(tiles + (size_t)s * kGemvTileBytes, &tmap, &full[s], slab * kGemvCols, rt * kGemvRows);
    };
    if (tid == 0) {
        for (int it = 0; it < STAGES && it < ntiles; ++it) issue(it);
    }
    if (kSmemC) {
        // stage the coefficients with many independent loads in flight
        const int rows = a.tiles_per_slab * kGemvRows;
#pragma unroll 8
        for (int i = tid; i < rows; i += kGemvThreads) cs[i] = (i < a.N) ? __ldg(a.c + i) : 0.f;
        __syncthreads();
    }
    const int slab0 = t0 / a.tiles_per_slab;
    int cur_slab = slab0;
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
    auto flush = [&](int slab) {
        // combine the 8 row groups of this slab's partial column sums
#pragma unroll
        for (int q = 0; q < 4; ++q) red[rg][4 * cg + q] = acc[q] + comp[q];
        __syncthreads();
        for (int col = tid; col < kGemvCols; col += kGemvThreads) {
            float y = 0.f;
#pragma unroll
            for (int r = 0; r < kGemvRG; ++r) y += red[r][col];
            a.part[((size_t)blockIdx.x * 2 + (slab - slab0)) * kGemvCols + col] = y;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) { acc[q] = 0.f; comp[q] = 0.f; }
    };
    bool timed_out = false;
    int it = 0;
    for (; it < ntiles; ++it) {
        const int s = it % STAGES;
        const uint32_t parity = (uint32_t)((it / STAGES) & 1);
        const int t = t0 + it;
        const int slab = t / a.tiles_per_slab;
        const int rt = t - slab * a.tiles_per_slab;
        if (slab != cur_slab) {
            flush(cur_slab);
            cur_slab = slab;
        }
        if (!mbar_wait(&full[s], parity)) { timed_out = true; }
        if (__syncthreads_or(timed_out)) { timed_out = true; break; }
        const float4 *tile = reinterpret_cast<const float4 *>(tiles + (size_t)s * kGemvTileBytes);
        const int r0 = rt * kGemvRows + kGemvRowsPerThread * rg;
        float in[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < kGemvRowsPerThread; ++r) {
            const int i = r0 + r;
            const float c = kSmemC ? cs[i] : ((i < a.N) ? __ldg(a.c + i) : 0.f);
            const float4 x = tile[(kGemvRowsPerThread * rg + r) * (kGemvCols / 4) + cg];
            in[0] = fmaf(c, x.x, in[0]);
            in[1] = fmaf(c, x.y, in[1]);
            in[2] = fmaf(c, x.z, in[2]);
            in[3] = fmaf(c, x.w, in[3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) two_sum_acc(acc[q], comp[q], in[q]);
        __syncthreads();   // every thread is done with buffer s
        if (tid == 0 && it + STAGES < ntiles) issue(it + STAGES);
    }
    if (timed_out) {
        if (tid == 0) {
            atomicExch(a.err_flag, 1);
            // drain copies still in flight into this CTA's buffers (bounded)
            const int issued = min(ntiles, it + STAGES);
            for (int k = it; k < issued; ++k) mbar_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1));
        }
        __syncthreads();
        return;
    }
    flush(cur_slab);
}

// ======================================================================
// K4 for one large chain: column pass split over CTAs
// ======================================================================
//
// Grid (column tiles) x (b-chunks).  Each CTA copies its chunk of the
// broadcast vector v into shared memory and runs the dense triangle pass for
// its columns over that chunk only; partial sums go to part[chunk][col].

template <int NT, int C, bool kRowPass>
__global__ void __launch_bounds__(NT) tri_split_kernel(TriSplitArgs a) {
    extern __shared__ float4 smem4[];
    float *sv = reinterpret_cast<float *>(smem4);
    if (a.state && a.state->done) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int cols_per_cta = NT * C;
    const int col0 = blockIdx.x * cols_per_cta;
    const int b0 = blockIdx.y * a.chunk;
    const int b1 = min(a.vlen, b0 + a.chunk);
    const int blen = b1 - b0;                 // multiple of kChain
    for (int b = tid; b < blen; b += NT) sv[b] = a.v[b0 + b];
    __syncthreads();
    const int wbase = col0 + wid * 32 * C;
    if (wbase >= a.N) return;
    const float eL = (float)a.scal[1];
    float mlo[C], mhi[C], out[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = wbase + 32 * c + lane;
        const float m = (col < a.N) ? a.m[col] : 0.f;
        mlo[c] = m;
        mhi[c] = m * eL;
    }
    tri_pass<C, kRowPass, kChain, false, false>(sv - b0, b0, b1, wbase, lane, mlo, mhi, out);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int col = wbase + 32 * c + lane;
        if (col < a.N) a.part[(size_t)blockIdx.y * a.ld_part + col] = out[c];
    }
}

// ======================================================================
// Persistent power iteration of one chain (fused mode)
// ======================================================================
//
// One cooperative launch (all CTAs resident) runs the steps of one chain
// with one grid barrier per step.  The column pass is cut into equal work
// units, (column tile of 256 columns) x (block of 32 rows), in tile-major
// order; CTA b takes the contiguous units [b U / G, (b+1) U / G), which cover
// at most a few tiles.  Per step k:
//   pass        for each tile segment of its units, the CTA stages the rows
//               of the broadcast vector v (scaled by 1/s of the previous
//               step) in shared memory, its warps split the rows and sum the
//               tile's columns over them (the same tile code as the split
//               pass), the warp partials are added in warp order into one
//               partial per (CTA, tile), and the last CTA to finish a tile
//               adds the tile's partials in CTA order into y_j, writes
//               v_{(j+l) mod N} = y_j rho_{(j+l) mod N} for the next pass and
//               the tile sum (y, v and the tile sums alternate buffers);
//   barrier
//   normalise   every CTA adds the tile sums in a fixed order (s) and, for its
//               slice of bins, forms pi^(k) = y / s (alternate buffer) and the
//               step d; its share of the statistics goes to its slot;
//   decide      on step k-1: every CTA adds the statistics of step k-1 in CTA
//               order and runs the stop rule on the same numbers, so all CTAs
//               stop together; pi^(k-1) is then the result.
// The barrier is a counter of arrivals since launch that every CTA polls;
// every wait is bounded: a CTA that gives up sets err_flag and poisons the
// count, which releases every other waiter, and all CTAs return.

constexpr int kRunNT = 256;
constexpr int kRunW = kRunNT / 32;
constexpr int kRunC = 8;
constexpr int kRunTW = 32 * kRunC;                      // columns per tile (one warp span)
constexpr int kRunTP = kRunTW / 32;                     // warp partials of a tile's sum
constexpr int kRunMaxChunk = 8192;                      // rows of v in shared memory at once
constexpr int kBarGen = 32;                             // a barrier's slot is 2 kBarGen words (its own lines)
static_assert(3 * 2 * kBarGen <= kMultiCountWord, "three barriers before the set counters");
constexpr uint32_t kGridSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void red_release_add_gpu(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned cas_release_gpu(unsigned *p, unsigned cmp, unsigned v) {
    unsigned old;
    asm volatile("atom.release.gpu.global.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "l"(p), "r"(cmp), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int add_acq_rel_gpu(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier over the G CTAs of a cooperative launch (b, the CTA's index, is
// kept for the callers' symmetry).  bar[0] counts arrivals since launch; every
// CTA adds one (release) and polls, with relaxed loads and a short sleep, until
// the count reaches (gen + 1) G, then acquires once (fence.acq_rel).  gen is
// the calling CTA's count of barriers passed (thread 0's copy is the one
// used).  A CTA that gives up after `limit` polls sets err_flag and adds
// kBarPoison, which releases every other waiter; a count at or above
// kBarPoison means the grid was aborted (false).
constexpr unsigned kBarPoison = 0x40000000u;

__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned &gen, int *err_flag, int *s_flag, int b,
                                          int G, uint32_t limit = kGridSpinLimit) {
    (void)b;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = (gen + 1u) * (unsigned)G;
        red_release_add_gpu(&bar[0], 1u);
        uint32_t spins = 0;
        unsigned v;
        bool ok = true;
        while ((v = ld_relaxed_gpu(&bar[0])) < target) {
            if (++spins > limit) {
                ok = false;
                break;
            }
            __nanosleep(32);
        }
        fence_acq_rel_gpu();   // acquire the arrivals' writes once, not at every poll
        if (!ok) {
            atomicExch(err_flag, 1);
            atomicAdd(&bar[0], kBarPoison);
        } else if (v >= kBarPoison) {
            ok = false;
        }
        gen += 1u;
        *s_flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

// 16-byte asynchronous global -> shared copies (generic proxy), completed
// per thread by cp_async_wait<n> (all but the newest n groups).
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory"); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// First unit of CTA b, and the CTA that owns unit u.
__device__ __forceinline__ long long run_unit0(int b, long long U, int G) { return (long long)b * U / G; }
__device__ __forceinline__ int run_owner(long long u, long long U, int G) {
    return (int)(((u + 1) * G + U - 1) / U) - 1;
}

// End of a tile segment of one CTA: the warp partials added in warp order.
// A tile the CTA covers whole is finished here (y, v and the tile sum, as in
// run_tile_reduce); a shared tile leaves the CTA's partial in its slot.
// The pass ran on the unnormalised broadcast vector of the previous step; inv
// (1 / sum of its y) normalises the column sums here.  The tile sum is left
// as kRunTP warp partials, tdst[kRunTP t + w].
__device__ __forceinline__ void run_flush(const ChainRunArgs &a, int t, int t_first, int b, bool own_first,
                                          bool own_last, int t_last, const float (&acc)[kRunC],
                                          float (*wred)[kRunTW], float inv, float *ydst, float *vdst,
                                          float *tdst) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, N = a.N;
#pragma unroll
    for (int c = 0; c < kRunC; ++c) wred[wid][32 * c + lane] = acc[c];
    __syncthreads();
    const bool owned = (t != t_first || own_first) && (t != t_last || own_last);
    if (tid < kRunTW) {
        float p = 0.f;
#pragma unroll
        for (int w = 0; w < kRunW; ++w) p += wred[w][tid];
        p *= inv;
        if (!owned) {
            a.part[((size_t)b * a.segs + (t - t_first)) * kRunTW + tid] = p;
        } else {
            const int col = t * kRunTW + tid;
            if (col < N) {
                ydst[col] = p;
                int r = col + a.l;
                r -= (r >= N) ? N : 0;
                vdst[r] = p * __ldg(a.rho + r);
            } else {
                p = 0.f;
            }
            const float ts = warp_sum(p);
            if (lane == 0) tdst[kRunTP * t + wid] = ts;
        }
    }
    __syncthreads();   // wred is reused
}

// Adds the tile's partials in CTA order (CTA bf may have started in an
// earlier tile; every later CTA of the tile starts inside it, slot 0) into
// y_j, writes v_{(j+l) mod N} = y_j rho_{(j+l) mod N} and the tile sum.
__device__ __forceinline__ void run_tile_reduce(const ChainRunArgs &a, int t, long long U, int G, float *ydst,
                                                float *vdst, float *tdst) {
    const int tid = threadIdx.x, N = a.N, RB = a.RB;
    const int bf = run_owner((long long)t * RB, U, G), bl = run_owner((long long)(t + 1) * RB - 1, U, G);
    const int col = t * kRunTW + tid;
    float yv = 0.f;
    if (tid < kRunTW && col < N) {
        int r = col + a.l;
        r -= (r >= N) ? N : 0;
        const float rr = __ldg(a.rho + r);
        const float *pp = a.part + tid;
        yv = __ldcg(pp + ((size_t)bf * a.segs + (t - (int)(run_unit0(bf, U, G) / RB))) * kRunTW);
#pragma unroll 8
        for (int bb = bf + 1; bb <= bl; ++bb) yv += __ldcg(pp + (size_t)bb * a.segs * kRunTW);
        ydst[col] = yv;
        vdst[r] = yv * rr;
    }
    if (tid < kRunTW) {
        const float ts = warp_sum(yv);
        if ((tid & 31) == 0) tdst[kRunTP * t + (tid >> 5)] = ts;
    }
}

// Every power step of one chain on the G CTAs of its group; b is this CTA's
// index in the group.
__device__ __forceinline__ void chain_run_body(const ChainRunArgs &a, const int b, const int G) {
    extern __shared__ float4 smem4[];
    float *sv = reinterpret_cast<float *>(smem4);
    __shared__ float wred[kRunW][kRunTW];
    __shared__ float red[9 * kRunW];                 // [0, 5 W) and [5 W, 9 W): the two step sums
    __shared__ int s_flag;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int N = a.N, T = a.T, RB = a.RB;
    const size_t vlen = (size_t)a.vlen;
    const long long U = (long long)T * RB;
    const long long u0 = run_unit0(b, U, G), u1 = run_unit0(b + 1, U, G);
    const int t_first = (int)(u0 / RB), t_last = (int)((u1 - 1) / RB);
    // tiles this CTA covers whole have no other contributor
    const bool own_first = u0 == (long long)t_first * RB && u1 >= (long long)(t_first + 1) * RB;
    const bool own_last = u1 == (long long)(t_last + 1) * RB && u0 <= (long long)t_last * RB;
    const float eL = (float)a.scal[1];
    ChainState *stp = a.state;
    StopState st = stp->st;                 // every CTA keeps the same copy
    const float tol_err = stp->tol_err;
    const int min_iter = stp->min_iter, max_iter = stp->max_iter;
    unsigned gen = 0u;
    // this CTA's slice of bins for the normalisation
    const int S = (N + G - 1) / G;
    const int j0 = min(N, b * S), j1 = min(N, j0 + S);
    const float *vsrc = a.v0;               // h^(0) = pi^(0)_{(k-l) mod N} rho_k
    float inv = 1.f;
    // windows of this CTA's units, staged as 16-byte async copies into buffer
    // w & 1 (a.chunk rows each, so a window is at most a.chunk / 32 units);
    // unit u holds rows (u mod RB) 32 ... + 31
    const int win_units = a.chunk / 32;
    const int nwin = (int)((u1 - u0 + win_units - 1) / win_units);
    auto stage = [&](int w) {
        const long long wu0 = u0 + (long long)w * win_units, wu1 = min(u1, wu0 + win_units);
        const int off0 = (int)(wu0 % RB);
        const int nq = (int)(wu1 - wu0) * 8;
        float *dst = sv + (w & 1) * a.chunk;
        for (int q = tid; q < nq; q += kRunNT) {
            int o = off0 + (q >> 3);
            o -= (o / RB) * RB;                     // 32-row block inside its tile
            cp_async16(dst + 4 * q, vsrc + 4 * (o * 8 + (q & 7)));
        }
        cp_async_commit();
    };
    stage(0);
    // arrivals expected at the shared first and last tiles, less one
    const int cnt_first = run_owner((long long)(t_first + 1) * RB - 1, U, G) - run_owner((long long)t_first * RB, U, G);
    const int cnt_last = run_owner((long long)(t_last + 1) * RB - 1, U, G) - run_owner((long long)t_last * RB, U, G);
    for (int k = 1;; ++k) {
        float *ydst = a.y + (k & 1) * vlen;
        float *vdst = a.vb + (k & 1) * vlen;
        float *tdst = a.tsum + (size_t)(k & 1) * kRunTP * T;
        // ---- pass k, in windows of at most kRunMaxChunk rows staged in unit order
        // into two shared buffers: window w + 1 is in flight while w is summed
        // (window 0 was issued before the previous step's normalisation)
        int cur_t = t_first;
        float mlo[kRunC], mhi[kRunC], acc[kRunC];
        // the first tile's column factors load with the staging
#pragma unroll
        for (int c = 0; c < kRunC; ++c) {
            const int col = t_first * kRunTW + 32 * c + lane;
            const float m = col < N ? __ldg(a.w + col) : 0.f;
            mlo[c] = m;
            mhi[c] = m * eL;
            acc[c] = 0.f;
        }
        for (int w = 0; w < nwin; ++w) {
            if (w + 1 < nwin) {
                stage(w + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const long long wu0 = u0 + (long long)w * win_units, wu1 = min(u1, wu0 + win_units);
            const int tw0 = (int)(wu0 / RB);
            const float *wbuf = sv + (w & 1) * a.chunk;
            for (int t = tw0; (long long)t * RB < wu1; ++t) {
                const long long su0 = max(wu0, (long long)t * RB), su1 = min(wu1, (long long)(t + 1) * RB);
                if (t != cur_t) {
                    run_flush(a, cur_t, t_first, b, own_first, own_last, t_last, acc, wred, inv, ydst, vdst, tdst);
#pragma unroll
                    for (int c = 0; c < kRunC; ++c) {
                        const int col = t * kRunTW + 32 * c + lane;
                        const float m = col < N ? __ldg(a.w + col) : 0.f;
                        mlo[c] = m;
                        mhi[c] = m * eL;
                        acc[c] = 0.f;
                    }
                    cur_t = t;
                }
                // warp wid takes 32-row blocks [wb0, wb1) of the segment
                const int rb0 = (int)(su0 - (long long)t * RB), rb1 = (int)(su1 - (long long)t * RB);
                const int nb = rb1 - rb0;
                const int wb0 = rb0 + (nb * wid) / kRunW, wb1 = rb0 + (nb * (wid + 1)) / kRunW;
                if (wb1 > wb0) {
                    const float *vt = wbuf + ((long long)t * RB - wu0) * 32;   // row r of tile t at vt[r]
                    float out[kRunC];
                    tri_pass<kRunC, false, kChain, true, false>(vt, 32 * wb0, 32 * wb1, t * kRunTW, lane, mlo, mhi,
                                                               out);
#pragma unroll
                    for (int c = 0; c < kRunC; ++c) acc[c] += out[c];
                }
            }
            __syncthreads();   // this buffer is restaged two windows later
        }
        run_flush(a, cur_t, t_first, b, own_first, own_last, t_last, acc, wred, inv, ydst, vdst, tdst);
        // shared tiles: the last CTA to finish one adds its partials
        __syncthreads();
        if (tid == 0) {
            int old0 = -1, old1 = -1;
            __threadfence();
            if (!own_first) old0 = atomicAdd(a.tile_ticket + t_first, 1);
            if (t_last != t_first && !own_last) old1 = atomicAdd(a.tile_ticket + t_last, 1);
            const bool last0 = old0 >= 0 && old0 == cnt_first;
            const bool last1 = old1 >= 0 && old1 == cnt_last;
            if (last0) a.tile_ticket[t_first] = 0;
            if (last1) a.tile_ticket[t_last] = 0;
            if (last0 || last1) __threadfence();
            s_flag = (last0 ? 1 : 0) | (last1 ? 2 : 0);
        }
        __syncthreads();
        const int lastmask = s_flag;
        if (lastmask & 1) run_tile_reduce(a, t_first, U, G, ydst, vdst, tdst);
        if (lastmask & 2) run_tile_reduce(a, t_last, U, G, ydst, vdst, tdst);
        if (!grid_sync(a.bar, gen, a.err_flag, &s_flag, b, G)) {
            if (b == 0) {
                stp->st = st;
                stp->done = 1;
                stp->status = ST_ENOCONV;
            }
            return;
        }
        // every h of step k is written: the next pass's first window is staged
        // while this step is normalised
        vsrc = vdst;
        stage(0);
        // ---- normalise step k, and decide on step k-1
        float *pcur = (k & 1) ? a.pi_alt : a.pi;
        const float *pprev = (k & 1) ? a.pi : a.pi_alt;
        // every load first: statistics of step k-1, tile sums, own bins
        float red5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (k >= 2) {
            const float4 *bs = reinterpret_cast<const float4 *>(a.blk + (size_t)((k - 1) & 1) * G * 4);
            // G is at most 2 kRunNT (two CTAs per SM): both loads in flight
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 x0 = tid < G ? __ldcg(bs + tid) : z;
            const float4 x1 = tid + kRunNT < G ? __ldcg(bs + tid + kRunNT) : z;
            red5[0] = x0.x + x1.x;
            red5[1] = x0.y + x1.y;
            red5[2] = x0.z + x1.z;
            red5[3] = x0.w + x1.w;
        }
        for (int t = tid; t < kRunTP * T; t += kRunNT) red5[4] += __ldcg(tdst + t);
        const int jf = j0 + tid;
        float fy = 0.f, fp = 0.f, f1 = 0.f, f2 = 0.f;
        if (jf < j1) {
            fy = __ldcg(ydst + jf);
            fp = pprev[jf];
            f1 = a.d1[jf];
            f2 = a.d2[jf];
        }
        block_sum_k_1bar<kRunNT, 5>(red5, red);
        inv = 1.f / red5[4];
        if (tid == 0) {
            int fin = 0;
            if (k >= 2) {
                const int su = stop_update(st, red5[0], red5[1], red5[2], red5[3], tol_err, min_iter);
                if (su != STOP_CONTINUE) fin = su == STOP_CONVERGED ? 1 : 2;
                else if (st.k >= max_iter) fin = 2;
                if (fin && b == 0) {
                    stp->st = st;
                    stp->done = 1;
                    stp->status = fin == 1 ? ST_OK : ST_ENOCONV;
                }
            }
            s_flag = fin;
        }
        float stats[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = jf; j < j1; j += kRunNT) {
            if (j != jf) {
                fy = __ldcg(ydst + j);
                fp = pprev[j];
                f1 = a.d1[j];
                f2 = a.d2[j];
            }
            const float pn = fy * inv;
            const float d = pn - fp;
            stats[0] += fabsf(d);
            stats[1] = fmaf(d, d, stats[1]);
            stats[2] = fmaf(d, f1, stats[2]);
            stats[3] = fmaf(d, f2, stats[3]);
            a.d2[j] = f1;
            a.d1[j] = d;
            pcur[j] = pn;
        }
        block_sum_k_1bar<kRunNT, 4>(stats, red + 5 * kRunW);   // its barrier also publishes s_flag
        if (s_flag) {
            // pi^(k-1) is the result; it lives in pi_alt when k-1 is odd
            if ((k - 1) & 1)
                for (int j = j0 + tid; j < j1; j += kRunNT) a.pi[j] = a.pi_alt[j];
            cp_async_wait<0>();   // the staged window is not used
            return;
        }
        if (tid == 0)
            reinterpret_cast<float4 *>(a.blk + (size_t)(k & 1) * G * 4)[b] =
                make_float4(stats[0], stats[1], stats[2], stats[3]);
    }
}

__global__ void __launch_bounds__(kRunNT, 2) chain_run_kernel(ChainRunArgs a) {
    chain_run_body(a, blockIdx.x, gridDim.x);
}

// Several chains in lockstep in one cooperative launch.  Step k of every
// chain still iterating runs in the same pass: the units of the active chains
// (the chain's 256-column tiles x 32-row blocks, chain after chain) are split
// evenly over the CTAs, each CTA leaves one partial per tile it touches and
// the last CTA to finish a shared tile adds them in CTA order; after one grid
// barrier the active chains' bins, chain after chain, are split evenly over
// the CTAs for the normalisation.  A second barrier publishes every CTA's
// step statistics; every CTA keeps an identical copy of each chain's stop
// state and decides on step k right then (the single-chain kernel decides one
// pass later instead, to save the barrier; here a pass is worth more than a
// barrier), so all CTAs drop a chain at the same step and re-split the work
// of the others, and no chain runs a pass past the step that ends it.

__device__ __forceinline__ long long lk_owner(long long u, long long U, int G) {
    return ((u + 1) * G + U - 1) / U - 1;
}

// Flush of tile t of chain g at the end of this CTA's segment of it: the warp
// partials added in warp order and normalised by inv; a tile that only this
// CTA touches is finished (y, v, the tile sum as one partial per warp), a shared
// tile leaves this CTA's partial in slot b - bf.
__device__ __forceinline__ void lk_flush(const ChainRunArgs &c, int t, int k, bool owned, int slot,
                                         const float (&acc)[kRunC], float (*wred)[kRunTW], float inv) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, N = c.N;
#pragma unroll
    for (int q = 0; q < kRunC; ++q) wred[wid][32 * q + lane] = acc[q];
    __syncthreads();
    if (tid < kRunTW) {
        float p = 0.f;
#pragma unroll
        for (int w = 0; w < kRunW; ++w) p += wred[w][tid];
        p *= inv;
        if (!owned) {
            c.part[((size_t)t * c.segs + slot) * kRunTW + tid] = p;
        } else {
            const int col = t * kRunTW + tid;
            if (col < N) {
                c.y[(size_t)(k & 1) * c.vlen + col] = p;
                int r = col + c.l;
                r -= (r >= N) ? N : 0;
                c.vb[(size_t)(k & 1) * c.vlen + r] = p * __ldg(c.rho + r);
            } else {
                p = 0.f;
            }
            const float ts = warp_sum(p);
            if (lane == 0) c.tsum[(size_t)(k & 1) * kRunTP * c.T + kRunTP * t + wid] = ts;
        }
    }
    __syncthreads();   // wred is reused
}

// The last CTA to finish shared tile t adds slots 0 .. nslot-1 in CTA order.
__device__ __forceinline__ void lk_tile_reduce(const ChainRunArgs &c, int t, int k, int nslot) {
    const int tid = threadIdx.x, N = c.N;
    const int col = t * kRunTW + tid;
    float yv = 0.f;
    if (tid < kRunTW && col < N) {
        int r = col + c.l;
        r -= (r >= N) ? N : 0;
        const float *pp = c.part + (size_t)t * c.segs * kRunTW + tid;
        yv = __ldcg(pp);
#pragma unroll 4
        for (int q = 1; q < nslot; ++q) yv += __ldcg(pp + (size_t)q * kRunTW);
        c.y[(size_t)(k & 1) * c.vlen + col] = yv;
        c.vb[(size_t)(k & 1) * c.vlen + r] = yv * __ldg(c.rho + r);
    }
    if (tid < kRunTW) {
        const float ts = warp_sum(yv);
        if ((tid & 31) == 0) c.tsum[(size_t)(k & 1) * kRunTP * c.T + kRunTP * t + (tid >> 5)] = ts;
    }
}

__global__ void __launch_bounds__(kRunNT, 2) chain_multi_kernel(const __grid_constant__ ChainMultiArgs m) {
    extern __shared__ float4 smem4[];
    float *sv = reinterpret_cast<float *>(smem4);
    __shared__ float wred[kRunW][kRunTW];
    __shared__ float red[8 * kRunW];                 // two alternating buffers of the per-chain sums
    __shared__ int s_flag;
    __shared__ long long s_ub[3][kChainMultiMax + 1];   // unit bases of the chains in step k's pass: slot k % 3
    __shared__ long long s_nb[3][kChainMultiMax + 1];   // bin bases (the normalisation of step k)
    __shared__ unsigned s_mask[3];                      // chains in step k's pass
    __shared__ float s_inv[kChainMultiMax];             // 1 / sum of y of each chain's last step
    __shared__ float s_eL[kChainMultiMax];
    __shared__ StopState s_st[kChainMultiMax];
    __shared__ int s_fin[kChainMultiMax];
    __shared__ int s_tile[6];                           // shared first / last tile: chain, tile, slots
    const int win_units = m.chunk / 32;   // a staging buffer holds m.chunk rows
    __shared__ int s_reg[2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned gen = 0u;
    // CTA sets: with two sets, the two CTAs of each SM go to different sets
    // (each set runs its own chains in lockstep with its own barrier), so one
    // CTA's barrier, normalisation and decisions overlap the other's FMA work
    int G = gridDim.x, b = blockIdx.x, n = m.n;
    const ChainRunArgs *cc = m.c;
    unsigned *sbar = m.words;
    if (m.nsets == 2) {
        if (tid == 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            const unsigned slot = atomicAdd(m.words + kMultiSlotWord + smid % kMultiSmSlots, 1u);
            s_reg[0] = (int)(slot & 1u);
            s_reg[1] = (int)atomicAdd(m.words + kMultiCountWord + (slot & 1u), 1u);
        }
        unsigned gen0 = 0u;
        // every CTA has registered before a set's size is read
        if (!grid_sync(m.words, gen0, m.c[0].err_flag, &s_flag, blockIdx.x, gridDim.x)) {
            if (tid < m.n) *m.c[tid].err_flag = 1;
            return;
        }
        const int set = s_reg[0];
        b = s_reg[1];
        G = (int)__ldcg(m.words + kMultiCountWord + set);
        cc = m.c + m.set_begin[set];
        n = m.set_begin[set + 1] - m.set_begin[set];
        sbar = m.words + (1 + set) * 2 * kBarGen;
        if (n == 0) return;   // a set without chains: nothing waits for its CTAs
    }

    // thread 0: unit and bin bases of the chains in `mask`, into slot sl
    auto bases = [&](int sl, unsigned mask) {
        long long u = 0, j = 0;
        for (int g = 0; g < n; ++g) {
            s_ub[sl][g] = u;
            s_nb[sl][g] = j;
            if (mask >> g & 1u) {
                u += (long long)cc[g].T * cc[g].RB;
                j += cc[g].N;
            }
        }
        s_ub[sl][n] = u;
        s_nb[sl][n] = j;
        s_mask[sl] = mask;
    };
    // this CTA's units [u0, u1) of step slot sl (all CTAs below min(G, U) get at least one)
    auto range = [&](int sl, long long &u0, long long &u1) {
        const long long U = s_ub[sl][n];
        const int Ge = (int)min((long long)G, U);
        u0 = b < Ge ? (long long)b * U / Ge : 0;
        u1 = b < Ge ? (long long)(b + 1) * U / Ge : 0;
    };
    // the chain holding unit u (chains without units this step are skipped)
    auto chain_of = [&](int sl, long long u) {
        int q = 0;
        while (s_ub[sl][q + 1] <= u) ++q;
        return q;
    };
    // windows: at most win_units units of one chain, in unit order
    auto win_first = [&](int sl, long long u0, long long u1, int &g, long long &lw0, long long &lw1) {
        if (u0 >= u1) return false;
        g = chain_of(sl, u0);
        lw0 = u0 - s_ub[sl][g];
        lw1 = min(lw0 + win_units, min(u1, s_ub[sl][g + 1]) - s_ub[sl][g]);
        return true;
    };
    auto win_next = [&](int sl, long long u1, int &g, long long &lw0, long long &lw1) {
        const long long end = min(u1, s_ub[sl][g + 1]) - s_ub[sl][g];
        if (lw1 < end) {
            lw0 = lw1;
            lw1 = min(lw0 + win_units, end);
            return true;
        }
        if (s_ub[sl][g + 1] >= u1) return false;
        g = chain_of(sl, s_ub[sl][g + 1]);
        lw0 = 0;
        lw1 = min((long long)win_units, min(u1, s_ub[sl][g + 1]) - s_ub[sl][g]);
        return true;
    };
    // 16-byte async copies of a window's rows into buffer buf; step k reads
    // the start vector (k = 1) or the previous step's broadcast vector
    auto stage = [&](int g, long long lw0, long long lw1, int buf, int k) {
        const ChainRunArgs &c = cc[g];
        const float *src = k == 1 ? c.v0 : c.vb + (size_t)((k - 1) & 1) * c.vlen;
        const int RB = c.RB;
        const int off0 = (int)(lw0 % RB);
        const int nq = (int)(lw1 - lw0) * 8;
        float *dst = sv + (size_t)buf * m.chunk;
        for (int q = tid; q < nq; q += kRunNT) {
            int o = off0 + (q >> 3);
            o -= (o / RB) * RB;                     // 32-row block inside its tile
            cp_async16(dst + 4 * q, src + 4 * (o * 8 + (q & 7)));
        }
        cp_async_commit();
    };

    if (tid < n) {
        s_st[tid] = cc[tid].state->st;
        s_inv[tid] = 1.f;
        s_eL[tid] = (float)cc[tid].scal[1];
    }
    if (tid == 0) bases(1, n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u));
    __syncthreads();
    {
        long long u0, u1, lw0, lw1;
        int g;
        range(1, u0, u1);
        if (win_first(1, u0, u1, g, lw0, lw1)) stage(g, lw0, lw1, 0, 1);
    }

    for (int k = 1;; ++k) {
        const int sl = k % 3;
        const unsigned mask = s_mask[sl];
        const long long U = s_ub[sl][n];
        const int Ge = (int)min((long long)G, U);
        long long u0, u1;
        range(sl, u0, u1);
        // ---- pass k over this CTA's units; window 0 is already in flight
        int cur_g = -1, cur_t = -1;
        float mlo[kRunC], mhi[kRunC], acc[kRunC];
        auto flush = [&]() {
            const ChainRunArgs &c = cc[cur_g];
            const long long tu = s_ub[sl][cur_g] + (long long)cur_t * c.RB;
            const int bf = (int)lk_owner(tu, U, Ge), bl = (int)lk_owner(tu + c.RB - 1, U, Ge);
            const int slot = b - bf;
            if (bf != bl && slot >= c.segs) {          // outside the partial slots: report, write nothing
                if (tid == 0) atomicExch(cc[0].err_flag, 1);
                return;
            }
            lk_flush(c, cur_t, k, bf == bl, slot, acc, wred, s_inv[cur_g]);
        };
        int g;
        long long lw0, lw1;
        bool more = win_first(sl, u0, u1, g, lw0, lw1);
        for (int wi = 0; more; ++wi) {
            int ng = g;
            long long nw0 = lw0, nw1 = lw1;
            const bool has_next = win_next(sl, u1, ng, nw0, nw1);
            if (has_next) {
                stage(ng, nw0, nw1, (wi + 1) & 1, k);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const ChainRunArgs &c = cc[g];
            const int RB = c.RB, N = c.N;
            const float *wbuf = sv + (size_t)(wi & 1) * m.chunk;
            for (int t = (int)(lw0 / RB); (long long)t * RB < lw1; ++t) {
                const long long su0 = max(lw0, (long long)t * RB), su1 = min(lw1, (long long)(t + 1) * RB);
                if (t != cur_t || g != cur_g) {
                    if (cur_g >= 0) flush();
#pragma unroll
                    for (int q = 0; q < kRunC; ++q) {
                        const int col = t * kRunTW + 32 * q + lane;
                        const float x = col < N ? __ldg(c.w + col) : 0.f;
                        mlo[q] = x;
                        mhi[q] = x * s_eL[g];
                        acc[q] = 0.f;
                    }
                    cur_g = g;
                    cur_t = t;
                }
                // warp wid takes 32-row blocks [wb0, wb1) of the segment
                const int rb0 = (int)(su0 - (long long)t * RB), rb1 = (int)(su1 - (long long)t * RB);
                const int nb = rb1 - rb0;
                const int wb0 = rb0 + (nb * wid) / kRunW, wb1 = rb0 + (nb * (wid + 1)) / kRunW;
                if (wb1 > wb0) {
                    const float *vt = wbuf + ((long long)t * RB - lw0) * 32;   // row r of tile t at vt[r]
                    float out[kRunC];
                    tri_pass<kRunC, false, kChain, true, false>(vt, 32 * wb0, 32 * wb1, t * kRunTW, lane, mlo, mhi,
                                                               out);
#pragma unroll
                    for (int q = 0; q < kRunC; ++q) acc[q] += out[q];
                }
            }
            __syncthreads();   // this buffer is restaged two windows later
            g = ng;
            lw0 = nw0;
            lw1 = nw1;
            more = has_next;
        }
        if (cur_g >= 0) flush();
        // shared first / last tile of the range: the last CTA to finish one adds its partials
        __syncthreads();
        if (tid == 0) {
            int mask2 = 0;
            if (u0 < u1) {
                long long ue[2] = {u0, u1 - 1};
                int prev_g = -1, prev_t = -1;
                for (int e = 0; e < 2; ++e) {
                    const int q = chain_of(sl, ue[e]);
                    const ChainRunArgs &c = cc[q];
                    const int t = (int)((ue[e] - s_ub[sl][q]) / c.RB);
                    if (q == prev_g && t == prev_t) break;
                    prev_g = q;
                    prev_t = t;
                    const long long tu = s_ub[sl][q] + (long long)t * c.RB;
                    const int bf = (int)lk_owner(tu, U, Ge), bl = (int)lk_owner(tu + c.RB - 1, U, Ge);
                    if (bf == bl) continue;
                    __threadfence();
                    const int old = atomicAdd(c.tile_ticket + t, 1);
                    if (old == bl - bf) {
                        c.tile_ticket[t] = 0;
                        __threadfence();
                        mask2 |= 1 << e;
                        s_tile[3 * e] = q;
                        s_tile[3 * e + 1] = t;
                        s_tile[3 * e + 2] = min(bl - bf + 1, c.segs);
                    }
                }
            }
            s_flag = mask2;
        }
        __syncthreads();
        const int lastmask = s_flag;
        if (lastmask & 1) lk_tile_reduce(cc[s_tile[0]], s_tile[1], k, s_tile[2]);
        if (lastmask & 2) lk_tile_reduce(cc[s_tile[3]], s_tile[4], k, s_tile[5]);
        if (!grid_sync(sbar, gen, cc[0].err_flag, &s_flag, b, G)) {
            if (tid < n) {
                *cc[tid].err_flag = 1;
                if (b == 0) {
                    ChainState *stp = cc[tid].state;
                    stp->st = s_st[tid];
                    stp->done = 1;
                    stp->status = ST_ENOCONV;
                }
            }
            return;
        }
        // ---- step k is complete: per chain (one warp each) the sum of y
        for (int q = wid; q < n; q += kRunW) {
            if (!(mask >> q & 1u)) continue;
            const ChainRunArgs &c = cc[q];
            const float *ts = c.tsum + (size_t)(k & 1) * kRunTP * c.T;
            const int nts = kRunTP * c.T;
            float sy = 0.f;
            for (int i = lane; i < nts; i += 128) {   // four independent loads per lane in flight
                const float x0 = __ldcg(ts + i);
                const float x1 = i + 32 < nts ? __ldcg(ts + i + 32) : 0.f;
                const float x2 = i + 64 < nts ? __ldcg(ts + i + 64) : 0.f;
                const float x3 = i + 96 < nts ? __ldcg(ts + i + 96) : 0.f;
                sy += (x0 + x1) + (x2 + x3);
            }
            sy = warp_sum(sy);
            if (lane == 0) s_inv[q] = 1.f / sy;
        }
        __syncthreads();
        // ---- normalise step k over this CTA's bins of the chains in the pass,
        // leaving this CTA's step statistics of each chain in blk
        const long long NB = s_nb[sl][n];
        const int GeN = (int)min((long long)G, NB);
        const long long j0 = b < GeN ? (long long)b * NB / GeN : 0, j1 = b < GeN ? (long long)(b + 1) * NB / GeN : 0;
        {
            int piece = 0;
            for (int q = 0; q < n; ++q) {
                if (!(mask >> q & 1u)) continue;
                const long long cb0 = s_nb[sl][q], cb1 = s_nb[sl][q + 1];
                if (cb1 <= j0 || cb0 >= j1) continue;
                const ChainRunArgs &c = cc[q];
                const int a0 = (int)(max(j0, cb0) - cb0), a1 = (int)(min(j1, cb1) - cb0);
                float *pcur = (k & 1) ? c.pi_alt : c.pi;
                const float *pprev = (k & 1) ? c.pi : c.pi_alt;
                const float *yk = c.y + (size_t)(k & 1) * c.vlen;
                const float inv = s_inv[q];
                float stats[4] = {0.f, 0.f, 0.f, 0.f};
                for (int j = a0 + tid; j < a1; j += kRunNT) {
                    const float pn = __ldcg(yk + j) * inv;
                    // written by whichever CTA held bin j in the last step (L2 loads)
                    const float d = pn - __ldcg(pprev + j);
                    const float f1 = __ldcg(c.d1 + j);
                    stats[0] += fabsf(d);
                    stats[1] = fmaf(d, d, stats[1]);
                    stats[2] = fmaf(d, f1, stats[2]);
                    stats[3] = fmaf(d, __ldcg(c.d2 + j), stats[3]);
                    c.d2[j] = f1;
                    c.d1[j] = d;
                    pcur[j] = pn;
                }
                // one barrier; consecutive chains alternate buffers, so a buffer
                // is rewritten only after every thread passed the barrier between
                block_sum_k_1bar<kRunNT, 4>(stats, red + (piece++ & 1) * 4 * kRunW);
                if (tid == 0)
                    reinterpret_cast<float4 *>(c.blk + (size_t)(k & 1) * G * 4)[b] =
                        make_float4(stats[0], stats[1], stats[2], stats[3]);
            }
        }
        // ---- every CTA's statistics of step k are written: one more barrier,
        // then the decision on step k itself (no pass is run past it)
        if (!grid_sync(sbar, gen, cc[0].err_flag, &s_flag, b, G)) {
            if (tid < n) {
                *cc[tid].err_flag = 1;
                if (b == 0) {
                    ChainState *stp = cc[tid].state;
                    stp->st = s_st[tid];
                    stp->done = 1;
                    stp->status = ST_ENOCONV;
                }
            }
            return;
        }
        for (int q = wid; q < n; q += kRunW) {
            if (!(mask >> q & 1u)) continue;
            const ChainRunArgs &c = cc[q];
            const long long cj0 = s_nb[sl][q];
            const int bF = (int)lk_owner(cj0, NB, GeN), bL = (int)lk_owner(cj0 + c.N - 1, NB, GeN);
            const float4 *bs = reinterpret_cast<const float4 *>(c.blk + (size_t)(k & 1) * G * 4);
            float sx = 0.f, sd = 0.f, s1 = 0.f, s2 = 0.f;
            for (int i = bF + lane; i <= bL; i += 32) {
                const float4 x = __ldcg(bs + i);
                sx += x.x;
                sd += x.y;
                s1 += x.z;
                s2 += x.w;
            }
            sx = warp_sum(sx);
            sd = warp_sum(sd);
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            if (lane == 0) {
                int fin = 0;
                const int su = stop_update(s_st[q], sx, sd, s1, s2, m.tol_err, m.min_iter);
                if (su != STOP_CONTINUE) fin = su == STOP_CONVERGED ? 1 : 2;
                else if (s_st[q].k >= m.max_iter) fin = 2;
                s_fin[q] = fin;
            }
        }
        __syncthreads();
        unsigned next = mask;
        for (int q = 0; q < n; ++q)
            if ((mask >> q & 1u) && s_fin[q]) next &= ~(1u << q);
        if (b == 0 && tid < n && (mask >> tid & 1u) && s_fin[tid]) {
            ChainState *stp = cc[tid].state;
            stp->st = s_st[tid];
            stp->done = 1;
            stp->status = s_fin[tid] == 1 ? ST_OK : ST_ENOCONV;
        }
        // a chain decided on step k keeps pi^(k); when it lives in pi_alt (k
        // odd), the CTA that normalised a bin copies it
        if (k & 1) {
            for (int q = 0; q < n; ++q) {
                if (!(mask >> q & 1u) || !s_fin[q]) continue;
                const long long cb0 = s_nb[sl][q], cb1 = s_nb[sl][q + 1];
                if (cb1 <= j0 || cb0 >= j1) continue;
                const ChainRunArgs &c = cc[q];
                const int a0 = (int)(max(j0, cb0) - cb0), a1 = (int)(min(j1, cb1) - cb0);
                for (int j = a0 + tid; j < a1; j += kRunNT) c.pi[j] = c.pi_alt[j];
            }
        }
        if (!next) return;   // every chain decided
        // the next step's partition, and its first window staged
        if (tid == 0) bases((k + 1) % 3, next);
        __syncthreads();
        {
            long long v0, v1, w0, w1;
            int q;
            range((k + 1) % 3, v0, v1);
            if (win_first((k + 1) % 3, v0, v1, q, w0, w1)) stage(q, w0, w1, 0, k + 1);
        }
    }
}

// Start of a multi-chain iteration, one block per chain: uniform pi^(0) (as
// init_iter_kernel without a warm start), cleared step vectors, the first
// broadcast vector h_k = pi^(0)_{(k-l) mod N} rho_k, the stop state, and the
// chain's error flag and tile tickets zeroed (block 0 also the launch's
// barrier words).
__global__ void __launch_bounds__(kRunNT) chain_multi_init_kernel(const __grid_constant__ ChainMultiArgs m) {
    const ChainRunArgs &a = m.c[blockIdx.x];
    const int N = a.N, tid = threadIdx.x;
    const float p0 = 1.f / (float)N;
    for (int j = tid; j < N; j += kRunNT) {
        a.pi[j] = p0;
        a.d1[j] = 0.f;
        a.d2[j] = 0.f;
    }
    for (int k = tid; k < a.vlen; k += kRunNT) {
        float *v0 = const_cast<float *>(a.v0);
        v0[k] = k < N ? p0 * a.rho[k] : 0.f;
    }
    for (int t = tid; t < a.T; t += kRunNT) a.tile_ticket[t] = 0;
    if (blockIdx.x == 0)
        for (int q = tid; q < kMultiWords; q += kRunNT) m.words[q] = 0u;
    if (tid == 0) {
        *a.err_flag = 0;
        ChainState *stp = a.state;
        StopState st;
        stop_init(st, 1.f, 0.f);
        stp->st = st;
        stp->done = 0;
        stp->status = ST_ENOCONV;
        stp->tol_err = m.tol_err;
        stp->max_iter = m.max_iter;
        stp->min_iter = m.min_iter;
    }
}

// End of a multi-chain iteration, one block per chain: the result copied to
// out + off[g] and the chain's report (as the single-chain call reports it).
__global__ void __launch_bounds__(kRunNT) chain_multi_finish_kernel(const __grid_constant__ ChainMultiArgs m,
                                                                    float *__restrict__ out,
                                                                    ReportDev *__restrict__ reps) {
    const ChainRunArgs &a = m.c[blockIdx.x];
    float *dst = out + m.off[blockIdx.x];
    for (int j = threadIdx.x; j < a.N; j += kRunNT) dst[j] = a.pi[j];
    if (threadIdx.x == 0 && reps) {
        const ChainState &h = *a.state;
        const int err = *a.err_flag;
        ReportDev r;
        r.iters = h.st.k;
        r.status = err ? ST_ETIMEOUT : (h.done && h.status == ST_OK ? ST_OK : ST_ENOCONV);
        r.last_step_l1 = h.st.k > 0 ? h.st.delta[(h.st.k - 1) & 7] : 0.f;
        r.err_bound = h.st.err;
        r.lambda2_abs = h.st.rho;
        r.lambda2_phase = h.st.theta;
        reps[m.idx[blockIdx.x]] = r;
    }
}

// ======================================================================
// Self-test of the bounded waits
// ======================================================================
//
// The waits of the kernels above give up after a limit and report; these two
// kernels make such waits run out on purpose, with short limits: an mbarrier
// phase that nothing completes, and a grid barrier that one CTA of a
// cooperative launch never reaches (both waiting CTAs give up, set the error
// flag and poison the arrival count).

__global__ void selftest_mbar_kernel(int *status, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        status[0] = mbar_wait(&bar, 0, limit) ? 0 : 1;   // nothing arrives
    }
}

__global__ void selftest_grid_kernel(unsigned *bar, int *err_flag, int *status, uint32_t limit) {
    __shared__ int s_flag;
    unsigned gen = 0u;
    if (blockIdx.x == gridDim.x - 1) return;             // this CTA never arrives
    const bool ok = grid_sync(bar, gen, err_flag, &s_flag, blockIdx.x, gridDim.x, limit);
    if (threadIdx.x == 0 && !ok) atomicAdd(status + 1, 1);
}

cudaError_t launch_selftest_waits(unsigned *bar, int *err_flag, int *status, cudaStream_t s) {
    selftest_mbar_kernel<<<1, 32, 0, s>>>(status, 1u << 14);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t limit = 1u << 16;
    void *params[] = {&bar, &err_flag, &status, &limit};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(selftest_grid_kernel), dim3(3), dim3(32), params,
                                       0, s);
}

// ======================================================================
// FP32 FMA throughput (the denominator of the FP32 rooflines)
// ======================================================================
//
// Every thread runs kFmaChains independent FMA chains x <- x a + b for `iters`
// rounds; the chains give each warp enough independent instructions to cover
// the FMA latency, and the unrolled inner loop keeps the loop overhead a few
// percent of the issue slots.  4 blocks of 256 threads per SM.  The sum of
// the chains is written so that no FMA can be removed.  Work per launch:
// 2 FLOP x kFmaChains x iters x threads.

constexpr int kFmaChains = 16;
constexpr int kFmaNT = 256;

__global__ void __launch_bounds__(kFmaNT) fma_peak_kernel(float *out, int iters, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) sum += x[k];
    out[(size_t)blockIdx.x * kFmaNT + threadIdx.x] = sum;
}

int fma_peak_blocks(int sms) { return 4 * sms; }
double fma_peak_flop(int sms, int iters) { return 2.0 * kFmaChains * (double)iters * fma_peak_blocks(sms) * kFmaNT; }
size_t fma_peak_out_floats(int sms) { return (size_t)fma_peak_blocks(sms) * kFmaNT; }

cudaError_t launch_fma_peak(float *out, int sms, int iters, cudaStream_t s) {
    fma_peak_kernel<<<fma_peak_blocks(sms), kFmaNT, 0, s>>>(out, iters, 0.9999999f, 1e-7f);
    return cudaGetLastError();
}

// ======================================================================
// Finish of one power step (whole GPU, two kernels)
// ======================================================================
//
// Stage 1 reduces the dense pass's partial column sums into y and sums y;
// stage 2 normalises, forms the step statistics, applies the stop rule and
// prepares the next broadcast vector:
//   materialised: c_i = pi_i / r_i           (row space)
//   fused:        h_k = pi_{(k-l) mod N} rho_k  (p-space)
// Each stage's grid-wide sum goes through per-CTA partials that the last CTA
// to arrive (an atomic ticket) adds in CTA order: the result does not depend
// on which CTA finishes last, and no CTA ever waits for another.

constexpr int kFinishNT = 256;

// Publishes this CTA's partials (written by thread 0 before the call) and
// tells whether it is the last CTA of the grid to do so.
__device__ __forceinline__ bool arrive_last(int *ticket, bool *s_last) {
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    return *s_last;
}

template <int NT>
__global__ void __launch_bounds__(NT) reduce_parts_kernel(FinishArgs a) {
    __shared__ float red[NT / 32 + 1];
    __shared__ bool s_last;
    ChainState *stp = a.state;
    if (stp->done) return;
    const int j = blockIdx.x * NT + threadIdx.x;
    float y = 0.f;
    if (j < a.N) {
        if (a.mode == 0) {
            // materialised: partials per (cta, slot)
            const int slab = j / kGemvCols, t = j - slab * kGemvCols;
            const int lo = slab * a.tiles_per_slab, hi = lo + a.tiles_per_slab - 1;
            const int c_lo = lo / a.tiles_per_cta, c_hi = hi / a.tiles_per_cta;
            for (int c = c_lo; c <= c_hi; ++c) {
                const int slot = slab - (c * a.tiles_per_cta) / a.tiles_per_slab;
                y += a.part[((size_t)c * 2 + slot) * kGemvCols + t];
            }
        } else {
            for (int q = 0; q < a.nparts; ++q) y += a.part[(size_t)q * a.ld_part + j];
        }
        a.y[j] = y;
    }
    const float bs = block_sum<NT>(y, red);
    if (threadIdx.x == 0) a.blk[blockIdx.x] = bs;
    if (!arrive_last(a.ticket, &s_last)) return;
    float t = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) t += __ldcg(a.blk + b);
    const float sum = block_sum<NT>(t, red);
    if (threadIdx.x == 0) {
        stp->ysum = sum;
        a.ticket[0] = 0;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) normalize_step_kernel(FinishArgs a) {
    __shared__ float red[4 * (NT / 32) + 4];
    __shared__ bool s_last;
    ChainState *stp = a.state;
    if (stp->done) return;
    const int N = a.N;
    const float inv = 1.f / stp->ysum;
    const int j = blockIdx.x * NT + threadIdx.x;
    float stats[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < N) {
        const float pn = a.y[j] * inv;
        const float d = pn - a.pi[j];
        const float e1 = a.d1[j], e2 = a.d2[j];
        stats[0] = fabsf(d);
        stats[1] = d * d;
        stats[2] = d * e1;
        stats[3] = d * e2;
        a.d2[j] = e1;
        a.d1[j] = d;
        a.pi[j] = pn;
    }
    if (j < a.vlen) {
        // next broadcast vector, from y (pi of another index may not be
        // written yet); y_i * inv is the same number as the new pi_i
        float h = 0.f;
        if (j < N) {
            if (a.mode == 0) {
                h = (a.y[j] * inv) / a.rowsum[j];
            } else {
                int i = j - a.l;
                i += (i < 0) ? N : 0;
                h = (a.y[i] * inv) * a.rho[j];
            }
        }
        a.v[j] = h;
    }
    block_sum_k<NT, 4>(stats, red);
    float *blk = a.blk + gridDim.x;     // stage 1 used the first gridDim.x (at most) floats
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) blk[4 * blockIdx.x + k] = stats[k];
    }
    if (!arrive_last(a.ticket + 1, &s_last)) return;
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] += __ldcg(blk + 4 * b + k);
    }
    block_sum_k<NT, 4>(t, red);
    if (threadIdx.x == 0) {
        StopState st = stp->st;
        const int su = stop_update(st, t[0], t[1], t[2], t[3], stp->tol_err, stp->min_iter);
        stp->st = st;
        if (su != STOP_CONTINUE) {
            stp->done = 1;
            stp->status = su == STOP_CONVERGED ? ST_OK : ST_ENOCONV;
        } else if (st.k >= stp->max_iter) {
            stp->done = 1;
            stp->status = ST_ENOCONV;
        }
        a.ticket[1] = 0;
    }
}

// Start of an iteration: pi = uniform or normalised warm weights; stop state
// reset; first broadcast vector.
template <int NT>
__global__ void __launch_bounds__(NT) init_iter_kernel(FinishArgs a, const float *__restrict__ warm) {
    __shared__ float red[8 * (NT / 32) + 8];
    const int N = a.N, tid = threadIdx.x;
    float ls = 0.f;
    for (int j = tid; j < N; j += NT) {
        const float x = warm ? fmaxf(warm[j], 0.f) : 1.f;
        a.pi[j] = x;
        ls += x;
        a.d1[j] = 0.f;
        a.d2[j] = 0.f;
    }
    const float s = block_sum<NT>(ls, red);
    const bool ok = s > 0.f && isfinite(s);
    for (int j = tid; j < N; j += NT) a.pi[j] = ok ? a.pi[j] / s : 1.f / (float)N;
    __syncthreads();
    for (int k = tid; k < a.vlen; k += NT) {
        float h = 0.f;
        if (k < N) {
            if (a.mode == 0) {
                h = a.pi[k] / a.rowsum[k];
            } else {
                int i = k - a.l;
                i += (i < 0) ? N : 0;
                h = a.pi[i] * a.rho[k];
            }
        }
        a.v[k] = h;
    }
    if (tid == 0) {
        StopState st;
        stop_init(st, 1.f, warm != nullptr ? kWarmRhoFloor : 0.f);
        a.state->st = st;
        a.state->done = 0;
        a.state->status = ST_ENOCONV;
    }
}

// rho_k = u_k / r'_k from the split row pass partials; also the row sums of
// the paper's P for inspection.
template <int NT>
__global__ void __launch_bounds__(NT) finish_rows_kernel(int N, int nparts, int ld_part,
                                                         const float *__restrict__ part,
                                                         const float *__restrict__ u, float *__restrict__ rho,
                                                         float *__restrict__ rowsum_p, int l) {
    for (int k = blockIdx.x * NT + threadIdx.x; k < N; k += gridDim.x * NT) {
        float r = 0.f;
        for (int q = 0; q < nparts; ++q) r += part[(size_t)q * ld_part + k];
        rho[k] = u[k] / r;
        // row i = (k - l) mod N of P has sum r'_k
        int i = k - l;
        i += (i < 0) ? N : 0;
        if (rowsum_p) rowsum_p[i] = r;
    }
}

// ======================================================================
// Launchers
// ======================================================================

int batch_threads_for(int nmax) { (void)nmax; return 256; }

template <int NT, int C, int LEVEL, bool STRUCT>
static cudaError_t launch_batch_one(const BatchArgs &a, int grid, size_t smem, cudaStream_t s) {
    auto k = batch_fused_kernel<NT, C, LEVEL, STRUCT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT, int C, bool STRUCT>
static cudaError_t launch_batch_c(const BatchArgs &a, int grid, size_t smem, cudaStream_t s) {
    if (a.state_level == 2) return launch_batch_one<NT, C, 2, STRUCT>(a, grid, smem, s);
    if (a.state_level == 1) return launch_batch_one<NT, C, 1, STRUCT>(a, grid, smem, s);
    return launch_batch_one<NT, C, 0, STRUCT>(a, grid, smem, s);
}

// Dense passes with 8 (default) or 4 columns per thread; the structured step
// has no column pass and runs with 8.
template <int NT, bool STRUCT>
static cudaError_t launch_batch_nt(const BatchArgs &a, int grid, size_t smem, cudaStream_t s) {
    if constexpr (!STRUCT) {
        if (a.cols == 4) return launch_batch_c<NT, 4, STRUCT>(a, grid, smem, s);
    }
    return launch_batch_c<NT, SPL_BATCH_C, STRUCT>(a, grid, smem, s);
}

cudaError_t launch_pixel_const(const PixelDev *px, int n, PixelConst *out, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    pixel_const_kernel<<<(n + 127) / 128, 128, 0, s>>>(px, n, out);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &a, int threads, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = launch_pixel_const(a.px, a.n, a.pconst, s);
    if (e != cudaSuccess) return e;
    if (a.structured) return launch_batch_nt<256, true>(a, grid, smem, s);
    if (threads == 512) return launch_batch_nt<512, false>(a, grid, smem, s);
    return launch_batch_nt<256, false>(a, grid, smem, s);
}

template <int NT, int C, int LEVEL, bool STRUCT>
static cudaError_t occupancy_one(size_t smem, int *bps) {
    auto k = batch_fused_kernel<NT, C, LEVEL, STRUCT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, NT, smem);
}

template <int NT, int C, bool STRUCT>
static cudaError_t occupancy_nt(int level, size_t smem, int *bps) {
    if (level == 2) return occupancy_one<NT, C, 2, STRUCT>(smem, bps);
    if (level == 1) return occupancy_one<NT, C, 1, STRUCT>(smem, bps);
    return occupancy_one<NT, C, 0, STRUCT>(smem, bps);
}

cudaError_t batch_occupancy(int threads, int level, bool structured, size_t smem, int *blocks_per_sm, int cols) {
    if (structured) return occupancy_nt<256, SPL_BATCH_C, true>(level, smem, blocks_per_sm);
    if (threads == 512)
        return cols == 4 ? occupancy_nt<512, 4, false>(level, smem, blocks_per_sm)
                         : occupancy_nt<512, SPL_BATCH_C, false>(level, smem, blocks_per_sm);
    return cols == 4 ? occupancy_nt<256, 4, false>(level, smem, blocks_per_sm)
                     : occupancy_nt<256, SPL_BATCH_C, false>(level, smem, blocks_per_sm);
}

int batch_pad_len(int n) { return pad_len(n, SPL_BATCH_C); }

// The vectors kept in shared memory at a state level (8, 3 or 1 of them) and
// the FP64 table of 64-bin blocks of the geometric flux factor.
size_t batch_smem_bytes(int npad, int level) {
    const size_t vec = (size_t)(level == 2 ? 8 : (level == 1 ? 3 : 1)) * npad * sizeof(float);
    return vec + (size_t)(npad / 64 + 2) * sizeof(double);
}

// Largest state level whose shared memory still lets three 256-thread blocks
// share an SM.
int batch_state_level(int npad, bool structured) {
    if (!structured && batch_smem_bytes(npad, 2) <= 100 * 1024) return 2;
    if (batch_smem_bytes(npad, 1) <= (structured ? 48 : 72) * 1024) return 1;
    return 0;
}

cudaError_t launch_chain_flux(const PixelDev &p, float *w, float *u, float *lam, double *F, double *scal, int npad,
                              cudaStream_t s) {
    const int threads = 256;
    int blocks = (npad + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    chain_flux_kernel<<<blocks, threads, 0, s>>>(p, w, u, lam, F, scal, npad);
    return cudaGetLastError();
}

cudaError_t launch_build_matrix(int N, int l, int ld, const float *w, const float *u, const double *scal, float *P,
                                float *rowsum, int num_sms, cudaStream_t s) {
    int blocks = num_sms * 8;
    const int need = (N + 7) / 8;
    if (blocks > need) blocks = need;
    build_matrix_kernel<<<blocks, 256, 0, s>>>(N, l, ld, w, u, scal, P, rowsum);
    return cudaGetLastError();
}

constexpr int kGemvStages = SPL_GEMV_STAGES;

int gemv_slab_cols() { return kGemvCols; }

size_t gemv_smem_bytes() { return (size_t)kGemvStages * kGemvTileBytes + 1024 + (size_t)kGemvMaxSmemC * 4; }

cudaError_t launch_gemv(const CUtensorMap *map, const GemvArgs &a, int grid, cudaStream_t s) {
    const bool smem_c = a.tiles_per_slab * kGemvRows <= kGemvMaxSmemC;
    const size_t smem = (size_t)kGemvStages * kGemvTileBytes + 1024 +
                        (smem_c ? (size_t)a.tiles_per_slab * kGemvRows * 4 : 0);
    cudaError_t e;
    if (smem_c) {
        auto k = gemv_tma_kernel<kGemvStages, true>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kGemvThreads, smem, s>>>(*map, a);
    } else {
        auto k = gemv_tma_kernel<kGemvStages, false>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kGemvThreads, smem, s>>>(*map, a);
    }
    return cudaGetLastError();
}

constexpr int kSplitNT = 128;
constexpr int kSplitC = 4;

int split_cols_per_cta() { return kSplitNT * kSplitC; }
int split_pad_len(int n) { return pad_len(n, kSplitC); }

cudaError_t launch_tri_split(const TriSplitArgs &a, bool row_pass, int chunks, cudaStream_t s) {
    const int cols = kSplitNT * kSplitC;
    dim3 grid((a.N + cols - 1) / cols, chunks);
    const size_t smem = (size_t)a.chunk * sizeof(float);
    cudaError_t e;
    if (row_pass) {
        auto k = tri_split_kernel<kSplitNT, kSplitC, true>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kSplitNT, smem, s>>>(a);
    } else {
        auto k = tri_split_kernel<kSplitNT, kSplitC, false>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kSplitNT, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish_rows(int N, int nparts, int ld_part, const float *part, const float *u, float *rho,
                               float *rowsum_p, int l, cudaStream_t s) {
    int blocks = (N + 255) / 256;
    finish_rows_kernel<256><<<blocks, 256, 0, s>>>(N, nparts, ld_part, part, u, rho, rowsum_p, l);
    return cudaGetLastError();
}

cudaError_t launch_finish_step(const FinishArgs &a, cudaStream_t s) {
    const int g1 = (a.N + kFinishNT - 1) / kFinishNT;
    const int g2 = (a.vlen + kFinishNT - 1) / kFinishNT;   // vlen >= N
    reduce_parts_kernel<kFinishNT><<<g1, kFinishNT, 0, s>>>(a);
    normalize_step_kernel<kFinishNT><<<g2, kFinishNT, 0, s>>>(a);
    return cudaGetLastError();
}

int chain_run_tile_cols() { return kRunTW; }
int chain_run_bar_words() { return 2 * kBarGen; }
int chain_run_max_grid() { return 2 * kRunNT; }
int chain_run_max_chunk() { return kRunMaxChunk; }
size_t chain_run_smem_bytes(int chunk) { return 2 * (size_t)chunk * sizeof(float); }   // two staging buffers

int chain_run_blocks_per_sm(int chunk) {
    const size_t smem = chain_run_smem_bytes(chunk);
    if (cudaFuncSetAttribute(chain_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chain_run_kernel, kRunNT, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_chain_run(const ChainRunArgs &a, int grid, cudaStream_t s) {
    const size_t smem = chain_run_smem_bytes(a.chunk);
    cudaError_t e = cudaFuncSetAttribute(chain_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ChainRunArgs args = a;
    void *params[] = {&args};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(chain_run_kernel), dim3(grid), dim3(kRunNT),
                                       params, smem, s);
}

cudaError_t launch_chain_multi(const ChainMultiArgs &m, int grid, float *out, ReportDev *reps, cudaStream_t s) {
    chain_multi_init_kernel<<<m.n, kRunNT, 0, s>>>(m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = chain_run_smem_bytes(m.chunk);
    e = cudaFuncSetAttribute(chain_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *params[] = {const_cast<ChainMultiArgs *>(&m)};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(chain_multi_kernel), dim3(grid), dim3(kRunNT),
                                    params, smem, s);
    if (e != cudaSuccess) return e;
    chain_multi_finish_kernel<<<m.n, kRunNT, 0, s>>>(m, out, reps);
    return cudaGetLastError();
}

int chain_multi_slots(int n_bins, int grid) {
    const long long T = (n_bins + kRunTW - 1) / kRunTW, RB = split_pad_len(n_bins) / 32;
    // every CTA of a lockstep partition gets at least max(1, floor(T RB / grid)) units
    const long long umin = T * RB / grid;
    const long long slots = umin >= 1 ? (RB + umin - 1) / umin + 1 : RB;
    return (int)(slots < grid ? slots : grid);
}

int chain_multi_blocks_per_sm(int chunk) {
    const size_t smem = chain_run_smem_bytes(chunk);
    if (cudaFuncSetAttribute(chain_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chain_multi_kernel, kRunNT, smem) != cudaSuccess) return 0;
    return nb;
}

size_t finish_blk_floats(int vlen) { return 5 * (size_t)((vlen + kFinishNT - 1) / kFinishNT); }

cudaError_t launch_init_iter(const FinishArgs &a, const float *warm, cudaStream_t s) {
    init_iter_kernel<1024><<<1, 1024, 0, s>>>(a, warm);
    return cudaGetLastError();
}

}  // namespace spl
