// Device-side building blocks shared by the libspl kernels (sm_103a).
//
// Notation (0-based): N bins, Delta = t_r / N, s_j = (j + 1/2) Delta,
// l = row shift, p_i = (i + l) mod N, Lambda = F(t_r), eL = exp(-Lambda).
//
// Eq. 6 with the roll of Sec. 3.4 gives the unnormalised kernel
//     P_ij = lambda_j exp(F_p - F_j - Lambda 1{p > j}),   p = p_i.
// It factors exactly into a row factor, a column factor and a two-valued
// triangle weight:
//     P_ij = u_p * w_j * mu(p, j),   u_k = exp(F_k - Lambda/2),
//     w_j = lambda_j exp(Lambda/2 - F_j),   mu(k, j) = 1 if k <= j else eL.
// (The Lambda/2 centring keeps both factors inside FP32 range for Lambda up
// to 120; it cancels in the product.)  u and w are formed in FP64 from the
// FP64 cumulative flux and rounded once to FP32, so a matrix entry carries
// ~2 FP32 roundings instead of the ~1e-6 relative error an FP32 exponent of
// a difference of cumulative fluxes of size ~10 would carry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spl {

// Per-pixel parameters after host validation.  t_d is already folded into l.
struct PixelDev {
    double t_r, tau, sigma, S, B;
    int32_t N;
    int32_t l;            // row shift in [0, N)
    int64_t out_off;      // offset of this pixel's pmf in the packed output
    int32_t index;        // position of the pixel in the caller's array
    int32_t pad_;
};

// Per-pixel constants of the batch flux phase (K1), formed once per pixel by
// pixel_const_kernel (one thread per pixel) and read by every thread of the
// block that takes the pixel.  They are FP64 transcendentals and quotients;
// this GPU runs FP64 at 1/64 of the FP32 rate, so forming them in every
// thread of a block cost as much as a dense pass.
struct PixelConst {
    double Phi0, Lambda, gnorm, delta, beta, inv_sigma, bg;
    double bgK_lo, bgK_hi;   // bg exp(Lambda/2 - S G) left / right of the pulse (G = -Phi0, 1 - Phi0)
    double half_z;           // Delta / (2 sigma)
    double tail_ratio;       // 2 sinh(beta/2) / beta (1 if beta = 0): bin-integrated / point tail weight
    double g0, q1, q64;      // exp(-beta/2), exp(-beta), exp(-64 beta): the geometric factor tables
    float bg_f, uK_lo, uK_hi, eL;   // uK: tail row factors exp(S G - Lambda/2) for B = 0; eL = exp(-Lambda)
    int32_t j_lo, j_hi;      // bins with |z| <= 9 (the pulse); the rest are tail bins
    int32_t pad0_, pad1_;
};

// Per-pixel result record written by the kernels (mirrors spl_report_t).
struct ReportDev {
    int32_t iters;
    int32_t status;
    float last_step_l1;
    float err_bound;
    float lambda2_abs;
    float lambda2_phase;
};

// Status codes used on the device (same values as spl_status_t).
enum : int32_t { ST_OK = 0, ST_ENOCONV = 4, ST_ETIMEOUT = 5 };

// ---------------------------------------------------------------- a2: flux, FP64

// Standard normal CDF via erfc (relative accuracy in both tails).
__device__ __forceinline__ double std_cdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752440); }

// Beyond |z| = 9 the Gaussian CDF is 0 or 1 to below 1.2e-19 and its density
// below 1.1e-18, far under FP64 resolution of F (>= B s_j / t_r) and of
// lambda (>= B / t_r) for every admissible pixel, so the erfc/exp is skipped.
constexpr double kTailZ = 9.0;

struct FluxConst {
    double Phi0;          // Phi(-tau / sigma)
    double Lambda;        // F(t_r), flux of one period (Theorem 1)
    double gnorm;         // 1 / (sigma sqrt(2 pi))
    double delta;         // t_r / N
};

__device__ __forceinline__ FluxConst flux_const(const PixelDev &p) {
    FluxConst c;
    c.Phi0 = std_cdf(-p.tau / p.sigma);
    const double zr = (p.t_r - p.tau) / p.sigma;
    const double Phir = (zr > kTailZ) ? 1.0 : std_cdf(zr);
    c.Lambda = p.S * (Phir - c.Phi0) + p.B;
    c.gnorm = 0.39894228040143267794 / p.sigma;
    c.delta = p.t_r / (double)p.N;
    return c;
}

// The constants above for one pixel (FP64).  Outside the pulse (|z| > 9)
// exp(Lambda/2 - F_j) splits into exp(Lambda/2 - S G) with G one of two
// constants, times exp(-B (j + 1/2) / N), a geometric sequence.
__device__ __forceinline__ void pixel_const(const PixelDev &p, PixelConst &c) {
    const FluxConst fc = flux_const(p);
    c.Phi0 = fc.Phi0;
    c.Lambda = fc.Lambda;
    c.gnorm = fc.gnorm;
    c.delta = fc.delta;
    c.beta = p.B / (double)p.N;
    c.inv_sigma = 1.0 / p.sigma;
    c.bg = p.B / p.t_r;
    c.bgK_lo = c.bg * exp(0.5 * fc.Lambda + p.S * fc.Phi0);
    c.bgK_hi = c.bg * exp(0.5 * fc.Lambda - p.S * (1.0 - fc.Phi0));
    c.half_z = 0.5 * fc.delta * c.inv_sigma;
    c.tail_ratio = c.beta > 0.0 ? 2.0 * sinh(0.5 * c.beta) / c.beta : 1.0;
    c.g0 = exp(-0.5 * c.beta);
    c.q1 = exp(-c.beta);
    c.q64 = exp(-64.0 * c.beta);
    c.bg_f = (float)c.bg;
    c.uK_lo = (float)exp(-0.5 * fc.Lambda - p.S * fc.Phi0);
    c.uK_hi = (float)exp(p.S * (1.0 - fc.Phi0) - 0.5 * fc.Lambda);
    c.eL = (float)exp(-fc.Lambda);
    // pulse bins: s_j within 9 sigma of tau, j in [(tau - 9 sigma)/Delta - 1/2, (tau + 9 sigma)/Delta - 1/2]
    const double lo = (p.tau - kTailZ * p.sigma) / fc.delta - 0.5;
    const double hi = (p.tau + kTailZ * p.sigma) / fc.delta - 0.5;
    c.j_lo = lo < 0.0 ? 0 : (int)ceil(lo);
    c.j_hi = hi >= (double)(p.N - 1) ? p.N - 1 : (int)floor(hi);
    c.pad0_ = c.pad1_ = 0;
}

// x^e for an integer e >= 0 by repeated squaring (FP64 products only).
__host__ __device__ __forceinline__ double pow_uint(double x, int e) {
    double r = 1.0;
    while (e > 0) {
        if (e & 1) r *= x;
        x *= x;
        e >>= 1;
    }
    return r;
}

// exp(x) for |x| <= 700 in FP64 operations only: x = n ln 2 + r with n the
// nearest integer to x / ln 2 and |r| <= ln(2)/2 (one fused multiply-add, so
// the only error of r is that of the rounded ln 2 times n, about
// n 2.7e-17), then e^r by its Taylor series to degree 10 (remainder below
// 3e-13 relative) and 2^n exactly.  About 14 FP64 operations against about
// twice that for a general-purpose exp; accurate to about 1e-12 relative
// over the arguments the flux factors use (|x| <= 125).
__host__ __device__ __forceinline__ double exp_series(double x) {
    constexpr double kLn2 = 0.69314718055994530942;
    constexpr double kInvLn2 = 1.44269504088896340736;
    const double n = rint(x * kInvLn2);
    const double r = fma(-n, kLn2, x);
    // 1/k! for k = 10 .. 0, Horner
    double q = 1.0 / 3628800.0;
    q = fma(q, r, 1.0 / 362880.0);
    q = fma(q, r, 1.0 / 40320.0);
    q = fma(q, r, 1.0 / 5040.0);
    q = fma(q, r, 1.0 / 720.0);
    q = fma(q, r, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    q = fma(q, r, 1.0);
    return ldexp(q, (int)n);
}

// Eq. 1 flux lambda(s_j) and Theorem 1's F(s_j) = S [Phi(z_j) - Phi(z_0)] + B s_j / t_r.
__device__ __forceinline__ void flux_bin(const PixelDev &p, const FluxConst &c, int j,
                                         double &F, double &lam) {
    const double s = ((double)j + 0.5) * c.delta;
    const double z = (s - p.tau) / p.sigma;
    double G, g;
    if (fabs(z) <= kTailZ) {
        G = std_cdf(z) - c.Phi0;
        g = exp(-0.5 * z * z) * c.gnorm;
    } else {
        G = (z > 0.0 ? 1.0 : 0.0) - c.Phi0;
        g = 0.0;
    }
    F = p.S * G + p.B * (s / p.t_r);
    lam = p.S * g + p.B / p.t_r;
}

// Column and row factors of bin j (see the header comment).
__device__ __forceinline__ void factors_bin(const PixelDev &p, const FluxConst &c, int j,
                                            float &w, float &u) {
    double F, lam;
    flux_bin(p, c, j, F, lam);
    const double e = exp(0.5 * c.Lambda - F);     // exp(Lambda/2 - F_j)
    w = (float)(lam * e);
    u = (float)(1.0 / e);
}

// Bin holding the pulse centre, floor(tau / Delta) clamped to [0, N): the
// origin of the learned warm start's frame (the network's output index i
// corresponds to bin (i + c) mod N).
__host__ __device__ __forceinline__ int mlp_frame_shift(double t_r, double tau, int N) {
    int c = (int)floor(tau * (double)N / t_r);
    c = c < 0 ? 0 : c;
    return c >= N ? N - 1 : c;
}

// ---------------------------------------------------------------- block reductions

template <int NT>
__device__ __forceinline__ float block_sum(float v, float *red) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float t = 0.f;
    if (wid == 0) {
        t = (lane < NW) ? red[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    return red[0];
}

// Sums K values at once (one pass of barriers); results land in out[0..K).
template <int NT, int K>
__device__ __forceinline__ void block_sum_k(float (&v)[K], float *red /* >= K * NT/32 */) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * NW + wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = (lane < NW) ? red[k * NW + lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[K * NW + k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[K * NW + k];
}

// One-barrier block reductions: each warp reduces in registers, lane 0
// publishes its partial in buf, one barrier, then every thread adds the
// partials in the same order (identical results in all threads).  The
// caller alternates buffers between consecutive reductions so a buffer is
// never rewritten before every thread has read it.
template <int NT>
__device__ __forceinline__ float block_sum_1bar(float v, float *buf /* NT/32 */) {
    constexpr int NW = NT / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += buf[w];
    return t;
}

template <int NT, int K>
__device__ __forceinline__ void block_sum_k_1bar(float (&v)[K], float *buf /* K * NT/32 */) {
    constexpr int NW = NT / 32;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) buf[k * NW + (threadIdx.x >> 5)] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += buf[k * NW + w];
        v[k] = t;
    }
}

// ---------------------------------------------------------------- stop rule

// Convergence state of one pixel's power iteration.  The error of the
// current iterate pi_k is bounded by the tail sum of the steps,
//   ||pi_k - pi|| <= sum_{m > k} delta_m,
// and the steps decay like |lambda_2|^m with an oscillation of frequency
// arg(lambda_2) (Sec. 4).  |lambda_2| and its phase are estimated from the
// step vectors d_k = pi_k - pi_{k-1} by fitting d_k = a d_{k-1} + b d_{k-2}
// (the roots of z^2 = a z + b are the dominant subdominant eigenvalue pair);
// the decayed envelope of the last W steps, W ~ one oscillation period,
// times rho / (1 - rho), bounds the remaining error.
struct StopState {
    float delta[8];       // last steps (ring, newest at (k-1) & 7)
    float g11, g12, g22;  // <d_{k-1},d_{k-1}>, <d_{k-1},d_{k-2}>, <d_{k-2},d_{k-2}>
    float rho, theta;     // current |lambda_2| and phase estimates (rho < 0: none yet)
    float err;            // last error bound
    float bmin, bmin_prev;  // smallest step of the current and the previous 8-step block
    float tau;            // a priori bound on |lambda_2| (ergodicity coefficient), 1 if unknown
    float rho_floor;      // warm starts: modulus the error estimate never assumes below (0: none)
    int32_t k;            // steps taken
    int32_t reliable;     // 1 once a fit was made on steps well above FP32 noise
};

// Steps above this L1 size are far above the FP32 rounding noise of an
// iterate (about 1e-7 to 4e-7), so a recurrence fit whose basis step
// d_{k-1} is above it is trustworthy.  A reliable fit is only replaced by a
// fit whose newest step is also above kRefitFloor (about 100x the noise): a
// fit on a step a few tens of times the noise can lock onto the rounding
// pattern instead of lambda_2.
constexpr float kFitFloor = 3e-6f;
constexpr float kRefitFloor = 1e-5f;
// Modulus assumed for lambda_2 while no trustworthy fit exists (a start that
// is already within noise of pi).  Over S, B in [0.01, 10] and t_d in
// [20, 150] (t_r = 100) the largest |lambda_2| is about 0.87.
constexpr float kRhoDefault = 0.9f;
// Below this L1 step the step-to-step ratio is dominated by rounding noise
// and is not used to raise the modulus estimate.
constexpr float kRatioFloor = 1e-6f;
// Rounding floor of the map: once the smallest of the last two steps no
// longer falls below a fraction of the smallest of the two before (the
// fraction a decay at the estimated |lambda_2| would give, at least 1/2),
// while the step is below these sizes, the iterate sits on the FP32 floor
// and further steps cannot reduce the error.
constexpr float kStallFloorReliable = 1e-6f;
constexpr float kStallFloor = 3e-7f;
// Long-window floor test.  A start already within noise of pi gives no step
// large enough for a trustworthy fit, and its noise floor can sit just above
// kStallFloor.  Over 8 steps a decay at |lambda_2| <= 0.9 shrinks the
// smallest step of a block to at most 0.43 of the previous block's (to
// rho^8 for a trusted estimate rho); steps below kRefitFloor whose block
// minimum stays above kBlockStall (or rho^4) of the previous one are
// rounding noise.  Below kStallFloorReliable the iterate is within the
// tolerance; above it the FP32 floor is too high for the tolerance, and
// further steps cannot help, so the iteration ends as not converged.
constexpr int kBlock = 8;
constexpr float kBlockStall = 0.7f;
// Warm starts.  A start close to pi can carry almost nothing along the
// slowest mode, so the first steps (and every fit made from them) show only
// faster modes while the slow one still holds an error of up to
// delta rho_s / (1 - rho_s).  For warm starts the estimate therefore never
// assumes a modulus below min(tau, kWarmRhoFloor).  Replayed on 2048 array
// pixels from the network's starts: without it the error at the stop reached
// 8.3e-7 (fits of 0.18-0.35 against |lambda_2| of 0.40-0.59); with 0.5 it
// stays below 4.4e-7 for 6 % more steps.  A uniform start excites every mode,
// so the fit sees the slow one and needs no floor.
constexpr float kWarmRhoFloor = 0.5f;

// Outcomes of stop_update.
enum : int { STOP_CONTINUE = 0, STOP_CONVERGED = 1, STOP_FLOOR = 2 };

// tau: an upper bound on |lambda_2| known before the iteration (Dobrushin's
// ergodicity coefficient, see batch_fused_kernel), or 1 when none is known.
// Every modulus estimate is capped at it, and it replaces kRhoDefault while
// no trustworthy fit exists.  With a bound tau < 1 the error estimate
// delta_k tau / (1 - tau) is rigorous in exact arithmetic: zero-sum vectors
// contract by tau in L1 at every step.
__host__ __device__ __forceinline__ void stop_init(StopState &s, float tau = 1.f, float rho_floor = 0.f) {
#pragma unroll
    for (int i = 0; i < 8; ++i) s.delta[i] = 0.f;
    s.g11 = s.g12 = s.g22 = 0.f;
    s.rho = -1.f;
    s.theta = 0.f;
    s.err = INFINITY;
    s.bmin = INFINITY;
    s.bmin_prev = INFINITY;
    s.tau = tau;
    s.rho_floor = rho_floor;
    s.k = 0;
    s.reliable = 0;
}

// Fit of the 2-term recurrence from the Gram data; returns false if degenerate.
// FP32 throughout: the Gram sums are FP32 already, and the only cancellation
// (det of nearly collinear steps) is routed to the single-mode ratio while
// det / (g11 g22) is still above 1e-3, where FP32 keeps about four digits of
// det; every thread of a block runs this once per step, so the FP64 pipe
// (1/64 of the FP32 rate on this GPU) is kept out of it.
__host__ __device__ __forceinline__ bool fit_lambda2(float g11, float g12, float g22, float h1, float h2,
                                            float &rho, float &theta) {
    if (!(g11 > 0.f) || !(g22 > 0.f)) return false;
    const float det = fmaf(g11, g22, -g12 * g12);
    float a, b;
    // Nearly collinear steps (one real mode dominates, or two close real
    // modes the FP32 Gram data cannot separate): single-mode ratio.
    if (det <= 1e-3f * g11 * g22) {
        a = h1 / g11;
        rho = fabsf(a);
        theta = a >= 0.f ? 0.f : 3.14159265358979f;
        return true;
    }
    const float inv = 1.f / det;
    a = (h1 * g22 - h2 * g12) * inv;
    b = (g11 * h2 - g12 * h1) * inv;
    const float disc = fmaf(a, a, 4.f * b);
    if (disc < 0.f) {
        rho = sqrtf(-b);
        theta = atan2f(sqrtf(-disc), a);
    } else {
        const float sq = sqrtf(disc);
        const float r1 = 0.5f * (a + sq), r2 = 0.5f * (a - sq);
        const float r = fabsf(r1) >= fabsf(r2) ? r1 : r2;
        rho = fabsf(r);
        theta = r >= 0.f ? 0.f : 3.14159265358979f;
    }
    return true;
}

// Consume one step's reductions: delta = ||d_k||_1, dd = <d_k,d_k>,
// d1 = <d_k,d_{k-1}>, d2 = <d_k,d_{k-2}>.  Returns STOP_CONVERGED when the
// bound on the error of pi_k is below tol_err or the iterate sits on an FP32
// floor below the tolerance, STOP_FLOOR when it sits on a floor above it
// (both only once k >= min_iter), else STOP_CONTINUE.
__host__ __device__ __forceinline__ int stop_update(StopState &s, float delta, float dd, float d1, float d2,
                                            float tol_err, int min_iter) {
    s.k += 1;
    const int k = s.k;
    s.delta[(k - 1) & 7] = delta;
    if (k >= 3) {
        const float basis = s.delta[(k - 2) & 7];
        const bool trusted = s.reliable ? (delta > kRefitFloor) : (basis > kFitFloor);
        if (trusted || !s.reliable) {
            float r, th;
            if (fit_lambda2(s.g11, s.g12, s.g22, d1, d2, r, th)) {
                s.rho = r;
                s.theta = th;
                s.reliable = trusted ? 1 : 0;
            }
        }
    }
    // shift the Gram window: new d_{k-1} := d_k, d_{k-2} := d_{k-1}
    s.g22 = s.g11;
    s.g12 = d1;
    s.g11 = dd;
    // With an a priori contraction bound the error of this iterate is at most
    // delta tau / (1 - tau) (the sum of all later steps, each at most tau
    // times the one before): no fit and no minimum step count needed.
    if (s.tau < 1.f && k >= min_iter) {
        const float rig = delta * s.tau / (1.f - s.tau);
        if (rig < tol_err) {
            s.err = rig;
            return STOP_CONVERGED;
        }
    }
    s.bmin = fminf(s.bmin, delta);
    int floor_long = STOP_CONTINUE;
    if (k % kBlock == 0) {
        if (k >= 2 * kBlock && s.bmin < kRefitFloor) {
            const float r2 = s.rho * s.rho;
            const float thr = s.reliable ? fmaxf(kBlockStall, r2 * r2) : kBlockStall;
            if (s.bmin >= thr * s.bmin_prev) floor_long = s.bmin < kStallFloorReliable ? STOP_CONVERGED : STOP_FLOOR;
        }
        s.bmin_prev = s.bmin;
        s.bmin = INFINITY;
    }
    if (k < 3) return STOP_CONTINUE;
    float ru;
    int W = 2;
    const float prev = s.delta[(k - 2) & 7];
    if (s.reliable) {
        ru = s.rho;
        if (prev > 0.f && delta > kRatioFloor) {
            const float ratio = delta / prev;
            if (ratio < 1.f) ru = fmaxf(ru, ratio);
        }
        ru = fminf(fmaxf(fminf(ru, s.tau), 0.05f), 0.9999f);
        if (s.theta >= 0.2f) W = min(8, max(2, (int)ceilf(6.2831853f / s.theta)));
    } else {
        ru = fmaxf(fminf(kRhoDefault, s.tau), 0.05f);
    }
    W = min(W, k);
    float env = 0.f, pw = 1.f;
    for (int m = 0; m < W; ++m) {
        env = fmaxf(env, s.delta[(k - 1 - m) & 7] * pw);
        pw *= ru;
    }
    s.err = env * ru / (1.f - ru);
    if (s.rho_floor > 0.f) {
        const float rf = fminf(s.tau, s.rho_floor);
        s.err = fmaxf(s.err, delta * rf / (1.f - rf));
    }
    if (delta == 0.f) s.err = 0.f;   // exact FP32 fixed point
    bool stalled = false;
    if (k >= 5 && delta < (s.reliable ? kStallFloorReliable : kStallFloor)) {
        const float lo_now = fminf(delta, prev);
        const float lo_old = fminf(s.delta[(k - 3) & 7], s.delta[(k - 4) & 7]);
        // the decay the latest fit predicts over two steps (an untrusted fit
        // still tells a slow mode from noise when the mode dominates)
        const float thr = s.rho >= 0.f ? fmaxf(0.5f, fminf(0.95f, 4.f * s.rho * s.rho)) : 0.5f;
        stalled = lo_now >= thr * lo_old;
    }
    if (k < min_iter) return STOP_CONTINUE;
    if (s.err < tol_err || stalled) return STOP_CONVERGED;
    return floor_long;
}

// ---------------------------------------------------------------- bounded waits

// Spin limit for any device-side wait (mbarrier phases, flags).
constexpr uint32_t kSpinLimit = 1u << 26;

}  // namespace spl
