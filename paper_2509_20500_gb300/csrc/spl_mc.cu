// K9: event-level Monte Carlo of the dead-time-filtered timestamp process on
// the GPU: the Monte Carlo reference of Sec. 5 (Fig. 3b and 3c), a
// free-running SPAD (Sec. 2.2) observed over many laser cycles.
//
// The experiment is specified exactly, so that its histograms can be checked
// bin by bin against an independent implementation drawing the same numbers:
//   - random words: Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel
//     random numbers: as easy as 1, 2, 3", SC 2011), key (seed, k 2^32 + r)
//     for run r of pixel k, counter (cycle, block, 0, 0); the four words of a
//     block are used in order, block after block, restarting at block 0 each
//     cycle; word w gives the uniform u = ((w >> 11) + 1/2) 2^-53;
//   - per cycle: a Poisson(S) signal count by inversion of one uniform
//     (sequential search of the CDF from exp(-S), term recurrence
//     p <- (p S) / k, at most kCap); each signal photon at
//     tau + sigma sqrt(-2 ln u1) cos(2 pi u2), kept if inside [0, t_r) (the
//     pulse of Eq. 1 lives on one period); then a Poisson(B) background count
//     the same way, each background photon at u t_r;
//   - the cycle's photons in increasing time (stable: signal before
//     background on ties) pass the non-paralysable dead-time filter: a photon
//     at t registers if t >= ready, then ready = t + t_d; ready is kept
//     relative to the current cycle's start (minus t_r at each new cycle) and
//     starts at -infinity;
//   - a registration at t counts in bin floor(t N / t_r), at most N - 1.
// All arithmetic is FP64 and written with explicit round-to-nearest
// operations, so no multiply-add is contracted.
//
// One thread simulates one (pixel, run) stream over all its cycles; its
// histogram lives in shared memory until the run ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "spl.h"
#include "spl_kernels.h"

using namespace spl;

namespace {

constexpr int kCap = 64;                 // photons per source and cycle
constexpr int kMaxArrivals = 2 * kCap;
constexpr double kMaxMean = 16.0;        // P(Poisson(16) > 64) < 1e-18
constexpr int kMcMaxBins = 16384;
constexpr int kHistSmemBytes = 128 * 1024;

struct McPixel {
    double t_r, t_d, tau, sigma, S, B;
    int32_t N, pad_;
    int64_t out;                          // first bin of run 0 in the output
};

// Philox4x64-10: ten rounds of two 64 x 64 -> 128-bit products, the key
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x64(uint64_t &c0, uint64_t &c1, uint64_t &c2, uint64_t &c3, uint64_t k0,
                                           uint64_t k1) {
    constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
    constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t lo0 = kM0 * c0, hi0 = __umul64hi(kM0, c0);
        const uint64_t lo1 = kM1 * c2, hi1 = __umul64hi(kM1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += kW0;
        k1 += kW1;
    }
}

struct Stream {
    uint64_t k0, k1, cycle, block;
    uint64_t w0, w1, w2, w3;
    int pos;

    __device__ __forceinline__ void start_cycle(uint64_t c) {
        cycle = c;
        block = 0;
        pos = 4;
    }
    __device__ __forceinline__ double uniform() {
        if (pos == 4) {
            uint64_t c0 = cycle, c1 = block, c2 = 0, c3 = 0;
            philox4x64(c0, c1, c2, c3, k0, k1);
            w0 = c0;
            w1 = c1;
            w2 = c2;
            w3 = c3;
            block += 1;
            pos = 0;
        }
        const uint64_t w = pos == 0 ? w0 : (pos == 1 ? w1 : (pos == 2 ? w2 : w3));
        pos += 1;
        constexpr double kTwoM53 = 1.0 / 9007199254740992.0;
        return __dmul_rn(__dadd_rn((double)(w >> 11), 0.5), kTwoM53);
    }
};

__device__ __forceinline__ int poisson_inv(double mean, double u) {
    double p = exp(-mean), F = p;
    int k = 0;
    while (u > F && k < kCap) {
        k += 1;
        p = __ddiv_rn(__dmul_rn(p, mean), (double)k);
        F = __dadd_rn(F, p);
    }
    return k;
}

__global__ void __launch_bounds__(32) mc_kernel(const McPixel *__restrict__ px, int n, int runs, int64_t cycles,
                                                uint64_t seed, int nmax, uint32_t *__restrict__ hist) {
    extern __shared__ uint32_t sh_hist[];
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= (int64_t)n * runs) return;   // no block-wide synchronisation below
    const int k = (int)(item / runs), r = (int)(item % runs);
    const McPixel p = px[k];
    const int N = p.N;
    uint32_t *h = sh_hist + (size_t)threadIdx.x * nmax;
    for (int b = 0; b < N; ++b) h[b] = 0u;

    constexpr double kPi = 3.14159265358979323846;
    const double two_pi = 2.0 * kPi;
    Stream s;
    s.k0 = seed;
    s.k1 = ((uint64_t)k << 32) | (uint64_t)r;
    double ready = -INFINITY;
    double t[kMaxArrivals];
    for (int64_t c = 0; c < cycles; ++c) {
        s.start_cycle((uint64_t)c);
        int na = 0;
        const int ns = poisson_inv(p.S, s.uniform());
        for (int i = 0; i < ns; ++i) {
            const double u1 = s.uniform(), u2 = s.uniform();
            const double z = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, log(u1))), cos(__dmul_rn(two_pi, u2)));
            const double x = __dadd_rn(p.tau, __dmul_rn(p.sigma, z));
            if (x >= 0.0 && x < p.t_r) t[na++] = x;
        }
        const int nb = poisson_inv(p.B, s.uniform());
        for (int i = 0; i < nb; ++i) t[na++] = __dmul_rn(s.uniform(), p.t_r);
        // stable insertion sort (na <= 2 kCap)
        for (int i = 1; i < na; ++i) {
            const double x = t[i];
            int j = i - 1;
            while (j >= 0 && t[j] > x) {
                t[j + 1] = t[j];
                --j;
            }
            t[j + 1] = x;
        }
        for (int i = 0; i < na; ++i) {
            const double x = t[i];
            if (x >= ready) {
                int b = (int)__ddiv_rn(__dmul_rn(x, (double)N), p.t_r);
                b = b > N - 1 ? N - 1 : b;
                h[b] += 1u;
                ready = __dadd_rn(x, p.t_d);
            }
        }
        ready = __dsub_rn(ready, p.t_r);
    }
    uint32_t *out = hist + p.out + (int64_t)r * N;
    for (int b = 0; b < N; ++b) out[b] = h[b];
}

bool valid(const spl_pixel_t &p) {
    if (!(std::isfinite(p.t_r) && std::isfinite(p.t_d) && std::isfinite(p.tau) && std::isfinite(p.sigma) &&
          std::isfinite(p.S) && std::isfinite(p.B)))
        return false;
    if (p.n_bins < 2 || p.n_bins > kMcMaxBins) return false;
    if (!(p.t_r > 0.0) || !(p.sigma > 0.0) || p.t_d < 0.0) return false;
    if (p.S < 0.0 || p.B < 0.0 || p.S > kMaxMean || p.B > kMaxMean || !(p.S + p.B > 0.0)) return false;
    if (p.tau < 0.0 || p.tau >= p.t_r) return false;
    return true;
}

}  // namespace

extern "C" spl_status_t spl_mc_histograms(const spl_pixel_t *h_pixels, int32_t n, int32_t runs, int64_t cycles,
                                          uint64_t seed, uint32_t *d_hist, void *stream) {
    if (!h_pixels || !d_hist || n < 1 || runs < 1 || cycles < 1) return SPL_EINVAL;
    if ((int64_t)n * runs > INT32_MAX) return SPL_EINVAL;
    std::vector<McPixel> px((size_t)n);
    int64_t off = 0;
    int nmax = 0;
    for (int32_t k = 0; k < n; ++k) {
        const spl_pixel_t &q = h_pixels[k];
        if (!valid(q)) return SPL_EINVAL;
        McPixel &d = px[(size_t)k];
        d.t_r = q.t_r;
        d.t_d = q.t_d;
        d.tau = q.tau;
        d.sigma = q.sigma;
        d.S = q.S;
        d.B = q.B;
        d.N = q.n_bins;
        d.pad_ = 0;
        d.out = (int64_t)runs * off;
        off += q.n_bins;
        nmax = std::max(nmax, (int)q.n_bins);
    }
    const int threads = std::max(1, std::min(32, kHistSmemBytes / (4 * nmax)));
    const size_t smem = (size_t)threads * nmax * sizeof(uint32_t);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaFuncSetAttribute(mc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return note_cuda_error(e, "mc smem attribute");
    McPixel *d_px = nullptr;
    if ((e = cudaMalloc(&d_px, sizeof(McPixel) * px.size())) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : note_cuda_error(e, "mc pixels");
    e = cudaMemcpyAsync(d_px, px.data(), sizeof(McPixel) * px.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int64_t items = (int64_t)n * runs;
        const int grid = (int)((items + threads - 1) / threads);
        mc_kernel<<<grid, threads, smem, s>>>(d_px, n, runs, cycles, seed, nmax, d_hist);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaError_t ef = cudaFree(d_px);
    if (e != cudaSuccess) return note_cuda_error(e, "mc kernel");
    if (ef != cudaSuccess) return note_cuda_error(ef, "mc free");
    return SPL_OK;
}
