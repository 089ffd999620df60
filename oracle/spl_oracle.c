/*
 * FP64 CPU oracle for the dead-time Markov chain of asynchronous single-photon
 * LiDAR timestamps ("Real-Time Markov Modeling for Single-Photon LiDAR",
 * arXiv 2509.20500).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no source, header, table or constant with the CUDA library.
 *
 * Everything is FP64.  A pixel is described by theta = {t_r, t_d, tau, sigma,
 * S, B} (Sec. 2.1, Eq. 1) and the number of bins N (n_b, Sec. 2.3).  Times are
 * all in one unit (ns in the workloads).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - bins are 0-based with centres s_j = (j + 1/2) Delta, Delta = t_r / N
 *    (state set of Sec. 2.3, operator D of Sec. 3.1);
 *  - the Gaussian pulse of Eq. 1 lives on one period [0, t_r) and is not
 *    renormalised after truncation, so Lambda := F(t_r), the exact flux of one
 *    period of the periodic replica used in Eq. 3;
 *  - in b of Eq. 3 the discretised rearm point D(a) enters the ceiling;
 *  - q = fmod(t_d, t_r) * N / t_r is evaluated in that order in IEEE FP64,
 *    so that integer dead-time shifts are exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#ifndef M_SQRT2
#define M_SQRT2 1.41421356237309504880
#endif

/* theta layout used by every entry point of this file */
enum { TH_TR = 0, TH_TD = 1, TH_TAU = 2, TH_SIGMA = 3, TH_S = 4, TH_B = 5 };

/* Standard normal CDF written with erfc so both tails keep relative accuracy. */
static double std_normal_cdf(double z) { return 0.5 * erfc(-z / M_SQRT2); }

/* Eq. 1: lambda(t) = S * N(t; tau, sigma^2) + B / t_r on one period.
 * (s(t) = E * N(t; 0, sigma_t^2), S = alpha E, B = t_r lambda_b.) */
double oracle_lambda(const double *th, double t)
{
    const double z = (t - th[TH_TAU]) / th[TH_SIGMA];
    const double gauss = exp(-0.5 * z * z) / (th[TH_SIGMA] * sqrt(2.0 * M_PI));
    return th[TH_S] * gauss + th[TH_B] / th[TH_TR];
}

/* Theorem 1: F(t) = int_0^t lambda, for t in [0, t_r], in closed form:
 * S [Phi((t - tau)/sigma) - Phi(-tau/sigma)] + B t / t_r. */
double oracle_F(const double *th, double t)
{
    const double sig = th[TH_SIGMA], tau = th[TH_TAU];
    return th[TH_S] * (std_normal_cdf((t - tau) / sig) - std_normal_cdf(-tau / sig))
         + th[TH_B] * t / th[TH_TR];
}

/* Flux of one period of the periodic replica lambda~ (Eq. 3). */
double oracle_Lambda(const double *th) { return oracle_F(th, th[TH_TR]); }

/* Cumulative flux of lambda~ up to time (period * t_r + s_k): every whole
 * period contributes Lambda, the partial period F(s_k). */
static double F_periodic(const double *th, double Lambda, int64_t period, double s_k)
{
    return (double)period * Lambda + oracle_F(th, s_k);
}

/* Relative dead time in units of bins: q = (t_d mod t_r) / Delta, written as
 * fmod(t_d, t_r) * N / t_r (x_d of Eq. 3, Delta of Sec. 2.3). */
double oracle_q(const double *th, int32_t N)
{
    const double x_d = fmod(th[TH_TD], th[TH_TR]);
    return x_d * (double)N / th[TH_TR];
}

/* Theorem 2's quantise-then-shift offset l = ceil(x_d / Delta). */
int64_t oracle_shift_l(const double *th, int32_t N)
{
    return (int64_t)ceil(oracle_q(th, N));
}

static int64_t floor_div(int64_t a, int64_t n) { int64_t d = a / n; if ((a % n) && ((a < 0) != (n < 0))) --d; return d; }
static int64_t ceil_div(int64_t a, int64_t n) { return -floor_div(-a, n); }

/*
 * Rapp's sequential construction (Eq. 3 discretised as Eq. 4).  For every
 * state pair (s_i, s_j), with s_i the current and s_j the next timestamp:
 *   a    = s_i + x_d                          (rearm point, Eq. 3)
 *   D(a) = (ceil(a / Delta) - 1/2) Delta      (operator D, Sec. 3.1)
 *   b    = ceil((D(a) - s_j) / t_r) t_r + s_j (first time >= D(a) congruent
 *                                              to s_j modulo t_r, Eq. 3)
 *   E_ij = exp(-int_{D(a)}^{D(b)} lambda~),   D(b) = b
 *   P_ij = lambda(s_j) E_ij / (1 - exp(-Lambda))
 * Times past one period are kept as (period, bin) pairs so the ceilings are
 * integer arithmetic: a / Delta = i + 1/2 + q, so D(a) sits on bin index
 * n_a = ceil(i + 1/2 + q) - 1 of the unrolled time axis, and
 * (D(a) - s_j) / t_r = (n_a - j) / N.
 * Writes the unnormalised N x N matrix, row-major.
 */
void oracle_build_seq(const double *th, int32_t N, double *P)
{
    const double t_r = th[TH_TR];
    const double Delta = t_r / (double)N;
    const double Lambda = oracle_Lambda(th);
    const double norm = -expm1(-Lambda);            /* 1 - exp(-Lambda) */
    const double q = oracle_q(th, N);
    for (int64_t i = 0; i < N; ++i) {
        const int64_t n_a = (int64_t)ceil((double)i + 0.5 + q) - 1;
        const int64_t a_period = floor_div(n_a, N);
        const int64_t a_bin = n_a - a_period * N;
        const double s_a = ((double)a_bin + 0.5) * Delta;
        const double F_a = F_periodic(th, Lambda, a_period, s_a);
        for (int64_t j = 0; j < N; ++j) {
            const double s_j = ((double)j + 0.5) * Delta;
            const int64_t b_period = ceil_div(n_a - j, N);
            const double F_b = F_periodic(th, Lambda, b_period, s_j);
            const double E = exp(-(F_b - F_a));
            P[i * N + j] = oracle_lambda(th, s_j) * E / norm;
        }
    }
}

/*
 * The paper's reparameterised construction (Eq. 6, Sec. 3.4): with
 * p_i = (i + shift) mod N the row of E_base that row i takes after the
 * dead-time roll J_l,
 *   E_ij = exp(-Lambda 1{s_p > s_j} - F(s_j) + F(s_p)),  P_ij = lambda_j E_ij.
 * Same normalising constant as the sequential form.  shift = l = ceil(q) is
 * Theorem 2; shift = ceil(q + 1/2) - 1 reproduces shift-then-quantise exactly.
 */
void oracle_build_reparam(const double *th, int32_t N, int64_t shift, double *P)
{
    const double Delta = th[TH_TR] / (double)N;
    const double Lambda = oracle_Lambda(th);
    const double norm = -expm1(-Lambda);
    int64_t sh = shift % N; if (sh < 0) sh += N;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t p = (i + sh) % N;
        const double F_p = oracle_F(th, ((double)p + 0.5) * Delta);
        for (int64_t j = 0; j < N; ++j) {
            const double s_j = ((double)j + 0.5) * Delta;
            const double ind = (p > j) ? 1.0 : 0.0;
            const double E = exp(-Lambda * ind - oracle_F(th, s_j) + F_p);
            P[i * N + j] = oracle_lambda(th, s_j) * E / norm;
        }
    }
}

/*
 * Bin-integrated variant of Eq. 6 (an ablation beyond the paper, which takes
 * the point flux lambda(s_j) at the bin centre, Sec. 3.4).  Entry (i, j) is
 * the probability, for a detector re-armed at the centre s_p of bin
 * p = (i + shift) mod N, that its next registration falls anywhere in bin
 * j = [j Delta, (j+1) Delta): the exact integral of lambda(t) exp(-(F(t) - F(s_p)))
 * over the bin, i.e. exp(F(s_p) - F(j Delta)) - exp(F(s_p) - F((j+1) Delta)),
 * times exp(-Lambda) when the bin is only reached after the period wraps
 * (p > j).  The point form is this integral by the midpoint rule.  Same
 * unnormalised scale as oracle_build_reparam (divided by 1 - exp(-Lambda)
 * and by Delta).
 */
void oracle_build_binint(const double *th, int32_t N, int64_t shift, double *P)
{
    const double Delta = th[TH_TR] / (double)N;
    const double Lambda = oracle_Lambda(th);
    const double norm = -expm1(-Lambda) * Delta;
    int64_t sh = shift % N; if (sh < 0) sh += N;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t p = (i + sh) % N;
        const double F_p = oracle_F(th, ((double)p + 0.5) * Delta);
        for (int64_t j = 0; j < N; ++j) {
            const double F_lo = oracle_F(th, (double)j * Delta);
            const double F_hi = oracle_F(th, (double)(j + 1) * Delta);
            const double wrap = (p > j) ? exp(-Lambda) : 1.0;
            P[i * N + j] = wrap * exp(F_p - F_lo) * -expm1(F_lo - F_hi) / norm;
        }
    }
}

/* Row normalisation P -> P~ (Sec. 2.3).  Returns 0, or -1 on a zero row. */
int oracle_normalize_rows(int32_t N, double *P)
{
    for (int64_t i = 0; i < N; ++i) {
        double r = 0.0;
        for (int64_t j = 0; j < N; ++j) r += P[i * N + j];
        if (!(r > 0.0)) return -1;
        for (int64_t j = 0; j < N; ++j) P[i * N + j] /= r;
    }
    return 0;
}

/*
 * Dense power iteration for the leading left eigenvector, pi P~ = pi
 * (Sec. 2.3): y_j = sum_i pi_i P~_ij, y /= sum(y), step = ||y - pi||_1.
 * Starts from pi_start if given (normalised here), else the uniform vector.
 * Stops when step < tol.  Returns the number of steps taken, or -1 if
 * max_iter steps did not reach tol (pi_out still holds the last iterate).
 */
int oracle_power(int32_t N, const double *Pt, double tol, int32_t max_iter,
                 const double *pi_start, double *pi_out, double *last_step)
{
    double *pi = (double *)malloc(sizeof(double) * (size_t)N);
    double *y = (double *)malloc(sizeof(double) * (size_t)N);
    if (!pi || !y) { free(pi); free(y); return -2; }
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) { pi[i] = pi_start ? pi_start[i] : 1.0; s += pi[i]; }
    for (int64_t i = 0; i < N; ++i) pi[i] /= s;
    int it = 0, done = 0;
    double step = INFINITY;
    while (it < max_iter) {
        for (int64_t j = 0; j < N; ++j) y[j] = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            const double c = pi[i];
            const double *row = Pt + i * N;
            for (int64_t j = 0; j < N; ++j) y[j] += c * row[j];
        }
        double sy = 0.0;
        for (int64_t j = 0; j < N; ++j) sy += y[j];
        step = 0.0;
        for (int64_t j = 0; j < N; ++j) { y[j] /= sy; step += fabs(y[j] - pi[j]); }
        double *t = pi; pi = y; y = t;
        ++it;
        if (step < tol) { done = 1; break; }
    }
    memcpy(pi_out, pi, sizeof(double) * (size_t)N);
    if (last_step) *last_step = step;
    free(pi); free(y);
    return done ? it : -1;
}

/*
 * Stationary pmf of one pixel: sequential build (shift_mode 0), or the
 * reparameterised build with an explicit row shift (shift_mode 1, shift
 * given), then normalisation and power iteration to tol from the uniform
 * vector.  Returns the iteration count (or a negative status).
 */
int oracle_stationary(const double *th, int32_t N, int32_t shift_mode, int64_t shift,
                      double tol, int32_t max_iter, double *pi_out)
{
    double *P = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
    if (!P) return -2;
    if (shift_mode == 0) oracle_build_seq(th, N, P);
    else if (shift_mode == 2) oracle_build_binint(th, N, shift, P);
    else oracle_build_reparam(th, N, shift, P);
    if (oracle_normalize_rows(N, P) != 0) { free(P); return -3; }
    int it = oracle_power(N, P, tol, max_iter, NULL, pi_out, NULL);
    free(P);
    return it;
}

/* Batch of pixels over host threads (one pixel per task).  thetas is [n][6],
 * Ns is [n], outputs are packed at offsets[k] (int64, [n + 1]).  iters_out[k]
 * receives each pixel's return value. */
typedef struct {
    const double *thetas; const int32_t *Ns; const int64_t *offsets;
    int32_t n; double tol; int32_t max_iter; double *out; int32_t *iters_out;
    int32_t next; pthread_mutex_t lock;
} batch_job_t;

static void *batch_worker(void *arg)
{
    batch_job_t *job = (batch_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        const int32_t k = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (k >= job->n) break;
        job->iters_out[k] = oracle_stationary(job->thetas + 6 * (int64_t)k, job->Ns[k], 0, 0,
                                              job->tol, job->max_iter, job->out + job->offsets[k]);
    }
    return NULL;
}

int oracle_batch_stationary(const double *thetas, const int32_t *Ns, int32_t n,
                            const int64_t *offsets, double tol, int32_t max_iter,
                            int32_t nthreads, double *out, int32_t *iters_out)
{
    batch_job_t job;
    job.thetas = thetas; job.Ns = Ns; job.offsets = offsets; job.n = n; job.tol = tol;
    job.max_iter = max_iter; job.out = out; job.iters_out = iters_out; job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *tids = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&tids[t], NULL, batch_worker, &job) == 0) ++started;
    if (started == 0) batch_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(tids[t], NULL);
    free(tids);
    pthread_mutex_destroy(&job.lock);
    return started;
}

/*
 * Event-level dead-time filter for the Monte Carlo ground truth (Sec. 2.2 and
 * Sec. 3.5): given sorted absolute photon arrival times T[0..n), a free-running
 * non-paralysable detector registers the first arrival and then every first
 * arrival at or after the previous registration plus t_d.  Writes the indices
 * of registered arrivals and returns their count.
 */
int64_t oracle_mc_deadtime(const double *T, int64_t n, double t_d, int64_t *idx_out)
{
    int64_t m = 0;
    double ready = -INFINITY;
    for (int64_t k = 0; k < n; ++k) {
        if (T[k] >= ready) { idx_out[m++] = k; ready = T[k] + t_d; }
    }
    return m;
}

/*
 * Counter-based event Monte Carlo: the Monte Carlo reference of Sec. 5
 * (Fig. 3b/3c) as an exactly specified random experiment, so that a GPU
 * implementation drawing the same numbers can be compared bin by bin.
 *
 * Random words: Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of two 64x64->128
 * multiplications on a 4-word counter with a 2-word key bumped by the Weyl
 * constants between rounds.
 *
 * The experiment for pixel k (theta, N) and run r:
 *   key = (seed, k * 2^32 + r); the uniforms of cycle c are the words of
 *   Philox(counter = (c, b, 0, 0)), b = 0, 1, ..., consumed in order, each
 *   mapped to u = ((w >> 11) + 1/2) 2^-53 in (0, 1).
 *   Per cycle: n_s = Poisson(S) by inversion of one uniform (sequential CDF
 *   search from exp(-S), term recurrence p <- (p * S) / k, at most 64); n_s
 *   signal photons t = tau + sigma * sqrt(-2 ln u1) cos(2 pi u2), kept if
 *   0 <= t < t_r (the pulse of Eq. 1 truncated to one period); then
 *   n_b = Poisson(B) the same way and n_b background photons t = u t_r.
 *   Arrivals are sorted (stable: signal before background on ties) and pass
 *   the non-paralysable dead-time filter of Sec. 2.2: a photon at t registers
 *   if t >= ready (time relative to this cycle's start), then ready = t + t_d;
 *   ready carries over to the next cycle as ready - t_r, and starts at -inf.
 *   A registration at t counts in bin floor(t N / t_r) (clamped to N - 1).
 * All arithmetic is FP64 with no contraction.
 */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL, PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL, PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void oracle_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out)
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        const unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        const unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint64_t key[2];
    uint64_t cycle, block;
    uint64_t buf[4];
    int pos;
} mc_stream_t;

static double mc_uniform(mc_stream_t *s)
{
    if (s->pos == 4) {
        const uint64_t ctr[4] = {s->cycle, s->block, 0, 0};
        oracle_philox4x64(ctr, s->key, s->buf);
        s->block += 1;
        s->pos = 0;
    }
    const uint64_t w = s->buf[s->pos++];
    return ((double)(w >> 11) + 0.5) * 0x1p-53;
}

enum { MC_CAP = 64 };

static int mc_poisson(double mean, double u)
{
    double p = exp(-mean), F = p;
    int k = 0;
    while (u > F && k < MC_CAP) {
        k += 1;
        p = (p * mean) / (double)k;
        F = F + p;
    }
    return k;
}

/* One run: cycles laser cycles of pixel k, histogram added into hist[N]. */
static void mc_run(const double *th, int N, uint64_t seed, uint64_t k, uint64_t r, int64_t cycles,
                   uint32_t *hist)
{
    const double t_r = th[TH_TR], t_d = th[TH_TD], tau = th[TH_TAU], sigma = th[TH_SIGMA];
    const double S = th[TH_S], B = th[TH_B];
    const double two_pi = 2.0 * M_PI;
    mc_stream_t s;
    s.key[0] = seed;
    s.key[1] = (k << 32) | r;
    double ready = -INFINITY;
    double t[2 * MC_CAP];
    for (int64_t c = 0; c < cycles; ++c) {
        s.cycle = (uint64_t)c;
        s.block = 0;
        s.pos = 4;
        int n = 0;
        const int ns = mc_poisson(S, mc_uniform(&s));
        for (int i = 0; i < ns; ++i) {
            const double u1 = mc_uniform(&s), u2 = mc_uniform(&s);
            const double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
            const double x = tau + sigma * z;
            if (x >= 0.0 && x < t_r) t[n++] = x;
        }
        const int nb = mc_poisson(B, mc_uniform(&s));
        for (int i = 0; i < nb; ++i) t[n++] = mc_uniform(&s) * t_r;
        /* insertion sort, stable */
        for (int i = 1; i < n; ++i) {
            const double x = t[i];
            int j = i - 1;
            while (j >= 0 && t[j] > x) { t[j + 1] = t[j]; --j; }
            t[j + 1] = x;
        }
        for (int i = 0; i < n; ++i) {
            if (t[i] >= ready) {
                int b = (int)((t[i] * (double)N) / t_r);
                if (b > N - 1) b = N - 1;
                hist[b] += 1;
                ready = t[i] + t_d;
            }
        }
        ready = ready - t_r;
    }
}

typedef struct {
    const double *thetas;
    const int32_t *Ns;
    const int64_t *offsets;
    int32_t n, runs;
    int64_t cycles;
    uint64_t seed;
    uint32_t *hist;
    int64_t next;
    pthread_mutex_t lock;
} mc_job_t;

static void *mc_worker(void *arg)
{
    mc_job_t *job = (mc_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        const int64_t item = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (item >= (int64_t)job->n * job->runs) break;
        const int32_t k = (int32_t)(item / job->runs), r = (int32_t)(item % job->runs);
        const int N = job->Ns[k];
        uint32_t *h = job->hist + (int64_t)job->runs * job->offsets[k] + (int64_t)r * N;
        memset(h, 0, sizeof(uint32_t) * (size_t)N);
        mc_run(job->thetas + 6 * (int64_t)k, N, job->seed, (uint64_t)k, (uint64_t)r, job->cycles, h);
    }
    return NULL;
}

/* Histograms of all (pixel, run) pairs: run r of pixel k at
 * hist[runs * offsets[k] + r * N_k .. + N_k). */
int oracle_mc_philox(const double *thetas, const int32_t *Ns, int32_t n, const int64_t *offsets, int32_t runs,
                     int64_t cycles, uint64_t seed, int32_t nthreads, uint32_t *hist)
{
    mc_job_t job;
    job.thetas = thetas; job.Ns = Ns; job.offsets = offsets; job.n = n; job.runs = runs;
    job.cycles = cycles; job.seed = seed; job.hist = hist; job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *tids = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int i = 0; i < nthreads; ++i)
        if (pthread_create(&tids[i], NULL, mc_worker, &job) == 0) ++started;
    if (started == 0) mc_worker(&job);
    for (int i = 0; i < started; ++i) pthread_join(tids[i], NULL);
    free(tids);
    pthread_mutex_destroy(&job.lock);
    return started;
}

/* One (pixel k, run r) stream of the experiment above, histogram zeroed and
 * filled: for checking sampled runs of a large launch. */
void oracle_mc_philox_run(const double *theta, int32_t N, uint64_t seed, uint64_t k, uint64_t r, int64_t cycles,
                          uint32_t *hist)
{
    memset(hist, 0, sizeof(uint32_t) * (size_t)N);
    mc_run(theta, N, seed, k, r, cycles, hist);
}
