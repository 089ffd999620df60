// libspl C ABI (declared in include/spl.h): validation, the dead-time shift
// (Theorem 2), chain objects, the iteration driver and the batch driver.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <cstdlib>
#include <functional>
#include <map>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "spl_host_pool.h"

#include "spl.h"
#include "spl_kernels.h"

using namespace spl;

namespace {

thread_local char g_cuda_err[256] = "";

}  // namespace

// The last CUDA failure of this thread, for spl_last_cuda_error (every
// translation unit of the library records through here).
spl_status_t spl::note_cuda_error(cudaError_t e, const char *where) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
    return SPL_ECUDA;
}

namespace {

spl_status_t cuda_fail(cudaError_t e, const char *where) { return note_cuda_error(e, where); }

#define SPL_CU(expr)                                                   \
    do {                                                               \
        cudaError_t e_ = (expr);                                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);            \
    } while (0)

bool finite_all(const spl_pixel_t &p) {
    return std::isfinite(p.t_r) && std::isfinite(p.t_d) && std::isfinite(p.tau) && std::isfinite(p.sigma) &&
           std::isfinite(p.S) && std::isfinite(p.B);
}

// Largest Lambda accepted: exp(+-Lambda/2) must stay inside FP32 with room for
// N-term sums (see the factorisation in spl_device.cuh).
constexpr double kLambdaMax = 120.0;
constexpr int32_t kMaxBins = 1 << 24;

}  // namespace

// a1: validate and derive the row shift.  q = fmod(t_d, t_r) * N / t_r is
// evaluated in IEEE FP64 in that order (no contraction: a product then a
// quotient), l = ceil(q) (Theorem 2), reduced modulo N.
spl_status_t spl::make_pixel(const spl_pixel_t &p, PixelDev &d) {
    if (!finite_all(p)) return SPL_EINVAL;
    if (p.n_bins < 2 || p.n_bins > kMaxBins) return SPL_EINVAL;
    if (!(p.t_r > 0.0) || !(p.sigma > 0.0) || p.t_d < 0.0 || p.S < 0.0 || p.B < 0.0) return SPL_EINVAL;
    if (!(p.S + p.B > 0.0)) return SPL_EINVAL;
    if (p.tau < 0.0 || p.tau >= p.t_r) return SPL_EINVAL;
    if (p.S + p.B > kLambdaMax) return SPL_EINVAL;
    if (p.shift_override < -1) return SPL_EINVAL;
    const int32_t N = p.n_bins;
    int64_t l;
    if (p.shift_override >= 0) {
        l = p.shift_override;
    } else {
        // fmod is exact and returns t_d itself when 0 <= t_d < t_r
        const volatile double x_d = p.t_d < p.t_r ? p.t_d : std::fmod(p.t_d, p.t_r);
        const volatile double num = x_d * (double)N;
        const double q = num / p.t_r;
        l = (int64_t)std::ceil(q);
    }
    l %= N;
    if (l < 0) l += N;
    d.t_r = p.t_r;
    d.tau = p.tau;
    d.sigma = p.sigma;
    d.S = p.S;
    d.B = p.B;
    d.N = N;
    d.l = (int32_t)l;
    d.out_off = 0;
    d.index = 0;
    d.pad_ = 0;
    return SPL_OK;
}

namespace {

int num_sms_current() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_tiled() {
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

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

}  // namespace

// ======================================================================
// Chains
// ======================================================================

struct spl_chain {
    PixelDev p{};
    spl_mode_t mode = SPL_FUSED;
    cudaStream_t stream = nullptr;
    int N = 0, vlen = 0, ld = 0;
    // per-bin vectors
    float *w = nullptr, *u = nullptr, *lam = nullptr;
    double *F = nullptr, *scal = nullptr;
    float *rowsum = nullptr, *rho = nullptr;
    // iteration vectors
    float *pi = nullptr, *y = nullptr, *d1 = nullptr, *d2 = nullptr, *v = nullptr;
    float *part = nullptr;
    ChainState *state = nullptr;
    ChainState *h_state = nullptr;   // pinned readback
    int *err_flag = nullptr;
    float *blk = nullptr;            // finish stages' per-CTA partials
    int *ticket = nullptr;           // finish stages' arrival counters
    // materialised
    float *P = nullptr;
    CUtensorMap tmap{};
    int gemv_grid = 0, tiles_per_slab = 0, tiles_per_cta = 0, total_tiles = 0;
    // fused split (row pass at build, standalone pass timing)
    int chunks = 0, chunk = 0, ld_part = 0;
    // fused persistent iteration: grid, tiles, row chunks and its buffers
    int run_grid = 0, run_T = 0, run_RB = 0, run_segs = 0, run_chunk = 0;
    float *run_y = nullptr, *run_vb = nullptr, *run_pi = nullptr, *run_tsum = nullptr, *run_part = nullptr,
          *run_blk = nullptr;
    int *run_ticket = nullptr;
    unsigned *run_bar = nullptr;
    size_t run_part_cap = 0;         // floats of run_part
    size_t run_blk_cap = 0;          // floats of run_blk
    // kGraphSteps power steps captured once as a CUDA graph, replayed per chunk
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t steps_exec = nullptr;
    bool graph_failed = false;
};

// Steps per replay of the captured chunk.  Every kernel returns at once when
// the device state says the iteration is done, so steps issued past the stop
// cost only their launch.
constexpr int kGraphSteps = 8;

static void chain_release(spl_chain *c) {
    if (!c) return;
    void *bufs[] = {c->w, c->u, c->lam, c->F, c->scal, c->rowsum, c->rho, c->pi, c->y,
                    c->d1, c->d2, c->v, c->part, c->state, c->err_flag, c->P, c->blk, c->ticket,
                    c->run_y, c->run_vb, c->run_pi, c->run_tsum, c->run_part, c->run_blk, c->run_ticket,
                    c->run_bar};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->steps_exec) cudaGraphExecDestroy(c->steps_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

static spl_status_t chain_alloc(spl_chain *c) {
    const int N = c->N, vl = c->vlen;
    SPL_CU(dalloc(&c->w, vl));
    SPL_CU(dalloc(&c->u, vl));
    SPL_CU(dalloc(&c->lam, N));
    SPL_CU(dalloc(&c->F, N));
    SPL_CU(dalloc(&c->scal, 2));
    SPL_CU(dalloc(&c->rowsum, N));
    SPL_CU(dalloc(&c->rho, vl));
    SPL_CU(dalloc(&c->pi, N));
    SPL_CU(dalloc(&c->y, N));
    SPL_CU(dalloc(&c->d1, N));
    SPL_CU(dalloc(&c->d2, N));
    SPL_CU(dalloc(&c->v, vl));
    SPL_CU(dalloc(&c->state, 1));
    SPL_CU(dalloc(&c->err_flag, 1));
    SPL_CU(dalloc(&c->blk, finish_blk_floats(vl)));
    SPL_CU(dalloc(&c->ticket, 2));
    SPL_CU(cudaMemset(c->ticket, 0, 2 * sizeof(int)));
    SPL_CU(cudaMallocHost(reinterpret_cast<void **>(&c->h_state), sizeof(ChainState)));
    return SPL_OK;
}

// Split layout for the multi-CTA dense passes: enough CTAs to cover every SM
// a few times with whole 128-entry chunks of the broadcast vector.
static void plan_split(spl_chain *c) {
    const int sms = num_sms_current();
    const int col_tiles = (c->N + split_cols_per_cta() - 1) / split_cols_per_cta();
    const int nblk = c->vlen / 128;
    int chunks = (4 * sms + col_tiles - 1) / col_tiles;
    chunks = std::max(1, std::min(chunks, nblk));
    const int blk_per_chunk = (nblk + chunks - 1) / chunks;
    c->chunk = blk_per_chunk * 128;
    c->chunks = (c->vlen + c->chunk - 1) / c->chunk;
    c->ld_part = c->vlen;
}

// Units [b U / G, (b+1) U / G) of CTA b: the partial slots one CTA needs
// (tiles its range touches) and the largest range.
static void run_partition(long long U, int RB, int G, int *segs, long long *umax) {
    *segs = 1;
    *umax = 0;
    for (int b = 0; b < G; ++b) {
        const long long u0 = (long long)b * U / G, u1 = (long long)(b + 1) * U / G;
        *segs = std::max(*segs, (int)((u1 - 1) / RB - u0 / RB) + 1);
        *umax = std::max(*umax, u1 - u0);
    }
}

// Plan of the persistent fused iteration (host arithmetic only): as many CTAs
// as stay resident (at most one per work unit), the work units (256-column
// tile x 32-row block) split evenly over them, the partial slots one CTA
// needs and the rows it stages at once.
extern "C" spl_status_t spl_chain_run_plan(int32_t n_bins, int32_t sms, int32_t blocks_per_sm, spl_run_plan_t *out) {
    if (!out || n_bins < 2 || n_bins > kMaxBins || sms < 1 || blocks_per_sm < 1) return SPL_EINVAL;
    const int vlen = split_pad_len(n_bins);
    const int T = (n_bins + chain_run_tile_cols() - 1) / chain_run_tile_cols();
    const int RB = vlen / 32;
    const long long U = (long long)T * RB;
    const int G = (int)std::min<long long>(std::min((long long)blocks_per_sm * sms, (long long)chain_run_max_grid()), U);
    int segs = 1;
    long long umax = 0;
    run_partition(U, RB, G, &segs, &umax);
    out->grid = G;
    out->tiles = T;
    out->row_blocks = RB;
    out->segs = segs;
    out->chunk = (int)std::min<long long>(chain_run_max_chunk(), umax * 32);
    out->vlen = vlen;
    return SPL_OK;
}

static spl_status_t plan_run(spl_chain *c) {
    const int bps = std::min(2, chain_run_blocks_per_sm(chain_run_max_chunk()));
    if (bps < 1) return cuda_fail(cudaErrorLaunchOutOfResources, "chain run occupancy");
    spl_run_plan_t pl;
    spl_status_t st = spl_chain_run_plan(c->N, num_sms_current(), bps, &pl);
    if (st != SPL_OK) return st;
    const int T = pl.tiles, G = pl.grid;
    c->run_T = T;
    c->run_RB = pl.row_blocks;
    c->run_segs = pl.segs;
    c->run_chunk = pl.chunk;
    c->run_grid = G;
    SPL_CU(dalloc(&c->run_y, 2 * (size_t)c->vlen));
    SPL_CU(dalloc(&c->run_vb, 2 * (size_t)c->vlen));
    SPL_CU(cudaMemset(c->run_vb, 0, 2 * sizeof(float) * c->vlen));
    SPL_CU(dalloc(&c->run_pi, (size_t)c->N));
    SPL_CU(dalloc(&c->run_tsum, 2 * (size_t)(chain_run_tile_cols() / 32) * T));   // [2][T][warps] tile-sum partials
    c->run_part_cap = (size_t)G * pl.segs * chain_run_tile_cols();
    SPL_CU(dalloc(&c->run_part, c->run_part_cap));
    c->run_blk_cap = 2 * (size_t)G * 4;
    SPL_CU(dalloc(&c->run_blk, c->run_blk_cap));
    SPL_CU(dalloc(&c->run_ticket, (size_t)T));
    SPL_CU(dalloc(&c->run_bar, (size_t)chain_run_bar_words()));
    SPL_CU(cudaMemset(c->run_ticket, 0, sizeof(int) * T));
    SPL_CU(cudaMemset(c->run_bar, 0, sizeof(unsigned) * chain_run_bar_words()));
    return SPL_OK;
}

static ChainRunArgs run_args(spl_chain *c) {
    ChainRunArgs a{};
    a.N = c->N;
    a.vlen = c->vlen;
    a.l = c->p.l;
    a.T = c->run_T;
    a.RB = c->run_RB;
    a.segs = c->run_segs;
    a.chunk = c->run_chunk;
    a.w = c->w;
    a.scal = c->scal;
    a.rho = c->rho;
    a.v0 = c->v;
    a.pi = c->pi;
    a.pi_alt = c->run_pi;
    a.d1 = c->d1;
    a.d2 = c->d2;
    a.y = c->run_y;
    a.vb = c->run_vb;
    a.tsum = c->run_tsum;
    a.part = c->run_part;
    a.blk = c->run_blk;
    a.tile_ticket = c->run_ticket;
    a.bar = c->run_bar;
    a.state = c->state;
    a.err_flag = c->err_flag;
    return a;
}

extern "C" spl_status_t spl_build(const spl_pixel_t *p, spl_mode_t mode, void *stream, spl_chain_t **out) {
    if (!p || !out) return SPL_EINVAL;
    *out = nullptr;
    if (mode != SPL_MATERIALIZED && mode != SPL_FUSED) return SPL_EINVAL;
    PixelDev d;
    spl_status_t st = make_pixel(*p, d);
    if (st != SPL_OK) return st;
    spl_chain *c = new (std::nothrow) spl_chain();
    if (!c) return SPL_ENOMEM;
    c->p = d;
    c->mode = mode;
    c->stream = static_cast<cudaStream_t>(stream);
    c->N = d.N;
    c->vlen = split_pad_len(d.N);
    plan_split(c);
    st = chain_alloc(c);
    if (st != SPL_OK) { chain_release(c); return st; }
    cudaStream_t s = c->stream;
    cudaError_t e = launch_chain_flux(d, c->w, c->u, c->lam, c->F, c->scal, c->vlen, s);
    if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "chain_flux"); }
    if (mode == SPL_MATERIALIZED) {
        const int N = d.N;
        c->ld = (N + 31) / 32 * 32;
        e = dalloc(&c->P, (size_t)N * c->ld);
        if (e != cudaSuccess) { chain_release(c); return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : cuda_fail(e, "P"); }
        e = launch_build_matrix(N, d.l, c->ld, c->w, c->u, c->scal, c->P, c->rowsum, num_sms_current(), s);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "build_matrix"); }
        // TMA descriptor over P: dims {cols, rows}, row pitch ld floats, slab-wide x 32-row boxes.
        const int SC = gemv_slab_cols();
        auto enc = get_encode_tiled();
        if (!enc) { chain_release(c); return cuda_fail(cudaErrorNotSupported, "cuTensorMapEncodeTiled"); }
        cuuint64_t gdim[2] = {(cuuint64_t)N, (cuuint64_t)N};
        cuuint64_t gstride[1] = {(cuuint64_t)c->ld * sizeof(float)};
        cuuint32_t box[2] = {(cuuint32_t)SC, 32};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = enc(&c->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->P, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { chain_release(c); return cuda_fail(cudaErrorInvalidValue, "tensor map encode"); }
        const int slabs = (N + SC - 1) / SC;
        c->tiles_per_slab = (N + 31) / 32;
        c->total_tiles = slabs * c->tiles_per_slab;
        int grid = num_sms_current();
        if (grid < slabs) grid = slabs;
        c->tiles_per_cta = (c->total_tiles + grid - 1) / grid;
        if (c->tiles_per_cta > c->tiles_per_slab) c->tiles_per_cta = c->tiles_per_slab;
        c->gemv_grid = (c->total_tiles + c->tiles_per_cta - 1) / c->tiles_per_cta;
        e = dalloc(&c->part, (size_t)c->gemv_grid * 2 * SC);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "part"); }
        e = cudaMemsetAsync(c->part, 0, sizeof(float) * (size_t)c->gemv_grid * 2 * SC, s);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "memset part"); }
    } else {
        e = dalloc(&c->part, (size_t)c->chunks * c->ld_part);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "part"); }
        // row pass: v = w, per-output factor u
        TriSplitArgs ta{};
        ta.N = d.N;
        ta.vlen = c->vlen;
        ta.chunk = c->chunk;
        ta.v = c->w;
        ta.m = c->u;
        ta.scal = c->scal;
        ta.part = c->part;
        ta.ld_part = c->ld_part;
        ta.state = nullptr;
        e = launch_tri_split(ta, true, c->chunks, s);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "row pass"); }
        e = launch_finish_rows(d.N, c->chunks, c->ld_part, c->part, c->u, c->rho, c->rowsum, d.l, s);
        if (e != cudaSuccess) { chain_release(c); return cuda_fail(e, "finish rows"); }
        st = plan_run(c);
        if (st != SPL_OK) { chain_release(c); return st; }
    }
    *out = c;
    return SPL_OK;
}

static FinishArgs finish_args(spl_chain *c) {
    FinishArgs a{};
    a.mode = c->mode == SPL_MATERIALIZED ? 0 : 1;
    a.N = c->N;
    a.l = c->p.l;
    a.vlen = c->vlen;
    a.tiles_per_slab = c->tiles_per_slab;
    a.tiles_per_cta = c->tiles_per_cta;
    a.nparts = c->chunks;
    a.ld_part = c->ld_part;
    a.part = c->part;
    a.y = c->y;
    a.pi = c->pi;
    a.d1 = c->d1;
    a.d2 = c->d2;
    a.rowsum = c->rowsum;
    a.rho = c->rho;
    a.v = c->v;
    a.state = c->state;
    a.blk = c->blk;
    a.ticket = c->ticket;
    return a;
}

// The dense pass of one power step: GEMV over P, or the regenerated split
// column pass; partial column sums into c->part.
static spl_status_t chain_pass(spl_chain *c, cudaStream_t s) {
    cudaError_t e;
    if (c->mode == SPL_MATERIALIZED) {
        GemvArgs g{};
        g.N = c->N;
        g.tiles_per_slab = c->tiles_per_slab;
        g.total_tiles = c->total_tiles;
        g.tiles_per_cta = c->tiles_per_cta;
        g.c = c->v;
        g.part = c->part;
        g.state = c->state;
        g.err_flag = c->err_flag;
        e = launch_gemv(&c->tmap, g, c->gemv_grid, s);
        if (e != cudaSuccess) return cuda_fail(e, "gemv");
    } else {
        TriSplitArgs ta{};
        ta.N = c->N;
        ta.vlen = c->vlen;
        ta.chunk = c->chunk;
        ta.v = c->v;
        ta.m = c->w;
        ta.scal = c->scal;
        ta.part = c->part;
        ta.ld_part = c->ld_part;
        ta.state = c->state;
        e = launch_tri_split(ta, false, c->chunks, s);
        if (e != cudaSuccess) return cuda_fail(e, "column pass");
    }
    return SPL_OK;
}

// One power step: the dense pass followed by the two finish kernels.
static spl_status_t chain_step(spl_chain *c, const FinishArgs &fa, cudaStream_t s) {
    spl_status_t st = chain_pass(c, s);
    if (st != SPL_OK) return st;
    cudaError_t e = launch_finish_step(fa, s);
    if (e != cudaSuccess) return cuda_fail(e, "finish step");
    return SPL_OK;
}

// Captures reps dense passes (whole_step false) or reps whole power steps on
// the chain's capture stream into an executable graph.
static spl_status_t capture_reps(spl_chain *c, const FinishArgs &fa, int reps, bool whole_step,
                                 cudaGraphExec_t *exec) {
    *exec = nullptr;
    if (!c->cap_stream) SPL_CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    SPL_CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    spl_status_t st = SPL_OK;
    for (int i = 0; i < reps && st == SPL_OK; ++i)
        st = whole_step ? chain_step(c, fa, c->cap_stream) : chain_pass(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != SPL_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return st != SPL_OK ? st : cuda_fail(e != cudaSuccess ? e : cudaErrorStreamCaptureInvalidated, "capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        *exec = nullptr;
        return cuda_fail(ei, "graph instantiate");
    }
    return SPL_OK;
}

// Captures kGraphSteps power steps of this chain once (on a private stream,
// so the caller's stream may be the legacy default stream) and keeps the
// executable graph; returns false if capture is unavailable, in which case the
// steps are launched one by one.
static bool chain_graph(spl_chain *c, const FinishArgs &fa) {
    if (c->steps_exec) return true;
    if (c->graph_failed) return false;
    bool ok = c->cap_stream || cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    cudaGraph_t g = nullptr;
    if (ok) ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        for (int i = 0; i < kGraphSteps && ok; ++i) ok = chain_step(c, fa, c->cap_stream) == SPL_OK;
        const bool ended = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess;
        ok = ok && ended && g;
    }
    if (ok) ok = cudaGraphInstantiate(&c->steps_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        c->steps_exec = nullptr;
        c->graph_failed = true;
        (void)cudaGetLastError();   // capture problems are not errors of the call
    }
    return ok;
}

static spl_status_t chain_report(spl_chain *c, cudaStream_t s, float *d_pi, spl_report_t *rep);

extern "C" spl_status_t spl_stationary(spl_chain_t *c, double tol, int32_t max_iter, const float *d_warm,
                                       float *d_pi, spl_report_t *rep) {
    if (!c || !d_pi || !(tol > 0.0) || max_iter < 1) return SPL_EINVAL;
    cudaStream_t s = c->stream;
    ChainState init{};
    init.tol_err = (float)(0.5 * tol);
    init.max_iter = max_iter;
    init.min_iter = 1;
    init.done = 0;
    SPL_CU(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    SPL_CU(cudaMemsetAsync(c->ticket, 0, 2 * sizeof(int), s));
    SPL_CU(cudaMemcpyAsync(c->state, &init, sizeof(ChainState), cudaMemcpyHostToDevice, s));
    const FinishArgs fa = finish_args(c);
    SPL_CU(launch_init_iter(fa, d_warm, s));
    if (c->mode == SPL_FUSED) {
        // one cooperative launch runs every step
        SPL_CU(cudaMemsetAsync(c->run_bar, 0, sizeof(unsigned) * chain_run_bar_words(), s));
        SPL_CU(cudaMemsetAsync(c->run_ticket, 0, sizeof(int) * c->run_T, s));
        SPL_CU(launch_chain_run(run_args(c), c->run_grid, s));
        SPL_CU(cudaMemcpyAsync(c->h_state, c->state, sizeof(ChainState), cudaMemcpyDeviceToHost, s));
        return chain_report(c, s, d_pi, rep);
    }
    // Steps are issued in chunks; every kernel exits at once when the device
    // state says done, so over-issuing within a chunk costs only launches.
    const bool graph = chain_graph(c, fa);
    int issued = 0;
    const int chunk = graph ? kGraphSteps : 4;
    for (;;) {
        const int n = graph ? chunk : std::min(chunk, max_iter - issued);
        if (graph) {
            SPL_CU(cudaGraphLaunch(c->steps_exec, s));
        } else {
            for (int i = 0; i < n; ++i) {
                spl_status_t st = chain_step(c, fa, s);
                if (st != SPL_OK) return st;
            }
        }
        issued += n;
        SPL_CU(cudaMemcpyAsync(c->h_state, c->state, sizeof(ChainState), cudaMemcpyDeviceToHost, s));
        SPL_CU(cudaStreamSynchronize(s));
        if (c->h_state->done || issued >= max_iter) break;
    }
    return chain_report(c, s, d_pi, rep);
}

// Error flag, result copy and report of a finished iteration (the state is
// already being copied to h_state on s).
static spl_status_t chain_report(spl_chain *c, cudaStream_t s, float *d_pi, spl_report_t *rep) {
    int herr = 0;
    SPL_CU(cudaMemcpyAsync(&herr, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPL_CU(cudaMemcpyAsync(d_pi, c->pi, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, s));
    SPL_CU(cudaStreamSynchronize(s));
    const ChainState &h = *c->h_state;
    spl_status_t st = herr ? SPL_ETIMEOUT : (h.done && h.status == ST_OK ? SPL_OK : SPL_ENOCONV);
    if (rep) {
        rep->iters = h.st.k;
        rep->status = st;
        rep->last_step_l1 = h.st.k > 0 ? h.st.delta[(h.st.k - 1) & 7] : 0.f;
        rep->err_bound = h.st.err;
        rep->lambda2_abs = h.st.rho;
        rep->lambda2_phase = h.st.theta;
    }
    return st;
}

// Times reps dense passes or reps whole steps, replayed from a captured graph
// (so no host launch overhead), after one untimed replay.
// Times one persistent fused launch of reps steps (after an untimed launch of
// a few): the stop rule is held open and max_iter = reps, so the launch makes
// reps steps plus the one pass its lagged stop decision needs.
static spl_status_t time_run(spl_chain *c, int32_t reps, float *ms_out) {
    cudaStream_t s = c->stream;
    const FinishArgs fa = finish_args(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPL_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        ChainState init{};
        init.tol_err = 0.f;
        init.max_iter = r == 0 ? std::min(reps, 4) : reps;
        init.min_iter = 1 << 30;
        if (e == cudaSuccess) e = cudaMemsetAsync(c->err_flag, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->run_bar, 0, sizeof(unsigned) * chain_run_bar_words(), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->run_ticket, 0, sizeof(int) * c->run_T, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->state, &init, sizeof(ChainState), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_init_iter(fa, nullptr, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_chain_run(run_args(c), c->run_grid, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "timing");
    if (herr) return SPL_ETIMEOUT;
    *ms_out = ms / reps;
    return SPL_OK;
}

static spl_status_t time_chain(spl_chain *c, int32_t reps, bool whole_step, float *ms_out) {
    if (whole_step && c->mode == SPL_FUSED) return time_run(c, reps, ms_out);
    cudaStream_t s = c->stream;
    // a valid broadcast vector and a state the stop rule never closes, so
    // no kernel exits early
    const FinishArgs fa = finish_args(c);
    ChainState init{};
    init.tol_err = 0.f;
    init.max_iter = 1 << 30;
    init.min_iter = 1 << 30;
    SPL_CU(cudaMemsetAsync(c->ticket, 0, 2 * sizeof(int), s));
    SPL_CU(cudaMemcpyAsync(c->state, &init, sizeof(ChainState), cudaMemcpyHostToDevice, s));
    SPL_CU(launch_init_iter(fa, nullptr, s));
    SPL_CU(cudaStreamSynchronize(s));
    cudaGraphExec_t exec = nullptr;
    spl_status_t st = capture_reps(c, fa, reps, whole_step, &exec);
    if (st != SPL_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);        // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "timing");
    *ms_out = ms / reps;
    return SPL_OK;
}

extern "C" spl_status_t spl_chain_time_pass(spl_chain_t *c, int32_t reps, float *ms_per_pass) {
    if (!c || reps < 1 || !ms_per_pass) return SPL_EINVAL;
    return time_chain(c, reps, false, ms_per_pass);
}

extern "C" spl_status_t spl_chain_time_step(spl_chain_t *c, int32_t reps, float *ms_per_step) {
    if (!c || reps < 1 || !ms_per_step) return SPL_EINVAL;
    return time_chain(c, reps, true, ms_per_step);
}

extern "C" spl_status_t spl_chain_time_build(spl_chain_t *c, int32_t reps, float *ms_per_build) {
    if (!c || reps < 1 || !ms_per_build || c->mode != SPL_MATERIALIZED) return SPL_EINVAL;
    cudaStream_t s = c->stream;
    cudaEvent_t e0, e1;
    SPL_CU(cudaEventCreate(&e0));
    SPL_CU(cudaEventCreate(&e1));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < reps + 1 && e == cudaSuccess; ++i) {
        if (i == 1) cudaEventRecord(e0, s);   // first build is a warm-up
        e = launch_build_matrix(c->N, c->p.l, c->ld, c->w, c->u, c->scal, c->P, c->rowsum, num_sms_current(), s);
    }
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "build timing");
    *ms_per_build = ms / reps;
    return SPL_OK;
}

extern "C" spl_status_t spl_matrix(spl_chain_t *c, float *d_P) {
    if (!c || !d_P || c->mode != SPL_MATERIALIZED) return SPL_EINVAL;
    SPL_CU(cudaMemcpy2DAsync(d_P, sizeof(float) * c->N, c->P, sizeof(float) * c->ld, sizeof(float) * c->N, c->N,
                             cudaMemcpyDeviceToDevice, c->stream));
    return SPL_OK;
}

extern "C" spl_status_t spl_chain_flux(spl_chain_t *c, float *d_lambda, double *d_F, double *h_Lambda,
                                       int32_t *h_shift) {
    if (!c) return SPL_EINVAL;
    if (d_lambda)
        SPL_CU(cudaMemcpyAsync(d_lambda, c->lam, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    if (d_F) SPL_CU(cudaMemcpyAsync(d_F, c->F, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    if (h_Lambda) {
        SPL_CU(cudaMemcpyAsync(h_Lambda, c->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SPL_CU(cudaStreamSynchronize(c->stream));
    }
    if (h_shift) *h_shift = c->p.l;
    return SPL_OK;
}

extern "C" void spl_free(spl_chain_t *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    chain_release(c);
}

// ======================================================================
// Batch
// ======================================================================

namespace {

// Device workspace reused across batch calls (grown on demand), one per
// device.  Calls on one device are serialised by its mutex.
struct BatchWorkspace {
    std::mutex mu;
    PixelDev *px = nullptr;
    size_t px_cap = 0;
    ReportDev *reps = nullptr;
    size_t reps_cap = 0;
    float *scratch = nullptr;
    size_t scratch_cap = 0;
    int *counter = nullptr;
    size_t counter_cap = 0;
    PixelConst *pconst = nullptr;
    size_t pconst_cap = 0;
    // staging of the host-buffer entry point
    float *d_warm = nullptr, *d_out = nullptr;
    size_t warm_cap = 0, out_cap = 0;
    int64_t *d_off = nullptr;
    size_t off_cap = 0;
    PixelDev *h_px = nullptr;        // pinned
    size_t h_px_cap = 0;
    ReportDev *h_reps = nullptr;     // pinned
    size_t h_reps_cap = 0;
    std::vector<int32_t> order;      // host scratch of make_work_list, kept across calls
    std::vector<int64_t> offs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    // copies of the host-buffer entry points overlap the next range's compute
    cudaStream_t copy_stream = nullptr;
    // barrier words and set counters of the multi-chain launch
    unsigned *multi_words = nullptr;
    size_t multi_words_cap = 0;
    // host-buffer calls: finished-pixel counts per caller range, their pinned
    // mirror, the stream that polls them and the end-of-kernel event
    int *range_done = nullptr;
    size_t range_done_cap = 0;
    int *h_range_done = nullptr;
    size_t h_range_done_cap = 0;
    cudaStream_t poll_stream = nullptr;
    cudaEvent_t ev_end = nullptr;
};

constexpr int kMaxDevices = 64;
BatchWorkspace g_ws[kMaxDevices];

template <typename T>
cudaError_t grow(T **p, size_t *cap, size_t need) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max(need, (size_t)1);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * n);
    if (e == cudaSuccess) *cap = n;
    return e;
}

template <typename T>
cudaError_t grow_host(T **p, size_t *cap, size_t need) {
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max(need, (size_t)1);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(p), sizeof(T) * n);
    if (e == cudaSuccess) *cap = n;
    return e;
}

spl_status_t ws_get(BatchWorkspace **out) {
    int dev = 0;
    SPL_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SPL_EINVAL;
    *out = &g_ws[dev];
    return SPL_OK;
}

spl_status_t status_of_alloc(cudaError_t e, const char *what) {
    return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : cuda_fail(e, what);
}

// Validates the pixels and writes the work list (sorted by decreasing N,
// ties by caller order) into pinned staging.  Offsets follow the caller's
// packed layout: either h_offsets (host) or the running sum of n_bins.
spl_status_t make_work_list(BatchWorkspace &ws, const spl_pixel_t *h_pixels, int32_t n, int *nmax_out) {
    cudaError_t e = grow_host(&ws.h_px, &ws.h_px_cap, (size_t)n);
    if (e != cudaSuccess) return status_of_alloc(e, "pinned work list");
    std::vector<int32_t> &order = ws.order;
    std::vector<int64_t> &off = ws.offs;
    order.resize((size_t)n);
    off.resize((size_t)n + 1);
    off[0] = 0;
    bool uniform = true;
    for (int32_t k = 0; k < n; ++k) {
        off[k + 1] = off[k] + h_pixels[k].n_bins;
        uniform = uniform && h_pixels[k].n_bins == h_pixels[0].n_bins;
    }
    std::iota(order.begin(), order.end(), 0);
    // largest pixels first; a batch of one size is already in that order
    if (!uniform)
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return h_pixels[a].n_bins > h_pixels[b].n_bins; });
    // the per-pixel records, in chunks on the host pool; the error reported is
    // that of the first bad pixel in work-list order, as a sequential loop
    // would report it
    std::atomic<int32_t> bad{n};
    std::atomic<int> bad_status{SPL_OK};
    std::atomic<int> nmax{2};
    std::mutex bad_mu;
    host_parallel_for(n, 4096, [&](int64_t lo, int64_t hi) {
        int cmax = 2;
        for (int64_t r = lo; r < hi; ++r) {
            const int32_t k = order[r];
            PixelDev d;
            const spl_status_t st = make_pixel(h_pixels[k], d);
            if (st != SPL_OK) {
                std::lock_guard<std::mutex> g(bad_mu);
                if ((int32_t)r < bad.load()) {
                    bad.store((int32_t)r);
                    bad_status.store(st);
                }
                return;
            }
            d.out_off = off[k];
            d.index = k;
            ws.h_px[r] = d;
            cmax = std::max(cmax, (int)d.N);
        }
        for (int m = nmax.load(); cmax > m && !nmax.compare_exchange_weak(m, cmax);) {
        }
    });
    if (bad.load() < n) return (spl_status_t)bad_status.load();
    *nmax_out = nmax.load();
    return SPL_OK;
}

// ---------------------------------------------------------------- batch launch configuration
//
// Launch configuration of the batch kernel: block size, columns per thread,
// state level and blocks per SM.  On the first large batch of a kind (padded
// N, pass kind, SM count) the feasible configurations are timed on a sample
// of the work list (tune_batch), the pick is kept in a cache, and
// SPL_TUNE_CACHE (a file path, optional) keeps the cache across processes.

struct LaunchCfg {
    int threads = 256, level = 2, bps = 0;   // bps: blocks per SM (at most the occupancy limit)
    int cols = 8;                            // columns per thread of the dense passes (8 or 4)
    size_t smem = 0;
};

spl_status_t batch_cfg(int threads, int level, int npad, bool structured, LaunchCfg *cfg, int cols = 8) {
    if (threads != 256 && threads != 512) return SPL_EINVAL;
    if (structured && threads != 256) return SPL_EINVAL;
    if (level < 0 || level > 2) return SPL_EINVAL;
    if (cols != 8 && cols != 4) return SPL_EINVAL;
    if (structured && cols != 8) return SPL_EINVAL;
    cfg->threads = threads;
    cfg->level = level;
    cfg->cols = cols;
    cfg->smem = batch_smem_bytes(npad, level);
    if (cfg->smem > 220 * 1024) return SPL_EINVAL;
    int bps = 0;
    SPL_CU(batch_occupancy(threads, level, structured, cfg->smem, &bps, cols));
    if (bps < 1) return SPL_EINVAL;
    cfg->bps = bps;
    return SPL_OK;
}

// Host-side fault injection for tests (SPL_FAULT in the environment, read at
// every batch call): "alloc" makes the call's first device allocation fail
// (SPL_ENOMEM), "launch" makes its kernel launch report a launch failure
// (SPL_ECUDA).  Nothing reaches the GPU in either case.
int injected_fault() {
    const char *f = std::getenv("SPL_FAULT");
    if (!f) return 0;
    if (!std::strcmp(f, "alloc")) return 1;
    if (!std::strcmp(f, "launch")) return 2;
    return 0;
}

using TuneKey = std::array<int, 3>;      // padded N, pass kind, SMs
using TuneVal = std::array<int, 4>;      // threads, state level, blocks per SM, columns per thread
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
bool g_tune_loaded = false;
constexpr int32_t kTuneMinPixels = 1024;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("SPL_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE *f = std::fopen(path, "r")) {
        // one entry per line: key (padded N, pass kind, SMs), then threads,
        // state level, blocks per SM and (optional, default 8) columns per thread
        char line[256];
        while (std::fgets(line, sizeof(line), f)) {
            int v[7];
            const int got = std::sscanf(line, "%d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6]);
            if (got == 6) v[6] = 8;
            else if (got != 7) break;   // a line broken off: the rest of the file is ignored
            g_tune[TuneKey{v[0], v[1], v[2]}] = TuneVal{v[3], v[4], v[5], v[6]};
        }
        std::fclose(f);
    }
}

void tune_store_locked(const TuneKey &k, const TuneVal &v) {
    g_tune[k] = v;
    const char *path = std::getenv("SPL_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "%d %d %d %d %d %d %d\n", k[0], k[1], k[2], v[0], v[1], v[2], v[3]);
        std::fclose(f);
    }
}

bool tune_lookup(const TuneKey &k, TuneVal *v) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

// One launch of the batch kernel over items [start, start + n) of the
// uploaded work list with configuration cfg (a holds everything else).
spl_status_t launch_cfg(BatchWorkspace &ws, BatchArgs a, const LaunchCfg &cfg, int32_t start, int32_t n, int npad,
                        cudaStream_t s) {
    int grid = cfg.bps * num_sms_current();
    if (grid > n) grid = n;
    const size_t per_block = cfg.level == 2 ? 0 : (size_t)(cfg.level == 1 ? 5 : 7) * npad;
    cudaError_t e;
    if (per_block && (e = grow(&ws.scratch, &ws.scratch_cap, (size_t)grid * per_block)) != cudaSuccess)
        return status_of_alloc(e, "scratch");
    SPL_CU(cudaMemsetAsync(ws.counter, 0, sizeof(int), s));
    a.px = ws.px + start;
    a.pconst = ws.pconst + start;
    a.n = n;
    a.scratch = ws.scratch;
    a.state_level = cfg.level;
    a.cols = cfg.cols;
    SPL_CU(launch_batch(a, cfg.threads, grid, cfg.smem, s));
    return SPL_OK;
}

// Times every feasible configuration on a sample of the work list and keeps
// the fastest.  State level and blocks per SM leave the pmfs unchanged bit
// for bit; the block size (the order of the block reductions) and the columns
// per thread (where the diagonal span cuts each column's sum into chunks)
// change them within rounding.  The configurations differ by a few percent at
// most, so the measurement guards against noise: a sample of up to
// kTuneSamplePerSm pixels per SM (a short sample is dominated by the tail of
// its last pixels), every configuration timed twice in two interleaved rounds
// (the minimum counts), and the heuristic's configuration `heur` kept unless
// another one beats it by more than kTuneMargin.
constexpr int32_t kTuneSamplePerSm = 48;
constexpr float kTuneMargin = 0.005f;

spl_status_t tune_batch(BatchWorkspace &ws, const BatchArgs &a, int32_t n, int npad, bool structured,
                        const LaunchCfg &heur, cudaStream_t s, LaunchCfg *best) {
    const int sms = num_sms_current();
    const int32_t sample = std::min<int32_t>(n, kTuneSamplePerSm * sms);
    if (!ws.ev0) SPL_CU(cudaEventCreate(&ws.ev0));
    if (!ws.ev1) SPL_CU(cudaEventCreate(&ws.ev1));
    // the heuristic first, then block size and columns per thread (dense
    // passes only), state level, and blocks per SM at the occupancy limit or
    // one below
    std::vector<LaunchCfg> cand{heur};
    const int nthr = structured ? 1 : 2, ncol = structured ? 1 : 2;
    for (int ti = 0; ti < nthr; ++ti)
    for (int ci = 0; ci < ncol; ++ci)
    for (int level = 2; level >= 0; --level) {
        LaunchCfg top;
        if (batch_cfg(ti ? 512 : 256, level, npad, structured, &top, ci ? 4 : 8) != SPL_OK) continue;
        for (int bps = top.bps; bps >= std::max(1, top.bps - 1); --bps) {
            LaunchCfg cfg = top;
            cfg.bps = bps;
            if (cfg.threads == heur.threads && cfg.level == heur.level && cfg.bps == heur.bps &&
                cfg.cols == heur.cols)
                continue;
            cand.push_back(cfg);
        }
    }
    std::vector<float> ms(cand.size(), INFINITY);
    for (int round = 0; round < 2; ++round) {
        for (size_t i = 0; i < cand.size(); ++i) {
            const LaunchCfg &cfg = cand[i];
            spl_status_t st;
            if (round == 0) {
                // untimed: loads the kernel's module and settles the clocks
                st = launch_cfg(ws, a, cfg, 0, std::min<int32_t>(sample, cfg.bps * sms), npad, s);
                if (st != SPL_OK) return st;
            }
            SPL_CU(cudaEventRecord(ws.ev0, s));
            if ((st = launch_cfg(ws, a, cfg, 0, sample, npad, s)) != SPL_OK) return st;
            SPL_CU(cudaEventRecord(ws.ev1, s));
            SPL_CU(cudaEventSynchronize(ws.ev1));
            float t = 0.f;
            SPL_CU(cudaEventElapsedTime(&t, ws.ev0, ws.ev1));
            ms[i] = std::min(ms[i], t);
        }
    }
    size_t bi = 0;
    for (size_t i = 1; i < cand.size(); ++i)
        if (ms[i] < ms[bi]) bi = i;
    if (!(ms[0] <= ms[bi] * (1.f + kTuneMargin))) *best = cand[bi];
    else *best = cand[0];
    return std::isfinite(ms[bi]) ? SPL_OK : SPL_EINVAL;
}

// Launches the persistent batch kernel; out/warm are packed by caller order.
// tune: 0 measured configuration (cached), 1 the fixed heuristic, 2 the
// caller's threads, state level and columns per thread.  range_done (device,
// [nranges], zeroed) receives the counts of finished pixels per caller range.
spl_status_t run_batch(BatchWorkspace &ws, int32_t n, int nmax, double tol, int32_t max_iter, const float *d_warm,
                       int warm_kind, int warm_ld, int min_iter, int threads_req, float *d_out,
                       const int64_t *d_offsets,
                       cudaStream_t s, bool time_kernel = false, int structured = 0, int flux_kind = 0,
                       int tune = 0, int level_req = -1, int cols_req = 0, int *range_done = nullptr,
                       int nranges = 0) {
    const int npad = batch_pad_len(nmax);
    const bool st_kind = structured == SPL_PASS_STRUCTURED;
    const int fault = injected_fault();
    if (fault == 1) return status_of_alloc(cudaErrorMemoryAllocation, "px (injected)");
    cudaError_t e;
    if ((e = grow(&ws.px, &ws.px_cap, (size_t)n)) != cudaSuccess) return status_of_alloc(e, "px");
    if ((e = grow(&ws.reps, &ws.reps_cap, (size_t)n)) != cudaSuccess) return status_of_alloc(e, "reports");
    if ((e = grow(&ws.counter, &ws.counter_cap, 1)) != cudaSuccess) return status_of_alloc(e, "counter");
    if ((e = grow(&ws.pconst, &ws.pconst_cap, (size_t)n)) != cudaSuccess) return status_of_alloc(e, "constants");
    SPL_CU(cudaMemcpyAsync(ws.px, ws.h_px, sizeof(PixelDev) * n, cudaMemcpyHostToDevice, s));
    BatchArgs a{};
    a.px = ws.px;
    a.n = n;
    a.counter = ws.counter;
    a.warm = d_warm;
    a.warm_kind = warm_kind;
    a.warm_ld = warm_ld;
    a.out = d_out;
    a.offsets = d_offsets;
    a.reports = ws.reps;
    a.npad_max = npad;
    a.tol_err = (float)(0.5 * tol);
    a.max_iter = max_iter;
    a.min_iter = std::max(1, min_iter);
    a.structured = st_kind ? 1 : 0;
    a.row_scan = structured == SPL_PASS_DENSE_ROWSCAN ? 1 : 0;
    a.flux_kind = flux_kind;
    a.pconst = ws.pconst;

    LaunchCfg cfg;
    spl_status_t st;
    if (tune == 2 || threads_req > 0) {
        const int level = level_req >= 0 ? level_req : batch_state_level(npad, st_kind);
        if ((st = batch_cfg(threads_req > 0 ? threads_req : 256, level, npad, st_kind, &cfg,
                            cols_req > 0 ? cols_req : 8)) != SPL_OK)
            return st;
    } else {
        // heuristic: 256 threads, the largest state level that keeps three
        // blocks' vectors in shared memory
        if ((st = batch_cfg(batch_threads_for(nmax), batch_state_level(npad, st_kind), npad, st_kind, &cfg)) !=
            SPL_OK)
            return st;
        if (tune == 0) {
            const TuneKey key{npad, structured, num_sms_current()};
            TuneVal v;
            LaunchCfg c2;
            if (tune_lookup(key, &v) && batch_cfg(v[0], v[1], npad, st_kind, &c2, v[3]) == SPL_OK &&
                v[2] >= 1 && v[2] <= c2.bps) {
                c2.bps = v[2];
                cfg = c2;
            } else if (n >= kTuneMinPixels) {
                if ((st = tune_batch(ws, a, n, npad, st_kind, cfg, s, &c2)) != SPL_OK) return st;
                cfg = c2;
                std::lock_guard<std::mutex> lock(g_tune_mu);
                tune_load_locked();
                tune_store_locked(key, TuneVal{cfg.threads, cfg.level, cfg.bps, cfg.cols});
            }
        }
    }
    if (fault == 2) return note_cuda_error(cudaErrorLaunchFailure, "batch launch (injected)");
    if (time_kernel) {
        if (!ws.ev0) SPL_CU(cudaEventCreate(&ws.ev0));
        if (!ws.ev1) SPL_CU(cudaEventCreate(&ws.ev1));
        SPL_CU(cudaEventRecord(ws.ev0, s));
    }
    if (range_done) {   // counted only in the launch that produces the result (not in tuning samples)
        a.range_done = range_done;
        a.nranges = nranges;
        a.range_n = n;
    }
    if ((st = launch_cfg(ws, a, cfg, 0, n, npad, s)) != SPL_OK) return st;
    if (time_kernel) {
        SPL_CU(cudaEventRecord(ws.ev1, s));
        ws.timed = true;
    }
    return SPL_OK;
}

spl_status_t collect_reports(BatchWorkspace &ws, int32_t n, spl_report_t *h_reports, cudaStream_t s) {
    cudaError_t e = grow_host(&ws.h_reps, &ws.h_reps_cap, (size_t)n);
    if (e != cudaSuccess) return status_of_alloc(e, "pinned reports");
    SPL_CU(cudaMemcpyAsync(ws.h_reps, ws.reps, sizeof(ReportDev) * n, cudaMemcpyDeviceToHost, s));
    SPL_CU(cudaStreamSynchronize(s));
    spl_status_t worst = SPL_OK;
    for (int32_t k = 0; k < n; ++k) {
        const ReportDev &r = ws.h_reps[k];
        spl_report_t &o = h_reports[k];
        o.iters = r.iters;
        o.status = r.status;
        o.last_step_l1 = r.last_step_l1;
        o.err_bound = r.err_bound;
        o.lambda2_abs = r.lambda2_abs;
        o.lambda2_phase = r.lambda2_phase;
        if (r.status > (int)worst) worst = (spl_status_t)r.status;
    }
    return worst;
}

}  // namespace

extern "C" spl_status_t spl_batch_stationary_ex(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                                const float *d_warm, float *d_out, const int64_t *d_offsets,
                                                spl_report_t *h_reports, void *stream, const spl_batch_opts_t *opts) {
    if (n < 0 || (n > 0 && (!h_pixels || !d_out || !d_offsets)) || !(tol > 0.0) || max_iter < 1) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    BatchWorkspace *ws = nullptr;
    spl_status_t st = ws_get(&ws);
    if (st != SPL_OK) return st;
    std::lock_guard<std::mutex> lock(ws->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nmax = 0;
    st = make_work_list(*ws, h_pixels, n, &nmax);
    if (st != SPL_OK) return st;
    const int kind = opts ? opts->warm_kind : 0;
    const int ld = opts ? opts->warm_ld : 0;
    if (d_warm && (kind < 0 || kind > 2)) return SPL_EINVAL;
    if (d_warm && kind == 2) {
        for (int32_t k = 0; k < n; ++k)
            if (ld < h_pixels[k].n_bins) return SPL_EINVAL;
    }
    const int min_iter = opts ? opts->min_iter : 1;
    const int threads = opts ? opts->threads : 0;
    const bool timed = opts && opts->time_kernel;
    const int structured = opts ? opts->pass_kind : 0;
    if (structured < SPL_PASS_DENSE || structured > SPL_PASS_DENSE_ROWSCAN) return SPL_EINVAL;
    const int flux_kind = opts ? opts->flux_kind : 0;
    if (flux_kind != SPL_FLUX_POINT && flux_kind != SPL_FLUX_BININT) return SPL_EINVAL;
    const int tune = opts ? opts->tune : 0;
    const int level = opts ? opts->state_level : -1;
    if (tune < 0 || tune > 2 || (tune == 2 && (level < 0 || level > 2))) return SPL_EINVAL;
    const int cols = opts ? opts->cols : 0;
    if (cols != 0 && cols != 4 && cols != 8) return SPL_EINVAL;
    st = run_batch(*ws, n, nmax, tol, max_iter, d_warm, kind, ld, min_iter, threads, d_out, d_offsets, s, timed,
                   structured, flux_kind, tune, tune == 2 ? level : -1, cols);
    if (st != SPL_OK) return st;
    if (h_reports) return collect_reports(*ws, n, h_reports, s);
    // The pinned work list is read by the copy engine asynchronously; keep the
    // next call from overwriting it before that copy ran.
    SPL_CU(cudaStreamSynchronize(s));
    return SPL_OK;
}

extern "C" spl_status_t spl_batch_stationary(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                             const float *d_warm, float *d_out, const int64_t *d_offsets,
                                             spl_report_t *h_reports, void *stream) {
    return spl_batch_stationary_ex(h_pixels, n, tol, max_iter, d_warm, d_out, d_offsets, h_reports, stream, nullptr);
}

// Host-buffer batch: pmfs into pinned or pageable h_out (packed in caller
// order), reports into h_reports (may be NULL).  One launch; in a batch of
// one size the copy-back of each of eight caller ranges (on a second stream)
// starts as soon as the kernel has finished that range, overlapping the rest
// of the kernel.
spl_status_t spl::batch_host_run(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                                 const float *d_warm, const float *h_warm, int warm_kind, int warm_ld, float *h_out,
                                 spl_report_t *h_reports, cudaStream_t s, const spl_batch_opts_t *opts) {
    if (n < 0 || (n > 0 && (!h_pixels || !h_out)) || !(tol > 0.0) || max_iter < 1) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    const int min_iter = opts ? opts->min_iter : 1;
    const int threads = opts ? opts->threads : 0;
    const int structured = opts ? opts->pass_kind : 0;
    const int flux_kind = opts ? opts->flux_kind : 0;
    const int tune = opts ? opts->tune : 0;
    const int level = opts ? opts->state_level : -1;
    if (structured < SPL_PASS_DENSE || structured > SPL_PASS_DENSE_ROWSCAN) return SPL_EINVAL;
    if (flux_kind != SPL_FLUX_POINT && flux_kind != SPL_FLUX_BININT) return SPL_EINVAL;
    if (tune < 0 || tune > 2 || (tune == 2 && (level < 0 || level > 2))) return SPL_EINVAL;
    BatchWorkspace *ws = nullptr;
    spl_status_t st = ws_get(&ws);
    if (st != SPL_OK) return st;
    std::lock_guard<std::mutex> lock(ws->mu);
    int nmax = 0;
    st = make_work_list(*ws, h_pixels, n, &nmax);
    if (st != SPL_OK) return st;
    if (d_warm && warm_kind == 2) {
        for (int32_t k = 0; k < n; ++k)
            if (warm_ld < h_pixels[k].n_bins) return SPL_EINVAL;
    }
    const std::vector<int64_t> &off = ws->offs;
    const size_t total = (size_t)off[(size_t)n];
    bool uniform = true;
    for (int32_t k = 1; k < n && uniform; ++k) uniform = h_pixels[k].n_bins == h_pixels[0].n_bins;
    cudaError_t e;
    if ((e = grow(&ws->d_out, &ws->out_cap, total)) != cudaSuccess) return status_of_alloc(e, "out");
    if (h_warm) {
        if ((e = grow(&ws->d_warm, &ws->warm_cap, total)) != cudaSuccess) return status_of_alloc(e, "warm");
        SPL_CU(cudaMemcpyAsync(ws->d_warm, h_warm, sizeof(float) * total, cudaMemcpyHostToDevice, s));
        d_warm = ws->d_warm;
        warm_kind = 0;
        warm_ld = 0;
    }
    if (!ws->copy_stream) SPL_CU(cudaStreamCreateWithFlags(&ws->copy_stream, cudaStreamNonBlocking));
    float *d_out = ws->d_out;
    cudaStream_t cs = ws->copy_stream;
    if (!uniform) {
        // ragged batch: the work list is sorted by size, so the output is
        // copied in one piece after the launch
        st = run_batch(*ws, n, nmax, tol, max_iter, d_warm, warm_kind, warm_ld, min_iter, threads, d_out, nullptr, s,
                       false, structured, flux_kind, tune, tune == 2 ? level : -1, opts ? opts->cols : 0);
        if (st != SPL_OK) return st;
        SPL_CU(cudaMemcpyAsync(h_out, d_out, sizeof(float) * total, cudaMemcpyDeviceToHost, s));
        if (h_reports) return collect_reports(*ws, n, h_reports, s);
        SPL_CU(cudaStreamSynchronize(s));
        return SPL_OK;
    }
    // A batch of one size keeps the caller's order in the work list, so each
    // of kHostRanges caller ranges is a contiguous slice of the output.  One
    // launch runs the whole batch; the kernel counts each range's finished
    // pixels, this thread polls the counts (a small copy on its own stream)
    // and starts a range's copy-back as soon as its count is full, while the
    // kernel runs on.  The wait ends when the kernel's end event completes.
    constexpr int kHostRanges = 8;
    const int K = std::min<int32_t>(kHostRanges, n);
    if ((e = grow(&ws->range_done, &ws->range_done_cap, (size_t)K)) != cudaSuccess)
        return status_of_alloc(e, "range counts");
    if ((e = grow_host(&ws->h_range_done, &ws->h_range_done_cap, (size_t)K)) != cudaSuccess)
        return status_of_alloc(e, "pinned range counts");
    if (!ws->poll_stream) SPL_CU(cudaStreamCreateWithFlags(&ws->poll_stream, cudaStreamNonBlocking));
    if (!ws->ev_end) SPL_CU(cudaEventCreateWithFlags(&ws->ev_end, cudaEventDisableTiming));
    SPL_CU(cudaMemsetAsync(ws->range_done, 0, sizeof(int) * K, s));
    st = run_batch(*ws, n, nmax, tol, max_iter, d_warm, warm_kind, warm_ld, min_iter, threads, d_out, nullptr, s,
                   false, structured, flux_kind, tune, tune == 2 ? level : -1, opts ? opts->cols : 0,
                   ws->range_done, K);
    if (st != SPL_OK) return st;
    SPL_CU(cudaEventRecord(ws->ev_end, s));
    bool sent[kHostRanges] = {};
    int nsent = 0;
    auto send = [&](int c) -> spl_status_t {
        const int64_t lo = (int64_t)n * c / K, hi = (int64_t)n * (c + 1) / K;
        const int64_t o0 = off[(size_t)lo], o1 = off[(size_t)hi];
        SPL_CU(cudaMemcpyAsync(h_out + o0, d_out + o0, sizeof(float) * (size_t)(o1 - o0), cudaMemcpyDeviceToHost,
                               cs));
        sent[c] = true;
        ++nsent;
        return SPL_OK;
    };
    while (nsent < K) {
        const cudaError_t q = cudaEventQuery(ws->ev_end);
        if (q == cudaSuccess) {            // the kernel is done: copy whatever is left
            for (int c = 0; c < K; ++c)
                if (!sent[c] && (st = send(c)) != SPL_OK) return st;
            break;
        }
        if (q != cudaErrorNotReady) return cuda_fail(q, "batch kernel");
        SPL_CU(cudaMemcpyAsync(ws->h_range_done, ws->range_done, sizeof(int) * K, cudaMemcpyDeviceToHost,
                               ws->poll_stream));
        SPL_CU(cudaStreamSynchronize(ws->poll_stream));
        for (int c = 0; c < K; ++c) {
            const int64_t size = (int64_t)n * (c + 1) / K - (int64_t)n * c / K;
            if (!sent[c] && ws->h_range_done[c] >= size && (st = send(c)) != SPL_OK) return st;
        }
        if (nsent < K) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    SPL_CU(cudaStreamSynchronize(cs));
    if (h_reports) return collect_reports(*ws, n, h_reports, s);
    SPL_CU(cudaStreamSynchronize(s));
    return SPL_OK;
}

extern "C" spl_status_t spl_chains_plan(const int32_t *n_bins, int32_t n, int32_t sms, int32_t blocks_per_sm,
                                        int32_t *slots) {
    if (!n_bins || !slots || n < 1 || n > kChainMultiMax || sms < 1 || blocks_per_sm < 1) return SPL_EINVAL;
    for (int32_t g = 0; g < n; ++g) {
        if (n_bins[g] < 2 || n_bins[g] > kMaxBins) return SPL_EINVAL;
        slots[g] = chain_multi_slots(n_bins[g], sms * blocks_per_sm);
    }
    return SPL_OK;
}

extern "C" spl_status_t spl_chains_stationary(spl_chain_t *const *chains, int32_t n, double tol, int32_t max_iter,
                                              float *d_out, spl_report_t *h_reports) {
    if (n < 0 || (n > 0 && (!chains || !d_out)) || !(tol > 0.0) || max_iter < 1) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    for (int32_t k = 0; k < n; ++k)
        if (!chains[k] || chains[k]->mode != SPL_FUSED || chains[k]->stream != chains[0]->stream) return SPL_EINVAL;
    for (int32_t k = 0; k < n; ++k)
        for (int32_t j = 0; j < k; ++j)
            if (chains[j] == chains[k]) return SPL_EINVAL;   // one chain's buffers hold one iteration
    BatchWorkspace *ws = nullptr;
    spl_status_t st = ws_get(&ws);
    if (st != SPL_OK) return st;
    std::lock_guard<std::mutex> lock(ws->mu);
    cudaStream_t s = chains[0]->stream;
    cudaError_t e = grow(&ws->reps, &ws->reps_cap, (size_t)n);
    if (e != cudaSuccess) return status_of_alloc(e, "reports");
    if ((e = grow(&ws->multi_words, &ws->multi_words_cap, (size_t)kMultiWords)) != cudaSuccess)
        return status_of_alloc(e, "barrier words");
    const int bps = std::min(2, chain_multi_blocks_per_sm(chain_run_max_chunk()));
    if (bps < 1) return cuda_fail(cudaErrorLaunchOutOfResources, "multi-chain occupancy");
    const int grid = bps * num_sms_current();
    static_assert(sizeof(ChainMultiArgs) < 30000, "kernel parameter size");
    ChainMultiArgs M;
    int64_t off = 0;
    for (int32_t k0 = 0; k0 < n; k0 += kChainMultiMax) {
        const int m = std::min<int32_t>(kChainMultiMax, n - k0);
        std::memset(&M, 0, sizeof(M));
        M.n = m;
        M.words = ws->multi_words;
        // two CTA sets (one CTA of each SM in each) when there are two CTAs per
        // SM and two chains or more.  The chains are dealt to the sets one by
        // one, in order, each to the set whose work per pass (N^2) stays the
        // smaller relative to its share kSet0Share : 1 - kSet0Share, so that
        // neighbouring chains (often similar ones) land in different sets.  The
        // first CTA to start on an SM (set 0) gets the larger share of the
        // SM's issue slots while both run (measured: with equal work, set 0
        // finished its steps in 0.73 of set 1's time), so it takes more work:
        // for 12 equal chains of N = 10000 the shares that deal 7:5, 8:4 and
        // 9:3 chains took 0.581, 0.538 and 0.575 ms.
        constexpr double kSet0Share = 0.64;
        M.nsets = (bps == 2 && m >= 2) ? 2 : 1;
        int order[kChainMultiMax];
        int n0 = m;
        if (M.nsets == 2) {
            int list[2][kChainMultiMax], cnt[2] = {0, 0};
            double load[2] = {0.0, 0.0};
            const double share[2] = {kSet0Share, 1.0 - kSet0Share};
            for (int g = 0; g < m; ++g) {
                const double w = (double)chains[k0 + g]->N * chains[k0 + g]->N;
                const int q = (load[0] + w) / share[0] <= (load[1] + w) / share[1] ? 0 : 1;
                load[q] += w;
                list[q][cnt[q]++] = g;
            }
            if (cnt[1] == 0) list[1][cnt[1]++] = list[0][--cnt[0]];   // every set gets a chain
            n0 = cnt[0];
            for (int q = 0; q < cnt[0]; ++q) order[q] = list[0][q];
            for (int q = 0; q < cnt[1]; ++q) order[n0 + q] = list[1][q];
        } else {
            for (int g = 0; g < m; ++g) order[g] = g;
        }
        M.set_begin[0] = 0;
        M.set_begin[1] = n0;
        M.set_begin[2] = m;
        M.tol_err = (float)(0.5 * tol);
        M.min_iter = 1;
        M.max_iter = max_iter;
        int64_t coff[kChainMultiMax];   // packed output offset of each chain, in the caller's order
        for (int g = 0; g < m; ++g) {
            coff[g] = off;
            off += chains[k0 + g]->N;
        }
        long long Us[2] = {0, 0};   // units of each set's first step
        for (int q = 0; q < m; ++q) {
            const int g = order[q];
            spl_chain *c = chains[k0 + g];
            Us[q < n0 ? 0 : 1] += (long long)c->run_T * c->run_RB;
            const int slots = chain_multi_slots(c->N, grid);
            const size_t need_part = (size_t)c->run_T * slots * chain_run_tile_cols();
            const size_t need_blk = 2 * (size_t)grid * 4;
            if (need_part > c->run_part_cap || need_blk > c->run_blk_cap) {
                // more partial slots or statistics slots than the chain's own plan
                SPL_CU(cudaStreamSynchronize(s));
                if (need_part > c->run_part_cap) {
                    float *np = nullptr;
                    if ((e = dalloc(&np, need_part)) != cudaSuccess) return status_of_alloc(e, "chain partials");
                    cudaFree(c->run_part);
                    c->run_part = np;
                    c->run_part_cap = need_part;
                }
                if (need_blk > c->run_blk_cap) {
                    float *nb = nullptr;
                    if ((e = dalloc(&nb, need_blk)) != cudaSuccess) return status_of_alloc(e, "chain statistics");
                    cudaFree(c->run_blk);
                    c->run_blk = nb;
                    c->run_blk_cap = need_blk;
                }
            }
            ChainRunArgs a = run_args(c);
            a.segs = slots;
            M.c[q] = a;
            M.off[q] = coff[g];
            M.idx[q] = g;
        }
        // rows of one staging buffer (the kernel's windows never exceed it): at
        // most chain_run_max_chunk(), and no more than the largest share of a
        // CTA in the first step of its set (grid / nsets CTAs per set)
        long long per_cta = 1;
        const long long Gs = grid / M.nsets;
        for (int q = 0; q < M.nsets; ++q)
            if (Us[q] > 0) per_cta = std::max(per_cta, (Us[q] + std::min(Gs, Us[q]) - 1) / std::min(Gs, Us[q]));
        M.chunk = (int)std::min<long long>(chain_run_max_chunk(), 32 * per_cta);
        SPL_CU(launch_chain_multi(M, grid, d_out, ws->reps + k0, s));
    }
    if (!h_reports) return SPL_OK;
    e = grow_host(&ws->h_reps, &ws->h_reps_cap, (size_t)n);
    if (e != cudaSuccess) return status_of_alloc(e, "pinned reports");
    SPL_CU(cudaMemcpyAsync(ws->h_reps, ws->reps, sizeof(ReportDev) * n, cudaMemcpyDeviceToHost, s));
    SPL_CU(cudaStreamSynchronize(s));
    spl_status_t worst = SPL_OK;
    for (int32_t k = 0; k < n; ++k) {
        const ReportDev &r = ws->h_reps[k];
        spl_report_t &o = h_reports[k];
        o.iters = r.iters;
        o.status = r.status;
        o.last_step_l1 = r.last_step_l1;
        o.err_bound = r.err_bound;
        o.lambda2_abs = r.lambda2_abs;
        o.lambda2_phase = r.lambda2_phase;
        if (r.status > (int)worst) worst = (spl_status_t)r.status;
    }
    return worst;
}

extern "C" spl_status_t spl_batch_stationary_host(const spl_pixel_t *h_pixels, int32_t n, double tol,
                                                  int32_t max_iter, const float *h_warm, float *h_out,
                                                  spl_report_t *h_reports, void *stream) {
    return batch_host_run(h_pixels, n, tol, max_iter, nullptr, h_warm, 0, 0, h_out, h_reports,
                          static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" spl_status_t spl_batch_spectral(const spl_pixel_t *h_pixels, int32_t n, int32_t subspace_iters,
                                           float *d_out, void *stream) {
    if (n < 0 || (n > 0 && (!h_pixels || !d_out)) || subspace_iters < 1) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    BatchWorkspace *ws = nullptr;
    spl_status_t st = ws_get(&ws);
    if (st != SPL_OK) return st;
    std::lock_guard<std::mutex> lock(ws->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nmax = 0;
    st = make_work_list(*ws, h_pixels, n, &nmax);
    if (st != SPL_OK) return st;
    if (nmax > 4096) return SPL_EINVAL;
    cudaError_t e;
    if ((e = grow(&ws->px, &ws->px_cap, (size_t)n)) != cudaSuccess) return status_of_alloc(e, "px");
    if ((e = grow(&ws->pconst, &ws->pconst_cap, (size_t)n)) != cudaSuccess) return status_of_alloc(e, "constants");
    SPL_CU(cudaMemcpyAsync(ws->px, ws->h_px, sizeof(PixelDev) * n, cudaMemcpyHostToDevice, s));
    SpectralArgs a{};
    a.pconst = ws->pconst;
    a.px = ws->px;
    a.n = n;
    a.npad_max = batch_pad_len(nmax);
    a.pi_iters = 500;
    a.subspace_iters = subspace_iters;
    a.out = d_out;
    const int grid = std::min(n, 2 * num_sms_current());
    SPL_CU(launch_spectral(a, grid, s));
    SPL_CU(cudaStreamSynchronize(s));   // the pinned work list is reused by the next call
    return SPL_OK;
}

extern "C" spl_status_t spl_batch_tune_lookup(int32_t n_bins_max, int32_t pass_kind, int32_t *threads,
                                              int32_t *state_level, int32_t *blocks_per_sm, int32_t *cols) {
    if (n_bins_max < 2 || !threads || !state_level || !blocks_per_sm) return SPL_EINVAL;
    if (pass_kind < SPL_PASS_DENSE || pass_kind > SPL_PASS_DENSE_ROWSCAN) return SPL_EINVAL;
    const TuneKey key{batch_pad_len(n_bins_max), pass_kind, num_sms_current()};
    TuneVal v;
    if (!tune_lookup(key, &v)) return SPL_ENOCONV;
    *threads = v[0];
    *state_level = v[1];
    *blocks_per_sm = v[2];
    if (cols) *cols = v[3];
    return SPL_OK;
}

extern "C" spl_status_t spl_batch_kernel_ms(float *ms) {
    if (!ms) return SPL_EINVAL;
    BatchWorkspace *ws = nullptr;
    spl_status_t st = ws_get(&ws);
    if (st != SPL_OK) return st;
    std::lock_guard<std::mutex> lock(ws->mu);
    if (!ws->timed) return SPL_EINVAL;
    SPL_CU(cudaEventSynchronize(ws->ev1));
    SPL_CU(cudaEventElapsedTime(ms, ws->ev0, ws->ev1));
    return SPL_OK;
}

extern "C" spl_status_t spl_fp32_fma_peak(int32_t iters, int32_t reps, void *stream, double *tflops_median,
                                          double *tflops_best, int32_t *sms_out) {
    if (iters < 1 || reps < 1 || !tflops_median) return SPL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return note_cuda_error(e, "fma peak: device query");
    float *out = nullptr;
    e = cudaMalloc(&out, fma_peak_out_floats(sms) * sizeof(float));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SPL_ENOMEM : note_cuda_error(e, "fma peak: alloc");
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e == cudaSuccess) e = launch_fma_peak(out, sms, iters, s);   // untimed
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(ev[2 * r], s);
        if (e == cudaSuccess) e = launch_fma_peak(out, sms, iters, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * r + 1], s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<float> ms((size_t)reps, 0.f);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(out);
    if (e != cudaSuccess) return note_cuda_error(e, "fma peak");
    std::sort(ms.begin(), ms.end());
    const double flop = fma_peak_flop(sms, iters);
    *tflops_median = flop / (ms[(size_t)reps / 2] * 1e-3) / 1e12;
    if (tflops_best) *tflops_best = flop / (ms[0] * 1e-3) / 1e12;
    if (sms_out) *sms_out = sms;
    return SPL_OK;
}

extern "C" spl_status_t spl_selftest_bounded_waits(void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *bar = nullptr;
    int *flags = nullptr;   // [0] error flag, [1] mbarrier wait gave up, [2] CTAs that saw the abort
    cudaError_t e = cudaMalloc(&bar, sizeof(unsigned) * chain_run_bar_words());
    if (e == cudaSuccess) e = cudaMalloc(&flags, 3 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(unsigned) * chain_run_bar_words(), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 3 * sizeof(int), s);
    if (e == cudaSuccess) e = launch_selftest_waits(bar, flags, flags + 1, s);
    int h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (bar) cudaFree(bar);
    if (flags) cudaFree(flags);
    if (e != cudaSuccess) return note_cuda_error(e, "bounded-wait self-test");
    // the mbarrier wait gave up; both CTAs that reached the grid barrier gave
    // up, set the error flag and left it as aborted
    return (h[0] == 1 && h[1] == 1 && h[2] == 2) ? SPL_OK : SPL_EINVAL;
}

// ======================================================================
// Misc
// ======================================================================

extern "C" const char *spl_strerror(spl_status_t s) {
    switch (s) {
        case SPL_OK: return "ok";
        case SPL_EINVAL: return "invalid argument";
        case SPL_ENOMEM: return "out of memory";
        case SPL_ECUDA: return "CUDA error";
        case SPL_ENOCONV: return "power iteration did not converge within max_iter";
        case SPL_ETIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

extern "C" const char *spl_last_cuda_error(void) { return g_cuda_err; }

extern "C" const char *spl_version(void) { return "libspl 0.1 (sm_103a)"; }
