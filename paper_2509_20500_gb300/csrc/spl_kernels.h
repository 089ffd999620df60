// Internal interface between the libspl host code and its kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spl.h"
#include "spl_device.cuh"

namespace spl {

// Records a CUDA failure for spl_last_cuda_error; returns SPL_ECUDA.
spl_status_t note_cuda_error(cudaError_t e, const char *where);

// a1: validates one pixel and derives its row shift l = ceil(q) mod N
// (Theorem 2; q = fmod(t_d, t_r) N / t_r in IEEE FP64) into d.  SPL_EINVAL
// for an invalid pixel.  Every entry point takes its pixels through here.
spl_status_t make_pixel(const spl_pixel_t &p, PixelDev &d);

// Device-resident state of one chain's iteration (single-pixel API).
struct ChainState {
    StopState st;
    int32_t done;
    int32_t status;
    float tol_err;
    int32_t max_iter;
    int32_t min_iter;
    float ysum;              // sum of the current step's y (finish stage 1 -> 2)
    int32_t pad_[2];
};

struct BatchArgs {
    const PixelDev *px;      // sorted work list
    int n;
    int *counter;            // work-queue head, zero before launch
    const float *warm;       // NULL, or the warm start (see warm_kind)
    int warm_kind;           // spl_warm_kind_t
    int warm_ld;             // row stride of learned-frame logits
    float *out;              // packed output
    const int64_t *offsets;  // [n + 1] caller offsets by caller index, or NULL (use px.out_off)
    ReportDev *reports;      // [n] by caller index, may be NULL
    float *scratch;          // [grid][5 or 7][npad_max] for the vectors not in shared memory
    int npad_max;
    int state_level;         // 2: all vectors in shared memory; 1: v, pi, rho; 0: v only
    float tol_err;
    int max_iter;
    int min_iter;
    int structured;          // 1: O(N) scan form of the power step (same result, no N^2 pass)
    int row_scan;            // 1 (dense steps): row sums by the scans of the structured form, not a dense pass
    int cols;                // columns per thread of the dense passes: 4, or 8 (any other value)
    int *range_done;         // NULL, or [nranges] counts of finished pixels per caller range (host-buffer calls)
    int nranges;             // caller ranges [range_n c / nranges, range_n (c+1) / nranges)
    int range_n;             // pixels of the call
    int flux_kind;           // spl_flux_kind_t: 0 point flux (Sec. 3.4), 1 bin-integrated
    PixelConst *pconst;      // [n] per-pixel constants (work-list order), written by launch_batch
};

struct GemvArgs {
    int N;
    int tiles_per_slab;      // ceil(N / 32)
    int total_tiles;         // slabs * tiles_per_slab
    int tiles_per_cta;
    const float *c;          // [N] row coefficients pi_i / r_i
    float *part;             // [grid][2][128]
    const ChainState *state; // early exit once converged (may be NULL)
    int *err_flag;
};

struct TriSplitArgs {
    int N;
    int vlen;                // padded length of v (multiple of 128)
    int chunk;               // b-chunk per CTA row (multiple of 128)
    const float *v;          // broadcast vector [vlen]
    const float *m;          // per-output factor: w (column pass) or u (row pass)
    const double *scal;      // [0] Lambda, [1] eL
    float *part;             // [chunks][ld_part]
    int ld_part;
    const ChainState *state; // may be NULL
};

// Persistent power iteration of one chain (fused mode): one cooperative
// launch runs every step.  The column pass is cut into T x RB equal units,
// (tile of chain_run_tile_cols() columns) x (32 rows), taken by the CTAs in
// contiguous ranges; each CTA leaves one partial per tile it touches, and the
// last CTA to finish a tile adds the tile's partials.
struct ChainRunArgs {
    int N, vlen, l;
    int T, RB;               // column tiles; 32-row blocks per tile (vlen / 32)
    int segs;                // partial slots per CTA (tiles one CTA's units may touch)
    int chunk;               // rows of h staged in shared memory at once (at most)
    const float *w;          // [vlen] column factors w_j (zero past N)
    const double *scal;      // [1] = e^{-Lambda}
    const float *rho;        // [vlen] rho_k = u_k / r'_k
    const float *v0;         // [vlen] first broadcast vector pi^(0)_{(k-l) mod N} rho_k, zero past N
    float *pi, *pi_alt;      // [N] iterates of even and odd steps (pi: pi^(0) in, the result out)
    float *d1, *d2;          // [N] the last two steps
    float *y;                // [2][vlen] unnormalised iterates (alternating)
    float *vb;               // [2][vlen] next broadcast vectors (alternating), zero past N
    float *tsum;             // [2][T][TW / 32] tile sums of y, one partial per warp of a tile
    float *part;             // [grid][segs][tile columns] per-CTA partial column sums
    float *blk;              // [2][grid][4] per-CTA step statistics (16-byte aligned)
    int *tile_ticket;        // [T] arrival counters, zero between uses
    unsigned *bar;           // [chain_run_bar_words()] grid barrier words (zero at launch)
    ChainState *state;
    int *err_flag;           // set if a CTA gave up waiting at the barrier
};

// Several fused chains in one cooperative launch (at most kChainMultiMax),
// in lockstep: the CTAs form nsets sets (with two, one CTA of each SM in
// each), set s runs chains [set_begin[s], set_begin[s+1]), and at every power
// step the work units of its chains still iterating are numbered one chain
// after the other and split evenly over the set's CTAs (their bins likewise
// for the normalisation), so a chain that stops leaves no CTA idle.
// c[g].segs is the number of partial slots per column tile of chain g;
// c[g].blk holds [2][grid][4] statistics; c[g].bar is unused (the launch's
// barriers are in words).  Results go to out + off[g], reports to
// reps[idx[g]].
constexpr int kChainMultiMax = 32;
struct ChainMultiArgs {
    ChainRunArgs c[kChainMultiMax];
    int64_t off[kChainMultiMax];
    int idx[kChainMultiMax];  // caller's position of chain g in this launch (its report slot)
    int n;
    int chunk;               // rows per staging buffer
    int nsets;               // 1: all CTAs run all chains; 2: two CTA sets, chains [set_begin[s], set_begin[s+1])
    int set_begin[3];
    unsigned *words;         // [kMultiWords] barrier words and set counters, zeroed by the start kernel
    float tol_err;
    int min_iter, max_iter;
};
// Layout of ChainMultiArgs::words: three barriers (the whole grid, set 0,
// set 1) of 64 words each, two set sizes, one CTA counter per SM id.
constexpr int kMultiCountWord = 192;
constexpr int kMultiSlotWord = 194;
constexpr int kMultiSmSlots = 1024;
constexpr int kMultiWords = kMultiSlotWord + kMultiSmSlots;

int chain_run_tile_cols();
int chain_run_bar_words();
int chain_run_max_grid();
int chain_run_max_chunk();
size_t chain_run_smem_bytes(int chunk);
// CTAs per SM the cooperative launch can keep resident (0 on error).
int chain_run_blocks_per_sm(int chunk);
cudaError_t launch_chain_run(const ChainRunArgs &a, int grid, cudaStream_t s);
// Multi-chain iteration: init kernel (uniform start, stop state tol_err /
// max_iter, cleared tickets, barrier and error flag), the cooperative launch
// of `grid` CTAs with `chunk` rows of shared staging, and the finish kernel
// (results to out, reports to reps if not NULL).
cudaError_t launch_chain_multi(const ChainMultiArgs &m, int grid, float *out, ReportDev *reps, cudaStream_t s);
// Partial slots per column tile that chain g needs when its units are part
// of a lockstep partition over `grid` CTAs.
int chain_multi_slots(int n_bins, int grid);
int chain_multi_blocks_per_sm(int chunk);
// Waits that run out on purpose (status[0]: the mbarrier wait gave up;
// status[1]: CTAs that left the grid barrier as aborted; err_flag set by the
// CTAs that gave up).  bar: chain_run_bar_words() zeroed words.
cudaError_t launch_selftest_waits(unsigned *bar, int *err_flag, int *status, cudaStream_t s);

// FP32 FMA throughput kernel on `sms` SMs: fma_peak_flop() FLOP per launch,
// fma_peak_out_floats() floats written to out.
int fma_peak_blocks(int sms);
double fma_peak_flop(int sms, int iters);
size_t fma_peak_out_floats(int sms);
cudaError_t launch_fma_peak(float *out, int sms, int iters, cudaStream_t s);

struct FinishArgs {
    int mode;                // 0 materialised (GEMV partials), 1 fused (split partials)
    int N, l;
    int vlen;
    // materialised partial layout
    int tiles_per_slab, tiles_per_cta;
    // fused partial layout
    int nparts, ld_part;
    const float *part;
    float *y, *pi, *d1, *d2;
    const float *rowsum;     // materialised: r_i
    const float *rho;        // fused: u_k / r'_k
    float *v;                // next broadcast vector
    ChainState *state;
    float *blk;              // per-CTA partial sums of the finish stages [finish_blk_floats(vlen)]
    int *ticket;             // [2] CTA arrival counters of the finish stages, zero between launches
};

struct SpectralArgs {
    const PixelDev *px;      // work list (index = caller position)
    int n;
    int npad_max;
    int pi_iters;            // power steps for pi (stops early at a 1e-7 step)
    int subspace_iters;      // orthogonal-iteration steps
    float *out;              // [n][2]: |lambda_2|, |arg lambda_2|
    PixelConst *pconst;      // [n] per-pixel constants, written by launch_spectral
};

size_t spectral_smem_bytes(int npad);
cudaError_t launch_spectral(const SpectralArgs &a, int grid, cudaStream_t s);

int batch_threads_for(int nmax);
size_t batch_smem_bytes(int npad, int level);
int batch_state_level(int npad, bool structured);
int batch_pad_len(int n);
cudaError_t batch_occupancy(int threads, int level, bool structured, size_t smem, int *blocks_per_sm, int cols = 8);
// The per-pixel constants of a work list (one thread per pixel); launch_batch
// and launch_spectral run it before their kernels.
cudaError_t launch_pixel_const(const PixelDev *px, int n, PixelConst *out, cudaStream_t s);

// Host-buffer batch shared by the plain and learned host entry points: pmfs
// into h_out (packed in caller order), reports into h_reports (may be NULL);
// the warm start is d_warm (device, warm_kind / warm_ld as the batch options),
// or h_warm (host weights), or none.
spl_status_t batch_host_run(const spl_pixel_t *h_pixels, int32_t n, double tol, int32_t max_iter,
                            const float *d_warm, const float *h_warm, int warm_kind, int warm_ld, float *h_out,
                            spl_report_t *h_reports, cudaStream_t s, const spl_batch_opts_t *opts);
cudaError_t launch_batch(const BatchArgs &a, int threads, int grid, size_t smem, cudaStream_t s);

cudaError_t launch_chain_flux(const PixelDev &p, float *w, float *u, float *lam, double *F, double *scal,
                              int npad, cudaStream_t s);
cudaError_t launch_build_matrix(int N, int l, int ld, const float *w, const float *u, const double *scal, float *P,
                                float *rowsum, int num_sms, cudaStream_t s);
size_t gemv_smem_bytes();
int gemv_slab_cols();
cudaError_t launch_gemv(const CUtensorMap *map, const GemvArgs &a, int grid, cudaStream_t s);

int split_cols_per_cta();
int split_pad_len(int n);
cudaError_t launch_tri_split(const TriSplitArgs &a, bool row_pass, int chunks, cudaStream_t s);
cudaError_t launch_finish_rows(int N, int nparts, int ld_part, const float *part, const float *u, float *rho,
                               float *rowsum_p, int l, cudaStream_t s);
cudaError_t launch_finish_step(const FinishArgs &a, cudaStream_t s);
size_t finish_blk_floats(int vlen);
cudaError_t launch_init_iter(const FinishArgs &a, const float *warm, cudaStream_t s);

}  // namespace spl
