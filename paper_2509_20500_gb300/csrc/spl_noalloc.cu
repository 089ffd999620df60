// spl_batch_stationary_noalloc: the batch solver without any allocation.
//
// Some callers may not allocate device memory at all: real-time sensor
// pipelines that ban allocation after start-up (cudaMalloc can synchronise
// the whole device and its latency is unbounded), and plug-ins running
// inside a host application whose own allocator owns the GPU memory budget.
// This entry point serves them.  It runs the same persistent batch kernel as
// spl_batch_stationary, but every piece of device scratch the kernel needs
// (work list, work-queue counter, per-pixel reports, per-pixel flux
// constants) lives in one file-scope __device__ array of fixed size (about
// 15.2 MB), and the host-side staging lives
// in static host arrays.  It calls no cudaMalloc, cudaFree, cudaMallocHost
// or any other allocating routine.
//
// Limits: at most kNoAllocMaxPixels pixels per call and at most
// kNoAllocMaxBins bins per pixel (with that many bins the per-pixel state of
// the kernel stays in shared memory, so no per-block global scratch is
// needed).  Larger requests return SPL_EINVAL.
//
// Every GPU that loads this library holds the array until the process
// exits.  With lazy module loading (the CUDA default) the array is reserved
// when this file's module is first loaded on a device, which the first
// call's cudaGetSymbolAddress does: that first call may therefore reserve
// memory and synchronise the device, so make it during start-up, before any
// stream capture.  All calls share it and it keeps the previous call's contents;
// what must start at zero (the work-queue counter) is cleared by each call.
// Two calls whose work overlaps on the GPU (for example on two streams)
// race on the array; issue them one after the other.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "spl.h"
#include "spl_kernels.h"

using namespace spl;

namespace {

constexpr int kNoAllocMaxPixels = 65536;
constexpr int kNoAllocMaxBins = 3072;

constexpr size_t kCounterBytes = 256;
constexpr size_t kWorkBytes = sizeof(PixelDev) * kNoAllocMaxPixels;
constexpr size_t kReportBytes = sizeof(ReportDev) * kNoAllocMaxPixels;
constexpr size_t kConstBytes = sizeof(PixelConst) * kNoAllocMaxPixels;
constexpr size_t kScratchBytes = kCounterBytes + kWorkBytes + kReportBytes + kConstBytes;
static_assert(kScratchBytes == 15204608, "scratch size stated in the header");

// The scratch array: 256 B counter + 64 B x 65536 work list + 24 B x 65536
// reports + 144 B x 65536 per-pixel constants = 15,204,608 bytes.  Host code must not use its name as an
// address: it is a host-side stand-in.  The device address comes from
// cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side staging, static as well.
static PixelDev g_host_work[kNoAllocMaxPixels];
static int32_t g_count_by_n[kNoAllocMaxBins + 2];

constexpr int kMaxDev = 64;
static void *g_dev_scratch[kMaxDev];
static std::mutex g_mu;

// Per-device set-up: the device address of the scratch array, looked up once
// with that device current.
spl_status_t scratch_ptr(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return SPL_ECUDA;
    if (!g_dev_scratch[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return SPL_ECUDA;
        g_dev_scratch[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_dev_scratch[dev]);
    return SPL_OK;
}

int sm_count() {
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

extern "C" spl_status_t spl_batch_stationary_noalloc(const spl_pixel_t *h_pixels, int32_t n, double tol,
                                                     int32_t max_iter, const float *d_warm, float *d_out,
                                                     const int64_t *d_offsets, spl_report_t *h_reports,
                                                     void *stream) {
    if (n < 0 || n > kNoAllocMaxPixels) return SPL_EINVAL;
    if (n > 0 && (!h_pixels || !d_out || !d_offsets)) return SPL_EINVAL;
    if (!(tol > 0.0) || max_iter < 1) return SPL_EINVAL;
    if (n == 0) return SPL_OK;
    for (int32_t k = 0; k < n; ++k)
        if (h_pixels[k].n_bins < 2 || h_pixels[k].n_bins > kNoAllocMaxBins) return SPL_EINVAL;

    std::lock_guard<std::mutex> lock(g_mu);
    unsigned char *base = nullptr;
    spl_status_t st = scratch_ptr(&base);
    if (st != SPL_OK) return st;
    int *d_counter = reinterpret_cast<int *>(base);
    PixelDev *d_work = reinterpret_cast<PixelDev *>(base + kCounterBytes);
    ReportDev *d_reps = reinterpret_cast<ReportDev *>(base + kCounterBytes + kWorkBytes);
    PixelConst *d_const = reinterpret_cast<PixelConst *>(base + kCounterBytes + kWorkBytes + kReportBytes);
    static_assert((kCounterBytes + kWorkBytes + kReportBytes) % alignof(PixelConst) == 0, "constants alignment");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Work list ordered by decreasing n_bins (counting sort, stable in the
    // caller's order), written into the static host staging array.
    std::memset(g_count_by_n, 0, sizeof(g_count_by_n));
    int nmax = 2;
    for (int32_t k = 0; k < n; ++k) {
        g_count_by_n[h_pixels[k].n_bins] += 1;
        if (h_pixels[k].n_bins > nmax) nmax = h_pixels[k].n_bins;
    }
    int32_t pos = 0;
    for (int nb = kNoAllocMaxBins; nb >= 2; --nb) {
        const int32_t c = g_count_by_n[nb];
        g_count_by_n[nb] = pos;
        pos += c;
    }
    for (int32_t k = 0; k < n; ++k) {
        PixelDev d;
        st = make_pixel(h_pixels[k], d);   // validation and row shift of every entry point
        if (st != SPL_OK) return st;
        d.index = k;
        g_host_work[g_count_by_n[d.N]++] = d;
    }

    const int threads = batch_threads_for(nmax);
    const int npad = batch_pad_len(nmax);
    if (batch_state_level(npad, false) != 2) return SPL_EINVAL;
    const size_t smem = batch_smem_bytes(npad, 2);
    int bps = 0;
    cudaError_t e = batch_occupancy(threads, 2, false, smem, &bps);
    if (e != cudaSuccess || bps < 1) return SPL_ECUDA;
    int grid = bps * sm_count();
    if (grid > n) grid = n;

    // Pageable source: the call returns once the data is staged, so the
    // static host array may be reused by the next call.
    if (cudaMemcpyAsync(d_work, g_host_work, sizeof(PixelDev) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SPL_ECUDA;
    if (cudaMemsetAsync(d_counter, 0, sizeof(int), s) != cudaSuccess) return SPL_ECUDA;

    BatchArgs a{};
    a.px = d_work;
    a.n = n;
    a.counter = d_counter;
    a.warm = d_warm;
    a.warm_kind = 0;
    a.warm_ld = 0;
    a.out = d_out;
    a.offsets = d_offsets;
    a.reports = d_reps;
    a.scratch = nullptr;          // per-pixel state stays in shared memory at these sizes
    a.npad_max = npad;
    a.state_level = 2;
    a.tol_err = (float)(0.5 * tol);
    a.max_iter = max_iter;
    a.min_iter = 1;
    a.structured = 0;
    a.pconst = d_const;
    if (launch_batch(a, threads, grid, smem, s) != cudaSuccess) return SPL_ECUDA;

    if (!h_reports) return SPL_OK;
    // spl_report_t and the device record have the same layout.
    static_assert(sizeof(spl_report_t) == sizeof(ReportDev), "report layout");
    if (cudaMemcpyAsync(h_reports, d_reps, sizeof(ReportDev) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPL_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPL_ECUDA;
    spl_status_t worst = SPL_OK;
    for (int32_t k = 0; k < n; ++k)
        if (h_reports[k].status > (int)worst) worst = (spl_status_t)h_reports[k].status;
    return worst;
}
