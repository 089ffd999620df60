// Host thread pool for the per-pixel host work of a batch call (building the
// work list of 65536 pixels takes about 0.5 ms on one core, during which the
// GPU would otherwise wait).
//
// run(nchunks, fn) calls fn(i) once for every i in [0, nchunks), on the pool's
// workers and the calling thread, and returns when every call has finished.
// Runs from several host threads are serialised.  The workers are started on
// first use and detached (the pool is never destroyed, so process exit does
// not wait on them).  In a process forked after the pool started the workers
// do not exist; there, and for a single chunk, run() calls fn on the calling
// thread in order.
#pragma once

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>

namespace spl {

class HostPool {
  public:
    static HostPool &get() {
        static HostPool *pool = new HostPool();
        return *pool;
    }

    void run(int nchunks, const std::function<void(int)> &fn) {
        if (nchunks <= 1 || nworkers_ == 0 || getpid() != pid_) {
            for (int i = 0; i < nchunks; ++i) fn(i);
            return;
        }
        std::lock_guard<std::mutex> one_run(run_mu_);
        {
            std::lock_guard<std::mutex> lk(mu_);
            task_ = &fn;
            nchunks_ = nchunks;
            next_.store(0);
            ++gen_;
        }
        cv_work_.notify_all();
        for (int i; (i = next_.fetch_add(1)) < nchunks;) fn(i);
        std::unique_lock<std::mutex> lk(mu_);
        // every chunk was claimed; wait for the workers still running one
        cv_done_.wait(lk, [&] { return active_ == 0; });
        task_ = nullptr;
    }

  private:
    HostPool() : pid_(getpid()) {
        const unsigned hw = std::thread::hardware_concurrency();
        nworkers_ = (int)std::min(7u, hw > 1 ? hw - 1 : 0u);
        for (int w = 0; w < nworkers_; ++w) std::thread([this] { worker(); }).detach();
    }

    void worker() {
        unsigned seen = 0;
        for (;;) {
            std::unique_lock<std::mutex> lk(mu_);
            cv_work_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            const std::function<void(int)> *task = task_;
            const int n = nchunks_;
            ++active_;
            lk.unlock();
            // a worker that wakes after its run ended finds every chunk claimed
            for (int i; task && (i = next_.fetch_add(1)) < n;) (*task)(i);
            lk.lock();
            if (--active_ == 0) cv_done_.notify_all();
        }
    }

    std::mutex run_mu_, mu_;
    std::condition_variable cv_work_, cv_done_;
    const std::function<void(int)> *task_ = nullptr;
    int nchunks_ = 0, active_ = 0, nworkers_ = 0;
    unsigned gen_ = 0;
    std::atomic<int> next_{0};
    pid_t pid_;
};

// fn(lo, hi) over [0, n) in chunks of at least min_chunk items (at most 16
// chunks), on the pool.
template <class F>
void host_parallel_for(int64_t n, int64_t min_chunk, F &&fn) {
    const int64_t nc = std::max<int64_t>(1, std::min<int64_t>(16, n / std::max<int64_t>(1, min_chunk)));
    const int64_t step = (n + nc - 1) / nc;
    HostPool::get().run((int)nc, [&](int c) {
        const int64_t lo = c * step, hi = std::min(n, lo + step);
        if (lo < hi) fn(lo, hi);
    });
}

}  // namespace spl
