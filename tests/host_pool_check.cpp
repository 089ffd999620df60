// Host check of the batch calls' thread pool (spl_host_pool.h): every chunk
// runs exactly once, runs from several threads are serialised correctly, the
// chunked loop covers [0, n) once, and a forked child (no workers) still
// completes its runs on the calling thread.
#include <sys/wait.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "spl_host_pool.h"

static int check_runs(int reps, int nchunks) {
    for (int r = 0; r < reps; ++r) {
        std::vector<std::atomic<int>> hits(nchunks);
        for (auto &h : hits) h.store(0);
        spl::HostPool::get().run(nchunks, [&](int i) { hits[i].fetch_add(1); });
        for (int i = 0; i < nchunks; ++i)
            if (hits[i].load() != 1) return 1;
    }
    return 0;
}

static int check_for(int64_t n, int64_t min_chunk) {
    std::vector<std::atomic<int>> hits(n);
    for (auto &h : hits) h.store(0);
    spl::host_parallel_for(n, min_chunk, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) hits[i].fetch_add(1);
    });
    for (int64_t i = 0; i < n; ++i)
        if (hits[i].load() != 1) return 1;
    return 0;
}

int main() {
    int bad = 0;
    bad += check_runs(2000, 16);
    bad += check_runs(200, 1);
    bad += check_runs(200, 100);
    for (int64_t n : {0, 1, 7, 4095, 4096, 65536, 100003}) bad += check_for(n, 4096);
    // four host threads running at once
    std::atomic<int> tb{0};
    std::vector<std::thread> ts;
    for (int t = 0; t < 4; ++t) ts.emplace_back([&] { tb += check_runs(300, 16); });
    for (auto &t : ts) t.join();
    bad += tb.load();
    // a forked child: the pool's workers are not there; runs still complete
    const pid_t pid = fork();
    if (pid == 0) _exit(check_runs(50, 16) + check_for(65536, 4096));
    int status = 0;
    waitpid(pid, &status, 0);
    bad += (WIFEXITED(status) && WEXITSTATUS(status) == 0) ? 0 : 1;
    std::printf("%s\n", bad ? "FAIL" : "ok");
    return bad ? 1 : 0;
}
