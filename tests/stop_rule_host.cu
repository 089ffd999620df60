// Host build of the power iteration's stop rule for CPU tests: replays a
// sequence of step vectors d_k = pi_k - pi_{k-1} through the same
// stop_update the batch kernel runs, with the step statistics the kernel
// reduces (||d_k||_1, <d_k,d_k>, <d_k,d_{k-1}>, <d_k,d_{k-2}>).
#include <cmath>
#include <cstddef>

#include "../paper_2509_20500_gb300/csrc/spl_device.cuh"

// Returns the step at which the rule ended (negative if it ended on an FP32
// floor above the tolerance), 0 if it never did within K steps.  tau is the
// a priori bound on |lambda_2| (1: none); rho_floor as the kernels set it for
// a warm start (0: a cold start).
extern "C" int stop_rule_replay_warm(const double *d, int K, int M, float tol_err, int min_iter, float tau,
                                     float rho_floor, float *err_out, float *rho_out, float *theta_out,
                                     int *reliable_out) {
    spl::StopState s;
    spl::stop_init(s, tau, rho_floor);
    int stop = 0;
    for (int k = 0; k < K; ++k) {
        const double *dk = d + (size_t)k * M;
        const double *dp = k >= 1 ? dk - M : nullptr;
        const double *dq = k >= 2 ? dk - 2 * (size_t)M : nullptr;
        double l1 = 0.0, dd = 0.0, d1 = 0.0, d2 = 0.0;
        for (int m = 0; m < M; ++m) {
            l1 += std::fabs(dk[m]);
            dd += dk[m] * dk[m];
            if (dp) d1 += dk[m] * dp[m];
            if (dq) d2 += dk[m] * dq[m];
        }
        const int r = spl::stop_update(s, (float)l1, (float)dd, (float)d1, (float)d2, tol_err, min_iter);
        if (r != spl::STOP_CONTINUE) {
            stop = r == spl::STOP_CONVERGED ? k + 1 : -(k + 1);
            break;
        }
    }
    *err_out = s.err;
    *rho_out = s.rho;
    *theta_out = s.theta;
    *reliable_out = s.reliable;
    return stop;
}

// A cold start (no warm-start floor).
extern "C" int stop_rule_replay(const double *d, int K, int M, float tol_err, int min_iter, float tau,
                                float *err_out, float *rho_out, float *theta_out, int *reliable_out) {
    return stop_rule_replay_warm(d, K, M, tol_err, min_iter, tau, 0.f, err_out, rho_out, theta_out,
                                 reliable_out);
}

// The warm-start floor the kernels use.
extern "C" float stop_rule_warm_floor(void) { return spl::kWarmRhoFloor; }
