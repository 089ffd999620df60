// Host build of the batch kernel's own FP64 helpers for CPU tests:
// exp_series (the exponential of the pulse-bin factors) and pow_uint (the
// geometric tables of the tail factors), from the same header the kernels use.
#include "../paper_2509_20500_gb300/csrc/spl_device.cuh"

extern "C" void exp_series_host(const double *x, double *y, int n) {
    for (int i = 0; i < n; ++i) y[i] = spl::exp_series(x[i]);
}

extern "C" void pow_uint_host(const double *x, const int *e, double *y, int n) {
    for (int i = 0; i < n; ++i) y[i] = spl::pow_uint(x[i], e[i]);
}
