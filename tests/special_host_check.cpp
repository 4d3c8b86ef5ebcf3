// Host build of erfc_half (the half-space erfc of the device header) for the
// host test of its accuracy: prints the largest relative difference from the
// C library's erfc (long double) over a dense grid of [-0.75, 0.75] (the
// series branch) and of [-3, 3] (both branches), in FP64 and FP32; then the
// largest relative difference of pow_pos from powl over [1/4, 4].
#include <cmath>
#include <cstdio>
#define HK_HD inline
#include "hgks_device.cuh"

template <typename R> static double worst(double lo, double hi, int n)
{
    double w = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double x = lo + (hi - lo) * i / n;
        const R xr = R(x);
        const long double ref = erfcl((long double)xr);
        const double got = double(hk::erfc_half<R>(xr));
        const double rel = (double)fabsl(((long double)got - ref) / ref);
        if (rel > w) w = rel;
    }
    return w;
}

// pow_pos (x^y as exp(y log x), the viscosity law's power) against the
// long-double pow over x in [lo, hi] for y = 0.76
template <typename R> static double worst_pow(double lo, double hi, int n)
{
    double w = 0.0;
    for (int i = 0; i <= n; ++i) {
        const R x = R(lo + (hi - lo) * i / n);
        const long double ref = powl((long double)x, (long double)R(0.76));
        const double got = double(hk::pow_pos<R>(x, R(0.76)));
        const double rel = (double)fabsl(((long double)got - ref) / ref);
        if (rel > w) w = rel;
    }
    return w;
}

int main()
{
    printf("%.3e %.3e %.3e %.3e %.3e %.3e\n", worst<double>(-0.75, 0.75, 200000), worst<double>(-3.0, 3.0, 200000),
           worst<float>(-0.75, 0.75, 200000), worst<float>(-3.0, 3.0, 200000), worst_pow<double>(0.25, 4.0, 200000),
           worst_pow<float>(0.25, 4.0, 200000));
    return 0;
}
