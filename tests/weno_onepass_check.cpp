// Host check of the one-pass WENO-AO combination of the device header
// (weno_ao, weno_ao_sp compiled for the host): for seeded stencils of every
// scale it compares the returned quadratic with the combination written out
// in the paper's form, eqs. (para) and (nonlinear) of Sec. 2: tau the mean of
// |beta0 - beta_m|, w = gamma (1 + (tau/(beta + eps))^p), normalised, and
// P~ = (w0/g0) P0 + sum (w_m - w0 g_m/g0) P_m, for p = 1 and 2.  The
// polynomials, indicators and stencils come from the same header.  Prints
// "ok" or the first failure.
#include <cmath>
#include <cstdio>
#include <random>
#define HK_HD inline
#include "hgks_device.cuh"

template <bool SP>
static void reference(const hk::Stencil<double> &st, const hk::Scheme &S, double out[9])
{
    const int nsub = SP ? 8 : 24;
    const double g0 = 1.0 - nsub * S.Gamma_lin, gm = S.Gamma_lin, eps = S.weno_eps;
    double a[9];
    if (SP) hk::big_stencil_P0_sp(st, a);
    else hk::big_stencil_P0(st, a);
    const double beta0 = hk::beta_quadratic(a);
    double b[24][3], beta[24], tau = 0.0;
    for (int m = 0; m < nsub; ++m) {
        if (SP) hk::sub_stencil_sp_rt(st, m, b[m]);
        else hk::sub_stencil_rt(st, m, b[m]);
        beta[m] = b[m][0] * b[m][0] + b[m][1] * b[m][1] + b[m][2] * b[m][2];
        tau += std::fabs(beta0 - beta[m]);
    }
    tau /= nsub;
    const int p = S.weno_pow;
    const double w0 = g0 * (1.0 + std::pow(tau / (beta0 + eps), p));
    double wsum = w0, lin[3] = {0, 0, 0};
    for (int m = 0; m < nsub; ++m) {
        const double wm = gm * (1.0 + std::pow(tau / (beta[m] + eps), p));
        wsum += wm;
        for (int d = 0; d < 3; ++d) lin[d] += (wm - w0 * gm / g0) * b[m][d];
    }
    for (int n = 0; n < 9; ++n) out[n] = ((w0 / g0) * a[n] + (n < 3 ? lin[n] : 0.0)) / wsum;
}

int main()
{
    std::mt19937_64 rng(2024);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    std::uniform_real_distribution<double> lg(-9.0, 1.0);
    hk::Scheme S{};
    S.gamma = 1.4;
    S.Gamma_lin = 0.0025;
    double worst = 0.0;
    for (int trial = 0; trial < 20000; ++trial) {
        S.weno_pow = 1 + (trial & 1);
        S.weno_eps = (trial % 3 == 0) ? 1e-8 : std::pow(10.0, lg(rng) - 3.0);
        const double scale = std::pow(10.0, lg(rng));
        hk::Stencil<double> st;
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                st.f[d][s] = scale * u(rng);
                st.f2[d][s] = scale * u(rng);
                st.e[d][s][0] = scale * u(rng);
                st.e[d][s][1] = scale * u(rng);
            }
        if (trial % 5 == 0) {  // smooth data: a linear field plus a small perturbation
            const double gx = u(rng), gy = u(rng), gz = u(rng);
            const double g[3] = {gx, gy, gz};
            for (int d = 0; d < 3; ++d) {
                st.f[d][1] = g[d] + 1e-6 * u(rng);
                st.f[d][0] = -g[d] + 1e-6 * u(rng);
                st.f2[d][1] = 2 * g[d];
                st.f2[d][0] = -2 * g[d];
                for (int sa = 0; sa < 2; ++sa)
                    for (int sb = 0; sb < 2; ++sb)
                        st.e[d][sa][sb] = (sa ? 1 : -1) * g[d] + (sb ? 1 : -1) * g[(d + 1) % 3] + 1e-6 * u(rng);
            }
        }
        for (int sp = 0; sp < 2; ++sp) {
            double got[9], ref[9], rad;
            if (sp) {
                hk::weno_ao_sp(st, S, got, rad);
                reference<true>(st, S, ref);
            } else {
                hk::weno_ao(st, S, got, rad);
                reference<false>(st, S, ref);
            }
            double m = 0.0;
            for (int n = 0; n < 9; ++n) m = std::fmax(m, std::fabs(ref[n]));
            for (int n = 0; n < 9; ++n) {
                const double err = std::fabs(got[n] - ref[n]) / (m > 0 ? m : 1.0);
                worst = std::fmax(worst, err);
                if (!(err <= 1e-12)) {
                    printf("FAIL trial %d sp %d p %d n %d got %.17g ref %.17g\n", trial, sp, S.weno_pow, n, got[n],
                           ref[n]);
                    return 1;
                }
            }
        }
    }
    printf("ok worst %.3g\n", worst);
    return 0;
}
