// Host build of the Gauss-point flux of the device header (gks_flux, in
// FP64 or FP32) for the host test of the flux arithmetic: reads n points of
// 40 values (left state, its three directional derivatives, right state,
// its derivatives, local frame) from a binary file and writes n x 10 values
// (F, dF/dt) to another.  Usage: flux_host_check R dt gamma mu Pr tau_eps
// tau_C n in out [gs], R = 64 or 32; with gs the gradients are passed as
// dW/gs together with the gradient scale gs (the uniform mesh's scaled
// frame), which must give the same flux.
#include <cstdio>
#include <cstdlib>
#include <vector>
#define HK_HD inline
#include "hgks_device.cuh"

template <typename R>
static void run(const hk::Scheme &S, double dt, double gs, int n, const std::vector<double> &in,
                std::vector<double> &out)
{
    for (int p = 0; p < n; ++p) {
        const double *x = in.data() + 40 * (size_t)p;
        R W[2][5], dW[2][3][5];
        for (int s = 0; s < 2; ++s)
            for (int v = 0; v < 5; ++v) {
                W[s][v] = R(x[20 * s + v]);
                for (int e = 0; e < 3; ++e) dW[s][e][v] = R(x[20 * s + 5 + 5 * e + v] / gs);
            }
        R F[5], dF[5];
        hk::gks_flux<R>(W[0], dW[0], W[1], dW[1], S, R(dt), F, dF, R(gs));
        for (int v = 0; v < 5; ++v) {
            out[10 * (size_t)p + v] = double(F[v]);
            out[10 * (size_t)p + 5 + v] = double(dF[v]);
        }
    }
}

int main(int argc, char **argv)
{
    if (argc != 11 && argc != 12) return 2;
    const double gs = argc == 12 ? atof(argv[11]) : 1.0;
    const int prec = atoi(argv[1]);
    const double dt = atof(argv[2]);
    hk::Scheme S{};
    S.gamma = atof(argv[3]);
    S.K = (5.0 - 3.0 * S.gamma) / (S.gamma - 1.0);
    S.mu = atof(argv[4]);
    S.Pr = atof(argv[5]);
    S.tau_eps = atof(argv[6]);
    S.tau_C = atof(argv[7]);
    S.weno_eps = 1e-8;
    S.Gamma_lin = 0.0025;
    S.weno_pow = 1;
    S.limiter = 1;
    hk::scheme_derive(S);
    const int n = atoi(argv[8]);
    std::vector<double> in(40 * (size_t)n), out(10 * (size_t)n);
    FILE *f = fopen(argv[9], "rb");
    if (!f || fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
    fclose(f);
    if (prec == 32) run<float>(S, dt, gs, n, in, out);
    else run<double>(S, dt, gs, n, in, out);
    f = fopen(argv[10], "wb");
    if (!f || fwrite(out.data(), sizeof(double), out.size(), f) != out.size()) return 4;
    fclose(f);
    return 0;
}
