// Operation counter of the hot-path arithmetic: instantiates the device
// templates of hgks_device.cuh on the host with a counting scalar and prints
// the counts per unit of work (one cell reconstruction, one Gauss-point
// flux).  A measurement tool for the roofline; not part of the library.
#include <cstdio>
#include <cmath>
// plain host build: the device qualifiers of the header become inline
#define HK_HD inline
#include "hgks_device.cuh"

struct Counts {
    long add = 0, mul = 0, div = 0, sqrt = 0, rsqrt = 0, exp = 0, expm1 = 0, erfc = 0, log = 0;
    void reset() { *this = Counts(); }
};
static Counts C;

struct CR {
    double v;
    CR() : v(0) {}
    CR(double x) : v(x) {}
};
inline CR operator+(CR a, CR b) { ++C.add; return CR(a.v + b.v); }
inline CR operator-(CR a, CR b) { ++C.add; return CR(a.v - b.v); }
inline CR operator*(CR a, CR b) { ++C.mul; return CR(a.v * b.v); }
inline CR operator/(CR a, CR b) { ++C.div; return CR(a.v / b.v); }
inline CR operator-(CR a) { return CR(-a.v); }
inline CR &operator+=(CR &a, CR b) { a = a + b; return a; }
inline CR &operator-=(CR &a, CR b) { a = a - b; return a; }
inline CR &operator*=(CR &a, CR b) { a = a * b; return a; }
inline bool operator<(CR a, CR b) { return a.v < b.v; }
inline bool operator>(CR a, CR b) { return a.v > b.v; }
inline CR m_exp(CR a) { ++C.exp; return CR(std::exp(a.v)); }
inline CR m_expm1(CR a) { ++C.expm1; return CR(std::expm1(a.v)); }
inline CR m_erfc(CR a) { ++C.erfc; return CR(std::erfc(a.v)); }
inline CR m_log(CR a) { ++C.log; return CR(std::log(a.v)); }
inline CR m_sqrt(CR a) { ++C.sqrt; return CR(std::sqrt(a.v)); }
inline CR m_rsqrt(CR a) { ++C.rsqrt; return CR(1.0 / std::sqrt(a.v)); }
inline CR m_abs(CR a) { return CR(std::fabs(a.v)); }
inline CR m_max(CR a, CR b) { return CR(a.v > b.v ? a.v : b.v); }

static void print(const char *name, long scale_num = 1)
{
    long fl = C.add + C.mul;
    printf("  \"%s\": {\"add\": %ld, \"mul\": %ld, \"div\": %ld, \"sqrt\": %ld, \"rsqrt\": %ld, \"exp\": %ld, "
           "\"expm1\": %ld, \"erfc\": %ld, \"addmul\": %ld}",
           name, C.add, C.mul, C.div, C.sqrt, C.rsqrt, C.exp, C.expm1, C.erfc, fl);
    (void)scale_num;
}

int main()
{
    hk::Scheme S;
    S.gamma = 1.4; S.K = 2.0; S.mu = 0.0; S.Pr = 1.0; S.tau_eps = 0.01; S.tau_C = 1.0;
    S.weno_eps = 1e-8; S.Gamma_lin = 0.0025; S.weno_pow = 1; S.limiter = 1;
    hk::scheme_derive(S);
    printf("{\n");
    // reconstruction of one cell: 5 variables and the positivity test
    C.reset();
    CR qc[5] = {1.0, 0.1, 0.2, 0.3, 2.6}, rad[5];
    for (int v = 0; v < 5; ++v) {
        hk::Stencil<CR> st;
        for (int d = 0; d < 3; ++d) { st.f[d][0] = CR(-0.01 * (d + 1)); st.f[d][1] = CR(0.012 * (d + 1)); }
        for (int p = 0; p < 3; ++p)
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) st.e[p][a][b] = CR(0.003 * (p + 1) * (a - b + 0.5));
        CR out[9];
        hk::weno_ao(st, S, out, rad[v]);
    }
    hk::positivity_certain(qc, rad, CR(1.4));
    print("recon_cell");
    printf(",\n");
    // one Gauss point: both sides' values and gradients, then the flux
    for (int viscous = 0; viscous < 2; ++viscous) {
        S.mu = viscous ? 1e-3 : 0.0;
        S.Pr = viscous ? 0.72 : 1.0;
        hk::scheme_derive(S);
        C.reset();
        CR X[3] = {0.5, 0.288, -0.288}, ih = 16.0;
        CR W[2][5], dW[2][3][5];
        const double base[5] = {1.0, 0.2, -0.1, 0.05, 2.6};
        for (int s = 0; s < 2; ++s)
            for (int v = 0; v < 5; ++v) {
                CR c[9], sv, gr[3];
                for (int n = 0; n < 9; ++n) c[n] = CR(0.001 * (n + 1) * (v + 1));
                hk::poly_value_grad(c, X, ih, sv, gr);
                W[s][v] = CR(base[v] + sv.v * (1 + 0.1 * s));
                for (int d = 0; d < 3; ++d) dW[s][d][v] = gr[d];
            }
        CR F[5], dF[5];
        hk::gks_flux(W[0], dW[0], W[1], dW[1], S, CR(1e-3), F, dF);
        print(viscous ? "gauss_point_ns_pr" : "gauss_point_euler");
        printf(viscous ? "\n" : ",\n");
    }
    printf("}\n");
    return 0;
}
