// Device arithmetic of the HGKS hot path for sm_103a: WENO-AO
// reconstruction on a uniform mesh of cubes (Sec. 2) and the gas-kinetic
// flux at a Gauss point (Sec. 3).  Everything is templated on the working
// precision R (double for the FP64 path, float for the mixed path).
#pragma once
#include <string.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

// host+device inline: the arithmetic below also compiles for the host so
// that the operation counter (opcount.cu) can instantiate it
#ifndef HK_HD
#define HK_HD __host__ __device__ __forceinline__
#endif

namespace hk {

// ---------------------------------------------------------------------------
// math overloads
// ---------------------------------------------------------------------------
HK_HD double m_exp(double x) { return exp(x); }
HK_HD float m_exp(float x) { return expf(x); }
HK_HD double m_expm1(double x) { return expm1(x); }
HK_HD float m_expm1(float x) { return expm1f(x); }
HK_HD double m_erfc(double x) { return erfc(x); }
HK_HD float m_erfc(float x) { return erfcf(x); }
HK_HD double m_sqrt(double x) { return sqrt(x); }
HK_HD float m_sqrt(float x) { return sqrtf(x); }
#ifdef __CUDA_ARCH__
HK_HD double m_rsqrt(double x) { return rsqrt(x); }
HK_HD float m_rsqrt(float x) { return rsqrtf(x); }
#else
HK_HD double m_rsqrt(double x) { return 1.0 / sqrt(x); }
HK_HD float m_rsqrt(float x) { return 1.0f / sqrtf(x); }
#endif
HK_HD double m_abs(double x) { return fabs(x); }
HK_HD double m_max(double a, double b) { return fmax(a, b); }
HK_HD float m_max(float a, float b) { return fmaxf(a, b); }
HK_HD float m_abs(float x) { return fabsf(x); }
HK_HD double m_log(double x) { return log(x); }
HK_HD float m_log(float x) { return logf(x); }
// x^y for x >= 0 as exp(y log x): the library's exp and log cost this GPU
// far fewer FP64 operations than its pow, and for the viscosity law's
// arguments (x = T/T_ref near 1, y = 0.76) the relative error stays at a
// few units in the last place, |y log x| being small
template <typename R> HK_HD R pow_pos(R x, R y) { return m_exp(y * m_log(x)); }

// Constants of the Gauss-point flux in one working precision, derived on the
// host (scheme_derive) so that no thread converts or divides them.
template <typename R> struct FluxK {
    R gamma, K, Kp3, iKp3, gm1;  // gamma, K, K + 3, 1/(K + 3), gamma - 1
    R mu2;                       // 2 mu
    R tau_eps, tau_C;
    R prfac;                     // 1/Pr - 1
    R mu_pow, iT_ref;            // viscosity law mu (T/T_ref)^mu_pow
};

// Scheme constants, passed by value to every kernel.  After any change of
// the fields above kd/kf, scheme_derive() must be called.
struct Scheme {
    double gamma;      // ratio of specific heats
    double K;          // internal degrees of freedom (5 - 3 gamma)/(gamma - 1)
    double mu, Pr;     // viscosity (0: Euler collision time) and Prandtl number
    double tau_eps, tau_C;
    double weno_eps;   // epsilon of the nonlinear weights
    double Gamma_lin;  // linear weight of each sub-stencil
    int weno_pow;      // exponent on tau/(beta + eps)
    int limiter;       // positivity fallback on/off
    int sprime = 0;       // 1: big stencil S' with 8 sub-stencils (Remark of Sec. 2)
    double mu_pow = 0.0;  // viscosity law mu (T/T_ref)^mu_pow (0: constant mu)
    double T_ref = 1.0;   // reference temperature p/rho of that law
    int viscous;       // mu > 0
    int prfix;         // mu > 0 and Pr != 1: Prandtl correction of the energy flux
    FluxK<double> kd;
    FluxK<float> kf;
};

template <typename R> HK_HD void fluxk_fill(const Scheme &S, FluxK<R> &k)
{
    k.gamma = R(S.gamma);
    k.K = R(S.K);
    k.Kp3 = R(S.K + 3.0);
    k.iKp3 = R(1.0 / (S.K + 3.0));
    k.gm1 = R(S.gamma - 1.0);
    k.mu2 = R(2.0 * S.mu);
    k.tau_eps = R(S.tau_eps);
    k.tau_C = R(S.tau_C);
    k.prfac = R(1.0 / S.Pr - 1.0);
    k.mu_pow = R(S.mu_pow);
    k.iT_ref = R(1.0 / S.T_ref);
}

inline void scheme_derive(Scheme &S)
{
    S.viscous = S.mu > 0.0;
    S.prfix = S.mu > 0.0 && S.Pr != 1.0;
    fluxk_fill(S, S.kd);
    fluxk_fill(S, S.kf);
}

// the constants in precision R: stored for double and float, converted for
// any other scalar (the host operation counter)
template <typename R> HK_HD FluxK<R> fluxk(const Scheme &S)
{
    FluxK<R> k;
    fluxk_fill(S, k);
    return k;
}
template <> HK_HD FluxK<double> fluxk<double>(const Scheme &S) { return S.kd; }
template <> HK_HD FluxK<float> fluxk<float>(const Scheme &S) { return S.kf; }

// Mesh: a uniform grid of cubes with GHOST = 3 ghost layers in the state
// arrays (the reconstruction of the ghost ring reaches two cells further
// with the big stencil S' of Sec. 2) and one ghost layer in the
// reconstruction arrays.
constexpr int GHOST = 3;
// Division by an invariant d >= 1 as a multiplication (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// the round-up method): with l = ceil(log2 d) and m = ceil(2^(31+l) / d),
// floor(n / d) = floor(m n / 2^(31+l)) for every 0 <= n < 2^31 (m d - 2^(31+l)
// < d <= 2^l); m < 2^32 for d <= 2^31.
struct Div32 {
    unsigned m;
    int s;
};
HK_HD Div32 div32_of(unsigned d)
{
    int l = 0;
    while (l < 31 && (1u << l) < d) ++l;
    const unsigned long long p = 1ull << (31 + l);
    return Div32{(unsigned)((p + d - 1) / d), 31 + l};
}
HK_HD unsigned div32(unsigned n, Div32 v) { return (unsigned)(((unsigned long long)v.m * n) >> v.s); }

struct Geo {
    int nx, ny, nz;          // interior cells
    int px, py, pz;          // padded state extents (n + 2 GHOST)
    int cx, cy, cz;          // reconstruction extents (n + 2)
    long long pstride;       // px*py*pz: variable stride of padded state arrays
    long long cstride;       // cx*cy*cz: term stride of coefficient arrays
    long long ncell;         // nx*ny*nz
    double h, inv_h;         // cell edge and its inverse
    int bc[6];               // per face: 0 periodic, 1 reflective, 2 outflow
    Div32 dv[4];             // division by nx, nx + 1, ny, ny + 1 (face index decode)
};

// the divisors of a Geo whose extents are set
inline void geo_divisors(Geo &g)
{
    g.dv[0] = div32_of((unsigned)g.nx);
    g.dv[1] = div32_of((unsigned)g.nx + 1u);
    g.dv[2] = div32_of((unsigned)g.ny);
    g.dv[3] = div32_of((unsigned)g.ny + 1u);
}

HK_HD long long pidx(const Geo &g, int i, int j, int k)
{
    return ((long long)(k + GHOST) * g.py + (j + GHOST)) * g.px + (i + GHOST);
}
// linear index -> (i, j, k) of an a x b x * box in 32-bit arithmetic (every
// box and face count of a handle fits: sizes are capped at creation)
HK_HD void split3(long long t, int a, int b, int &i, int &j, int &k)
{
    const unsigned u = (unsigned)t, ua = (unsigned)a, ub = (unsigned)b;
    const unsigned r = u / ua;
    i = (int)(u - r * ua);
    k = (int)(r / ub);
    j = (int)(r - (unsigned)k * ub);
}

// The split q = hi + lo of the mixed path, hi = fl32(q), lo = fl32(q - hi)
// (q - hi is exact in FP64), from the IEEE 754 bit fields of q with integer
// operations where hi and lo are both normal FP32 numbers (unbiased exponent
// of q in [-72, 126]); elsewhere (zeros, tiny or huge values, infinities,
// NaNs) by the FP64 arithmetic it replaces.  With q = M 2^(e-52), M the
// 53-bit significand: hi keeps the top 24 bits of M rounded to nearest,
// ties to even (a carry out renormalises); the residual q - hi is
// R 2^(e-52) with R the dropped 29 bits, minus 2^29 when hi rounded up, and
// lo is R rounded the same way to 24 bits.  The two FP32 conversions and
// the FP64 subtraction of the plain form run on this GPU's FP64 pipe.
HK_HD void split_f64(double q, float &hi, float &lo)
{
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
#else
    unsigned long long b;
    memcpy(&b, &q, 8);
#endif
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -72 || e > 126) {
        hi = float(q);
        lo = float(q - double(hi));
        return;
    }
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
    const unsigned drop = (unsigned)(M & 0x1fffffffu);  // the low 29 bits
    unsigned kept = (unsigned)(M >> 29);                 // 24 bits, top bit set
    const bool up = drop > 0x10000000u || (drop == 0x10000000u && (kept & 1u));
    int eh = e;
    kept += up ? 1u : 0u;
    if (kept == (1u << 24)) {
        kept = 1u << 23;
        eh += 1;
    }
    const unsigned hb = sgn | ((unsigned)(eh + 127) << 23) | (kept & 0x7fffffu);
    // residual R 2^(e-52), |R| <= 2^28
    const int R = up ? (int)drop - (1 << 29) : (int)drop;
    unsigned lb = 0u;  // R = 0: q - hi = +0
    if (R != 0) {
        unsigned A = (unsigned)(R < 0 ? -R : R);
        const unsigned ls = (R < 0) ? (sgn ^ 0x80000000u) : sgn;
#ifdef __CUDA_ARCH__
        int P = 31 - __clz(A);
#else
        int P = 31 - __builtin_clz(A);
#endif
        unsigned k2;
        if (P > 23) {
            const int sh = P - 23;
            const unsigned d2 = A & ((1u << sh) - 1u), half = 1u << (sh - 1);
            k2 = A >> sh;
            k2 += (d2 > half || (d2 == half && (k2 & 1u))) ? 1u : 0u;
            if (k2 == (1u << 24)) {
                k2 = 1u << 23;
                P += 1;
            }
        } else {
            k2 = A << (23 - P);
        }
        lb = ls | ((unsigned)(e - 52 + P + 127) << 23) | (k2 & 0x7fffffu);
    }
#ifdef __CUDA_ARCH__
    hi = __uint_as_float(hb);
    lo = __uint_as_float(lb);
#else
    memcpy(&hi, &hb, 4);
    memcpy(&lo, &lb, 4);
#endif
}

HK_HD long long cidx(const Geo &g, int i, int j, int k)
{
    return ((long long)(k + 1) * g.cy + (j + 1)) * g.cx + (i + 1);
}

// Reconstruction storage per cell, in the working precision: for each of
// the 5 variables the cell average Q_c (slot 0) and the 9 coefficients of
// P~ - Q_c (slots 1..9).  The per-face arrays of the characteristic
// variables and the mapped mesh's arrays keep one array per slot (term
// stride = the number of faces or cells); the uniform mesh keeps one record
// per cell (Rec below).
constexpr int NCOEF = 50;
HK_HD int coef_slot(int v, int n) { return v * 10 + n; }

// One record per cell of the uniform mesh: variable v's 10 values at
// v * VS .. v * VS + 9, every variable on a 16-byte boundary (FP32: 12
// floats with 2 unused, loaded as 3 float4; FP64: 10 doubles, 5 double2),
// so that the face flux reads a cell with a few vector loads at constant
// offsets.
template <typename R> struct Rec {
    static constexpr int VS = sizeof(R) == 4 ? 12 : 10;
    static constexpr int N = 5 * VS;
};
template <typename R> HK_HD long long rec_idx(long long cell, int v, int n)
{
    return cell * Rec<R>::N + v * Rec<R>::VS + n;
}

// One record per cell of a mapped mesh: the cell frame (centroid (3), 1/h,
// the cell means of the quadratic monomials in the scaled frame (6)) at
// 0 .. 9, then variable v's 10 values (Q_c, the 9 coefficients of P~ - Q_c)
// at VS (1 + v) .. VS (1 + v) + 9; every part on a 16-byte boundary (FP32:
// 12 floats with 2 unused; FP64: 10 doubles), so that the face flux reads a
// cell with vector loads at constant offsets.
template <typename R> struct MRec {
    static constexpr int VS = sizeof(R) == 4 ? 12 : 10;
    static constexpr int N = 6 * VS;
};
template <typename R> HK_HD long long mrec_idx(long long cell, int v, int n)
{
    return cell * MRec<R>::N + MRec<R>::VS * (1 + v) + n;
}

// Per-handle device control block: time, step and status.
struct Ctl {
    double t, dt;
    unsigned long long minbits;  // CFL reduction accumulator (bits of a positive double)
    int active;                  // 1 while the current step has dt > 0
    int status;                  // bit 0: nonphysical state produced
    int steps_done;
    int flagged;                 // cells that took the positivity fallback (last stage)
    unsigned nmarked;            // cells the reconstruction left to the literal positivity check
    double mapS, mapC;           // mapped mesh: sin(omega t), cos(omega t) at the stage time
                                 // (S = 1, C = 0 on a static mesh), set by the geometry kernel
    float mapAS, mapAUC;         // amp S and amp omega C in FP32 (mixed path)
};

// ---------------------------------------------------------------------------
// Maxwellian moments (Sec. 3).  For g = rho (lam/pi)^{(K+3)/2}
// exp(-lam(|u-U|^2 + xi^2)) the normalised moments factorise,
// <u^a v^b w^c xi^2d> = <u^a><v^b><w^c><xi^2d>, and each 1D moment obeys
// <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n>, on the whole line and on
// either half line (the boundary term vanishes for n >= 1 at u = 0).
// ---------------------------------------------------------------------------
template <typename R>
HK_HD void mom_full_1d(R U, R th, R *m)
{
    m[0] = R(1);
    m[1] = U;
#pragma unroll
    for (int n = 2; n < 7; ++n) m[n] = U * m[n - 1] + R(n - 1) * th * m[n - 2];
}

// 1/(n! (2n + 1)), the magnitude of the n-th coefficient of the Maclaurin
// series erf(x) = (2/sqrt(pi)) sum_n (-1)^n x^(2n+1)/(n! (2n+1)) (exact in
// double for the n used: n! (2n+1) < 2^53)
constexpr double erf_term(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return 1.0 / (f * (2 * n + 1));
}

// erfc(x) of the half-space moments.  For |x| < 3/4 from the Maclaurin
// series of erf summed by Horner in x^2 (FP64 15 terms, truncation below
// 4e-18; FP32 9 terms, below 7e-10; erfc >= 0.28 there, so 1 - erf loses
// nothing); the argument sqrt(lam) U is about the Mach number of the
// interface state, so smooth low-speed flows stay on this branch.
// Otherwise the library's erfc.  The branch is chosen per point, from x
// alone (a warp whose points straddle |x| = 3/4 runs both): the two sides
// of a face with the same argument, such as a reflecting wall's, then get
// the same value and their mass fluxes cancel exactly, and every result
// stays independent of which points share a warp.
template <typename R> HK_HD R erfc_half(R x)
{
    if (m_abs(x) < R(0.75)) {
        constexpr int N = sizeof(R) == 4 ? 9 : 15;
        const R y = x * x;
        R acc = R(((N - 1) & 1) ? -erf_term(N - 1) : erf_term(N - 1));
#pragma unroll
        for (int n = N - 2; n >= 0; --n) acc = acc * y + R((n & 1) ? -erf_term(n) : erf_term(n));
        return R(1) - R(1.12837916709551257390) * x * acc;
    }
    return m_erfc(x);
}

// half line u > 0 (side = +1) or u < 0 (side = -1):
// <1> = erfc(-side sqrt(lam) U)/2, <u> = U <1> + side exp(-lam U^2)/(2 sqrt(pi lam))
template <typename R>
HK_HD void mom_half_1d(R U, R lam, R th, R side, R *m)
{
    const R inv_sqrt_pi = R(0.56418958354775628695);
    const R isl = m_rsqrt(lam);
    m[0] = R(0.5) * erfc_half(-side * (lam * isl) * U);
    m[1] = U * m[0] + side * R(0.5) * inv_sqrt_pi * m_exp(-lam * U * U) * isl;
#pragma unroll
    for (int n = 2; n < 7; ++n) m[n] = U * m[n - 1] + R(n - 1) * th * m[n - 2];
}

// ---------------------------------------------------------------------------
// Moments in the frame moving with a Maxwellian's tangential velocity.
// With v' = v - V and w' = w - W the tangential velocities are central
// Gaussians (odd moments vanish, <v'^2> = <w'^2> = th = 1/(2 lam)), and
// psi = T psi' for psi' = (1, u, v', w', E'), E' = (u^2 + r)/2,
// r = v'^2 + w'^2 + xi^2, with
//   T x' = (x'0, x'1, x'2 + V x'0, x'3 + W x'0,
//           x'4 + V x'2 + W x'3 + (V^2 + W^2)/2 x'0).
// A slope a (a . psi) becomes a' = T^T a, found directly from the
// transformed moment data b' = T^{-1} b.  Moments in u stay as they are
// (whole or half line), m[n] = <u^n>, n = 0..6.
// ---------------------------------------------------------------------------
template <typename R> struct BMom {
    R m[7];
    R th;  // <v'^2> = <w'^2>
    R r1;  // <r>      = (K + 2) th
    R r2;  // <r^2>    = (K + 2)(K + 4) th^2
    R vr;  // <v'^2 r> = (K + 4) th^2
};

template <typename R> HK_HD void bmom_tangential(BMom<R> &B, R th, R K)
{
    B.th = th;
    B.r1 = (K + R(2)) * th;
    B.vr = (K + R(4)) * th * th;
    B.r2 = (K + R(2)) * B.vr;
}

// x = T x' (in place)
template <typename R> HK_HD void boost_out(R V, R W, R x[5])
{
    // x4 + V x2 + W x3 + (V^2 + W^2)/2 x0 as a chain of multiply-adds
    const R k = R(0.5) * (V * V + W * W);
    R e = x[4];
    e += V * x[2];
    e += W * x[3];
    e += k * x[0];
    x[4] = e;
    x[2] += V * x[0];
    x[3] += W * x[0];
}

// b' = T^{-1} b (in place)
template <typename R> HK_HD void boost_in(R V, R W, R b[5])
{
    b[2] -= V * b[0];
    b[3] -= W * b[0];
    // b4 - V b2' - W b3' - (V^2 + W^2)/2 b0 as a chain of multiply-adds
    R e = b[4];
    e -= V * b[2];
    e -= W * b[3];
    e -= (R(0.5) * (V * V + W * W)) * b[0];
    b[4] = e;
}

// The moment combinations below depend only on the Maxwellian and on n, so
// the compiler shares them between the calls for one Maxwellian; what is
// left per call is a few multiply-adds with the slope c.
//   E0 = <u^n E'>, E1 = <u^{n+1} E'>, E2 = <u^n E'^2>, Q = <u^n v'^2 E'>.
template <int N, typename R> HK_HD R bm_E0(const BMom<R> &B) { return R(0.5) * (B.m[N + 2] + B.r1 * B.m[N]); }
template <int N, typename R> HK_HD R bm_E2(const BMom<R> &B)
{
    return R(0.25) * (B.m[N + 4] + R(2) * B.r1 * B.m[N + 2] + B.r2 * B.m[N]);
}
template <int N, typename R> HK_HD R bm_Q(const BMom<R> &B) { return R(0.5) * (B.th * B.m[N + 2] + B.vr * B.m[N]); }

// <u^n psi'>
template <int N, typename R> HK_HD void bpsi(const BMom<R> &B, R o[5])
{
    o[0] = B.m[N];
    o[1] = B.m[N + 1];
    o[2] = o[3] = R(0);
    o[4] = bm_E0<N>(B);
}

// <u^n (c . psi') psi'>
template <int N, typename R> HK_HD void bapsi(const BMom<R> &B, const R c[5], R o[5])
{
    const R *m = B.m;
    const R E0 = bm_E0<N>(B), E1 = bm_E0<N + 1>(B), E2 = bm_E2<N>(B);
    const R tm = B.th * m[N];
    R e = c[0] * m[N];
    e += c[1] * m[N + 1];
    e += c[4] * E0;
    o[0] = e;
    e = c[0] * m[N + 1];
    e += c[1] * m[N + 2];
    e += c[4] * E1;
    o[1] = e;
    o[2] = c[2] * tm;
    o[3] = c[3] * tm;
    e = c[0] * E0;
    e += c[1] * E1;
    e += c[4] * E2;
    o[4] = e;
}

// <u^n v' (c1 . psi') psi'> + <u^n w' (c2 . psi') psi'>: the tangential
// terms of two slopes, which share their moment factors (v' and w' are
// central, <v'^2> = <w'^2> = th, so only c1's v'-component and c2's
// w'-component reach the mass and u-momentum, and the energy through Q)
template <int N, typename R> HK_HD void bapsi_tt(const BMom<R> &B, const R c1[5], const R c2[5], R o[5])
{
    const R *m = B.m;
    const R ct = c1[2] + c2[3];
    const R tm0 = B.th * m[N], tm1 = B.th * m[N + 1], Q = bm_Q<N>(B);
    o[0] = ct * tm0;
    o[1] = ct * tm1;
    R d = c1[0] * tm0;
    d += c1[1] * tm1;
    d += c1[4] * Q;
    o[2] = d;
    d = c2[0] * tm0;
    d += c2[1] * tm1;
    d += c2[4] * Q;
    o[3] = d;
    o[4] = ct * Q;
}

template <typename R> struct Prim {
    R rho, U, V, W, lam, p;
    R ir;  // 1/rho
    R th;  // 1/(2 lam)
    R q2;  // U^2 + (K+3)/(2 lam)
    R c4;  // 4 lam^2/(K+3)
    R H;   // (rho E + p)/rho
};

// iKp3 = 1/(K+3)
template <typename R> HK_HD Prim<R> primitive(const R Wc[5], R gamma, R Kp3, R iKp3)
{
    Prim<R> s;
    s.rho = Wc[0];
    s.ir = R(1) / Wc[0];
    s.U = Wc[1] * s.ir;
    s.V = Wc[2] * s.ir;
    s.W = Wc[3] * s.ir;
    R m2 = Wc[1] * s.U;
    m2 += Wc[2] * s.V;
    m2 += Wc[3] * s.W;
    const R eint = Wc[4] - R(0.5) * m2;
    s.p = (gamma - R(1)) * eint;
    s.H = (Wc[4] + s.p) * s.ir;
    // rho E = rho |U|^2/2 + (K+3) rho/(4 lam)
    s.lam = Kp3 * Wc[0] / (R(4) * eint);
    s.th = R(2) * iKp3 * eint * s.ir;
    s.q2 = s.U * s.U + Kp3 * s.th;
    s.c4 = R(4) * s.lam * s.lam * iKp3;
    return s;
}

// Solve <(a . psi') psi'> = sc b for a Maxwellian with velocity (U, 0, 0)
// and lam (the closed form in peculiar velocity, tangential velocities zero).
// The solution is linear in the data, so the scale sc (1/rho, and the
// gradient units) multiplies the Maxwellian's constants, which the calls
// with one scale share, instead of the five data values of every call.
template <typename R> HK_HD void micro_slope_u(const Prim<R> &s, const R b[5], R sc, R a[5])
{
    const R r1 = b[1] - s.U * b[0];
    // a4 = c4 (2 b4 - q2 b0 - 2 U r1) sc
    R e = (R(2) * s.c4 * sc) * b[4];
    e -= (s.c4 * s.q2 * sc) * b[0];
    e -= (R(2) * s.c4 * s.U * sc) * r1;
    a[4] = e;
    const R kl = R(2) * s.lam * sc;
    a[1] = kl * r1 - s.U * a[4];
    a[2] = kl * b[2];
    a[3] = kl * b[3];
    e = sc * b[0] - s.U * a[1];
    e -= (R(0.5) * s.q2) * a[4];
    a[0] = e;
}

// out += dF_i, the derivative of the Euler flux in direction i for the
// derivative d of the conservative variables.  For a Maxwellian g_W and the
// slope a with (a . psi) g = dg/dx_i this equals <u_i (a . psi) psi g>, the
// moment the compatibility condition needs, in closed form.  With
// delta_j = d(rho u_j) - u_j d rho = rho du_j:
//   d(rho u_j u_i) = d(rho u_i) u_j + u_i delta_j,
//   d(u_i (rho E + p)) = delta_i H + u_i (d(rho E) + dp),  H = (rho E + p)/rho.
template <int I, typename R> HK_HD void euler_dflux(const Prim<R> &s, R gm1, const R d[5], R out[5])
{
    const R u[3] = {s.U, s.V, s.W};
    R dl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) dl[j] = d[1 + j] - u[j] * d[0];
    // dp = (gamma - 1)(d4 + |u|^2/2 d0 - u . d), as a chain of multiply-adds
    R e = d[4];
    e += (R(0.5) * (s.U * s.U + s.V * s.V + s.W * s.W)) * d[0];
    e -= s.U * d[1];
    e -= s.V * d[2];
    e -= s.W * d[3];
    const R dp = gm1 * e;
    out[0] += d[1 + I];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        R o = out[1 + j];
        o += d[1 + I] * u[j];
        o += u[I] * dl[j];
        out[1 + j] = o;
    }
    out[1 + I] += dp;
    R o4 = out[4];
    o4 += dl[I] * s.H;
    o4 += u[I] * (d[4] + dp);
    out[4] = o4;
}

// ---------------------------------------------------------------------------
// Gas-kinetic flux at one Gauss point (Sec. 3), local frame (n_x, n_y, n_z),
// n_x from the left to the right cell.  Reading: g_l carries u > 0 and g_r
// u < 0 in eq. (flux), as in the half-space split of Q0.  Returns the flux
// per unit area F^n and its time derivative, found from the time integrals
// over dt and dt/2 (eq. expansion-1) in closed form.
//
// Every velocity moment of a Maxwellian is taken in the frame moving with
// its tangential velocity (BMom), and the compatibility condition's
// right-hand sides sum_i <u_i (a_i . psi) psi> are the Euler flux
// derivatives (euler_dflux); both are exact rewritings of the moments.
// ---------------------------------------------------------------------------
// gs: the physical gradient is gs times dWl, dWr (1 for physical
// gradients; 1/h for derivatives in the scaled frame of a cube of edge h).
template <typename R>
HK_HD void gks_flux(const R Wl[5], const R dWl[3][5], const R Wr[5], const R dWr[3][5],
                                         const Scheme &S, R dt, R F[5], R dF[5], R gs = R(1))
{
    const FluxK<R> C = fluxk<R>(S);
    const R gamma = C.gamma, K = C.K, Kp3 = C.Kp3, gm1 = C.gm1, iKp3 = C.iKp3;
    const bool prfix = S.prfix != 0;

    R W0[5], dW0[3][5], Fa[5], Fb[5], Fc[5], Sa[5], Sb[5], Sc[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        W0[k] = Fa[k] = Fb[k] = Fc[k] = Sb[k] = Sc[k] = R(0);
        dW0[0][k] = dW0[1][k] = dW0[2][k] = R(0);
    }
    R pside[2];

#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const R *Wc = side ? Wr : Wl;
        const R(*dW)[5] = side ? dWr : dWl;
        const Prim<R> s = primitive(Wc, gamma, Kp3, iKp3);
        pside[side] = s.p;
        // slope data per unit density: b_i = gs dW_i / rho, and for the time
        // slope b_A = -(gs/rho) sum_i dF_i(dW_i); the scales go to the solves
        const R irg = s.ir * gs;
        R bA[5] = {R(0), R(0), R(0), R(0), R(0)};
        euler_dflux<0>(s, gm1, dW[0], bA);
        euler_dflux<1>(s, gm1, dW[1], bA);
        euler_dflux<2>(s, gm1, dW[2], bA);
        // spatial and time slopes in the tangentially moving frame
        R a[3][5], A[5];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R b[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) b[k] = dW[i][k];
            boost_in(s.V, s.W, b);
            micro_slope_u(s, b, irg, a[i]);
        }
        boost_in(s.V, s.W, bA);
        micro_slope_u(s, bA, -irg, A);
        // u on the half line of this side
        BMom<R> B;
        mom_half_1d(s.U, s.lam, s.th, side ? R(-1) : R(1), B.m);
        bmom_tangential(B, s.th, K);
        R t[5];
        bpsi<0>(B, t);
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) W0[k] += s.rho * t[k];
        R d1[5], d2[5];  // <(a_1 . psi') psi'>, <(a_2 . psi') psi'> (also used by Sb)
        bapsi<0>(B, a[1], d1);
        bapsi<0>(B, a[2], d2);
        bapsi<0>(B, a[0], t);
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            dW0[0][k] += s.rho * t[k];
            t[k] = d1[k];
        }
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            dW0[1][k] += s.rho * t[k];
            t[k] = d2[k];
        }
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) dW0[2][k] += s.rho * t[k];
        bpsi<1>(B, t);
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) Fa[k] += s.rho * t[k];
        {
            // <u (u a_0 + v a_1 + w a_2) . psi psi> with v = V + v', w = W + w';
            // the V and W parts as one slope V a_1 + W a_2 (bapsi is linear in it)
            R cvw[5], t0[5], t1[5], tt[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) cvw[k] = s.V * a[1][k] + s.W * a[2][k];
            bapsi<2>(B, a[0], t0);
            bapsi<1>(B, cvw, t1);
            bapsi_tt<1>(B, a[1], a[2], tt);
#pragma unroll
            for (int k = 0; k < 5; ++k) t[k] = t0[k] + t1[k] + tt[k];
            boost_out(s.V, s.W, t);
#pragma unroll
            for (int k = 0; k < 5; ++k) Fb[k] += s.rho * t[k];
        }
        bapsi<1>(B, A, t);
        boost_out(s.V, s.W, t);
#pragma unroll
        for (int k = 0; k < 5; ++k) Fc[k] += s.rho * t[k];
        if (prfix) {
            // sum_i <u_i (a_i . psi) psi> and <(A . psi) psi> on this half line
            R t0[5], tt[5];
            bapsi<1>(B, a[0], t0);
            bapsi_tt<0>(B, a[1], a[2], tt);
#pragma unroll
            for (int k = 0; k < 5; ++k) t[k] = t0[k] + s.V * d1[k] + s.W * d2[k] + tt[k];
            boost_out(s.V, s.W, t);
#pragma unroll
            for (int k = 0; k < 5; ++k) Sb[k] += s.rho * t[k];
            bapsi<0>(B, A, t);
            boost_out(s.V, s.W, t);
#pragma unroll
            for (int k = 0; k < 5; ++k) Sc[k] += s.rho * t[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) Sa[k] = W0[k];

    // equilibrium state at the interface and its slopes
    const Prim<R> s0 = primitive(W0, gamma, Kp3, iKp3);
    const R ir0 = s0.ir;
    // S0b = sum_i <u_i (abar_i . psi) psi g0> (density rho0 included)
    R abar[3][5], Abar[5], S0b[5] = {R(0), R(0), R(0), R(0), R(0)};
    euler_dflux<0>(s0, gm1, dW0[0], S0b);
    euler_dflux<1>(s0, gm1, dW0[1], S0b);
    euler_dflux<2>(s0, gm1, dW0[2], S0b);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) b[k] = dW0[i][k];
        boost_in(s0.V, s0.W, b);
        micro_slope_u(s0, b, ir0, abar[i]);
    }
    {
        R b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) b[k] = S0b[k];
        boost_in(s0.V, s0.W, b);
        micro_slope_u(s0, b, -ir0, Abar);
    }
    BMom<R> B0;
    {
        mom_full_1d(s0.U, s0.th, B0.m);
        bmom_tangential(B0, s0.th, K);
    }
    R F0a[5], F0b[5], F0c[5];
    bpsi<1>(B0, F0a);
    boost_out(s0.V, s0.W, F0a);
    {
        R cvw[5], t0[5], t1[5], tt[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) cvw[k] = s0.V * abar[1][k] + s0.W * abar[2][k];
        bapsi<2>(B0, abar[0], t0);
        bapsi<1>(B0, cvw, t1);
        bapsi_tt<1>(B0, abar[1], abar[2], tt);
#pragma unroll
        for (int k = 0; k < 5; ++k) F0b[k] = t0[k] + t1[k] + tt[k];
        boost_out(s0.V, s0.W, F0b);
    }
    bapsi<1>(B0, Abar, F0c);
    boost_out(s0.V, s0.W, F0c);

    // collision time (Sec. 4)
    R jump = m_abs((pside[0] - pside[1]) / (pside[0] + pside[1]));
    R tau;
    if (S.viscous) {
        // mu/p0 with p0 = rho0/(2 lam0); with the viscosity law, mu at the
        // temperature T0 = p0/rho0 = 1/(2 lam0) of g0
        R mu2 = C.mu2;
        if (S.mu_pow != 0.0) mu2 *= pow_pos(s0.th * C.iT_ref, C.mu_pow);
        tau = mu2 * s0.lam * s0.ir + C.tau_C * jump * dt;
    }
    else
        tau = (C.tau_eps + C.tau_C * jump) * dt;

    // F = (4 Fh(dt/2) - Fh(dt))/dt and dF = 4 (Fh(dt) - 2 Fh(dt/2))/dt^2 for
    // Fh(delta) = sum_j q_j(delta) M_j, with q_j the time integrals of the
    // factors of eq. (flux); the combinations c_j, d_j below are those
    // integrals worked out with e2 = exp(-dt/(2 tau)), e1 = e2^2.
    const R idt = R(1) / dt;
    R x = R(0.5) * dt / tau;
    // om = 1 - e2; once exp(-x) is below half an ulp of 1 (x > 40 in FP64,
    // 20 in FP32; the viscous collision times of the workloads give x near
    // 100) the limits om = 1, e2 = 0 are the rounded values
    R om, e2;
    if (x > R(sizeof(R) == 4 ? 20 : 40)) {
        om = R(1);
        e2 = R(0);
    } else {
        om = -m_expm1(-x);
        e2 = R(1) - om;
    }
    R e1 = e2 * e2;
    R r = tau * idt;
    R E3 = om * (R(3) - e2);
    R Dq = om * om;
    R c3 = r * E3, c0 = R(1) - c3, c2 = -tau * c0, c5 = -tau * c3;
    R c1 = tau * (e1 - R(2) * e2 - R(1)) + R(2) * tau * r * E3;
    R c4 = -tau - c1;
    R d0 = R(4) * r * Dq * idt, d3 = -d0, d2 = R(1) - tau * d0, d5 = tau * d0;
    R d1 = R(4) * r * (e2 - e1) - R(8) * r * r * Dq, d4 = -d1;

    const R rc0 = s0.rho * c0, rc1 = s0.rho * c1, rc2 = s0.rho * c2;
    const R rd0 = s0.rho * d0, rd1 = s0.rho * d1, rd2 = s0.rho * d2;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        R e = rc0 * F0a[k];
        e += rc1 * F0b[k];
        e += rc2 * F0c[k];
        e += c3 * Fa[k];
        e += c4 * Fb[k];
        e += c5 * Fc[k];
        F[k] = e;
        e = rd0 * F0a[k];
        e += rd1 * F0b[k];
        e += rd2 * F0c[k];
        e += d3 * Fa[k];
        e += d4 * Fb[k];
        e += d5 * Fc[k];
        dF[k] = e;
    }
    if (prfix) {
        // heat flux about U0 of the time-integrated distribution:
        // q = F_E - U0.F_m + |U0|^2/2 F_rho - U0_x (S_E - U0.S_m + |U0|^2/2 S_rho),
        // S the psi-moments of the same terms (S of the g0 A-term is -S0b).
        R uu = R(0.5) * (s0.U * s0.U + s0.V * s0.V + s0.W * s0.W);
        R Sx[5], Sd[5];
        // S0b carries the density rho0 already
        const R c03 = c0 + c3, c12 = c1 - c2, d03 = d0 + d3, d12 = d1 - d2;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            R e = c03 * Sa[k];
            e += c12 * S0b[k];
            e += c4 * Sb[k];
            e += c5 * Sc[k];
            Sx[k] = e;
            e = d03 * Sa[k];
            e += d12 * S0b[k];
            e += d4 * Sb[k];
            e += d5 * Sc[k];
            Sd[k] = e;
        }
        // the g0 and initial terms both carry W0-like psi moments: the g0
        // term's zeroth piece is W0 itself and the half-space pieces sum to W0
        R qf = F[4] - (s0.U * F[1] + s0.V * F[2] + s0.W * F[3]) + uu * F[0]
               - s0.U * (Sx[4] - (s0.U * Sx[1] + s0.V * Sx[2] + s0.W * Sx[3]) + uu * Sx[0]);
        R qd = dF[4] - (s0.U * dF[1] + s0.V * dF[2] + s0.W * dF[3]) + uu * dF[0]
               - s0.U * (Sd[4] - (s0.U * Sd[1] + s0.V * Sd[2] + s0.W * Sd[3]) + uu * Sd[0]);
        const R fac = C.prfac;
        F[4] += fac * qf;
        dF[4] += fac * qd;
    }
}

// ---------------------------------------------------------------------------
// WENO-AO reconstruction on a uniform mesh of cubes (Sec. 2).
//
// In scaled coordinates X = (x - x_c)/h the row of the big-stencil least
// squares for neighbour offset (i, j, k) is [i, j, k, i^2, j^2, k^2, ij, ik,
// jk]; over the 18 cells of S the normal matrix is diag(10 I_3,
// 6 I_3 + 4 11^T, 4 I_3), so P0 has the closed form
//   a_d  = (1/10) sum o_d dQ,   a_de = (1/4) sum o_d o_e dQ,
//   a_dd = (1/6)(s_dd - (2/9)(s_xx + s_yy + s_zz)),  s_dd = sum o_d^2 dQ.
// A sub-stencil {c, s_a e_a, s_b e_b, s_a e_a + s_b e_b, s_c e_c} gives
//   b_a = s_a (2 dQ_a - dQ_b + dQ_ab)/3, b_b = s_b (2 dQ_b - dQ_a + dQ_ab)/3,
//   b_c = s_c dQ_c.
// Smoothness indicators (eq. indicator, each multi-index once):
//   beta_m = |b|^2,
//   beta_0 = sum_d [a_d^2 + (4 a_dd^2 + sum_{e != d} a_de^2)/12]
//            + 4 sum_d a_dd^2 + sum_{d<e} a_de^2.
// ---------------------------------------------------------------------------
template <typename R> struct Stencil {
    // dQ of the 18 neighbours: face neighbours f[d][0/1] (-/+), edge
    // neighbours e[plane][sa][sb] for planes (x,y), (y,z), (z,x)
    R f[3][2];
    R e[3][2][2];
    R f2[3][2];  // S' only: the axis cells two steps away (-/+)
};

template <typename R> HK_HD void big_stencil_P0(const Stencil<R> &st, R a[9])
{
    // linear: sum over offsets of o_d dQ; face cells and the 8 edge cells with o_d != 0
    R sd[3], sdd[3], sde[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // edges in plane (d, d+1) and plane (d-1, d) (= plane index (d+2)%3 with d second)
        int p1 = d, p2 = (d + 2) % 3;
        R lin = st.f[d][1] - st.f[d][0];
        R quad = st.f[d][1] + st.f[d][0];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            // plane p1: d is the first axis
            lin += st.e[p1][1][s] - st.e[p1][0][s];
            quad += st.e[p1][1][s] + st.e[p1][0][s];
            // plane p2: d is the second axis
            lin += st.e[p2][s][1] - st.e[p2][s][0];
            quad += st.e[p2][s][1] + st.e[p2][s][0];
        }
        sd[d] = lin;
        sdd[d] = quad;
        // cross moment sum o_a o_b dQ over the plane (a, b) = (d, d+1)
        sde[d] = st.e[d][1][1] + st.e[d][0][0] - st.e[d][1][0] - st.e[d][0][1];
    }
    const R tr = sdd[0] + sdd[1] + sdd[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        a[d] = R(0.1) * sd[d];
        a[3 + d] = (sdd[d] - R(2.0 / 9.0) * tr) * R(1.0 / 6.0);
    }
    // xy = plane 0, xz = plane 2 (z,x) -> same product, yz = plane 1
    a[6] = R(0.25) * sde[0];
    a[7] = R(0.25) * sde[2];
    a[8] = R(0.25) * sde[1];
}

template <typename R> HK_HD R beta_quadratic(const R a[9])
{
    const R ax = a[0], ay = a[1], az = a[2], axx = a[3], ayy = a[4], azz = a[5], axy = a[6], axz = a[7], ayz = a[8];
    const R d2 = R(4) * (axx * axx + ayy * ayy + azz * azz);
    const R m2 = axy * axy + axz * axz + ayz * ayz;
    return ax * ax + ay * ay + az * az + (d2 + R(2) * m2) * R(1.0 / 12.0) + d2 + m2;
}

// sub-stencil m = 8 p + s: plane (a, b) = (p, p+1), out-of-plane c = p+2,
// signs in the order (+++), (-++), (+-+), (--+), (++-), (-+-), (+--), (---)
// (every index is a compile-time constant: the stencil stays in registers)
template <int M, typename R> HK_HD void sub_stencil(const Stencil<R> &st, R b[3])
{
    constexpr int p = M >> 3, s = M & 7;
    constexpr int sa = (s & 1) ? 0 : 1, sb = (s & 2) ? 0 : 1, sc = (s & 4) ? 0 : 1;
    constexpr int a = p, bb = (p + 1) % 3, c = (p + 2) % 3;
    const R qa = st.f[a][sa], qb = st.f[bb][sb], qab = st.e[p][sa][sb], qc = st.f[c][sc];
    const R ba = (R(2) * qa - qb + qab) * R(1.0 / 3.0);
    const R bbv = (R(2) * qb - qa + qab) * R(1.0 / 3.0);
    b[a] = sa ? ba : -ba;
    b[bb] = sb ? bbv : -bbv;
    b[c] = sc ? qc : -qc;
}

// expands X(m) for the 24 sub-stencils m = 0..23
#define HK_FOR_SUBSTENCILS(X)                                                                             \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) \
        X(19) X(20) X(21) X(22) X(23)

// sub-stencil m chosen at run time (for the rare literal positivity check)
template <typename R> HK_HD void sub_stencil_rt(const Stencil<R> &st, int m, R b[3])
{
    switch (m) {
#define HK_CASE(M)                \
    case M:                       \
        sub_stencil<M>(st, b);    \
        break;
        HK_FOR_SUBSTENCILS(HK_CASE)
#undef HK_CASE
    default:
        b[0] = b[1] = b[2] = R(0);
    }
}

// rigorous bound of |P(X) - Q_c| over the cell (|X_d| <= 1/2)
template <typename R> HK_HD R bound_linear(const R b[3])
{
    return R(0.5) * (m_abs(b[0]) + m_abs(b[1]) + m_abs(b[2]));
}
// the same for every linear P_m at once, at the cell's 24 face Gauss points
// (where the positivity check looks), from the largest indicator
// beta_m = |b|^2: |b . X| <= |b| |X| and every Gauss point has |X|^2 =
// 1/4 + 2/12 = 5/12 (Cauchy-Schwarz)
template <typename R> HK_HD R bound_linear_gauss(R beta_max)
{
    return m_sqrt(R(5.0 / 12.0) * beta_max);
}
template <typename R> HK_HD R bound_quadratic(const R a[9])
{
    return R(0.5) * (m_abs(a[0]) + m_abs(a[1]) + m_abs(a[2]))
           + R(1.0 / 6.0) * (m_abs(a[3]) + m_abs(a[4]) + m_abs(a[5]))
           + R(0.25) * (m_abs(a[6]) + m_abs(a[7]) + m_abs(a[8]));
}

// value of Q_c + sum c_n p_n at scaled X (p = X, Y, Z, X^2-1/12, ..., XY, XZ, YZ)
template <typename R> HK_HD R poly9(const R c[9], const R X[3])
{
    const R tw = R(1.0 / 12.0);
    return c[0] * X[0] + c[1] * X[1] + c[2] * X[2] + c[3] * (X[0] * X[0] - tw) + c[4] * (X[1] * X[1] - tw)
           + c[5] * (X[2] * X[2] - tw) + c[6] * X[0] * X[1] + c[7] * X[0] * X[2] + c[8] * X[1] * X[2];
}


// P~ - Q_c and its physical gradient at scaled X (ih = 1/h)
template <typename R> HK_HD void poly_value_grad(const R c[9], const R X[3], R ih, R &s, R grad[3])
{
    s = poly9(c, X);
    grad[0] = (c[0] + R(2) * c[3] * X[0] + c[6] * X[1] + c[7] * X[2]) * ih;
    grad[1] = (c[1] + R(2) * c[4] * X[1] + c[6] * X[0] + c[8] * X[2]) * ih;
    grad[2] = (c[2] + R(2) * c[5] * X[2] + c[7] * X[0] + c[8] * X[1]) * ih;
}

// ---------------------------------------------------------------------------
// The alternative stencil S' (Remark of Sec. 2): S plus the six axis cells
// two steps away, and 8 sub-stencils {c, s_x e_x, s_y e_y, s_z e_z}, one per
// octant.  On cubes the normal matrix of P0 over S' is diag(18 I_3,
// 38 I_3 + 4 11^T, 4 I_3), so
//   a_d  = (1/18) sum o_d dQ,   a_de = (1/4) sum o_d o_e dQ,
//   a_dd = (s_dd - (2/25) sum_e s_ee)/38,   s_dd = sum o_d^2 dQ,
// and each octant sub-stencil is square: b_d = s_d dQ(s_d e_d).
// ---------------------------------------------------------------------------
template <typename R> HK_HD void big_stencil_P0_sp(const Stencil<R> &st, R a[9])
{
    R sd[3], sdd[3], sde[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int p1 = d, p2 = (d + 2) % 3;
        R lin = st.f[d][1] - st.f[d][0] + R(2) * (st.f2[d][1] - st.f2[d][0]);
        R quad = st.f[d][1] + st.f[d][0] + R(4) * (st.f2[d][1] + st.f2[d][0]);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            lin += st.e[p1][1][s] - st.e[p1][0][s];
            quad += st.e[p1][1][s] + st.e[p1][0][s];
            lin += st.e[p2][s][1] - st.e[p2][s][0];
            quad += st.e[p2][s][1] + st.e[p2][s][0];
        }
        sd[d] = lin;
        sdd[d] = quad;
        sde[d] = st.e[d][1][1] + st.e[d][0][0] - st.e[d][1][0] - st.e[d][0][1];
    }
    const R tr = sdd[0] + sdd[1] + sdd[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        a[d] = sd[d] * R(1.0 / 18.0);
        a[3 + d] = (sdd[d] - R(2.0 / 25.0) * tr) * R(1.0 / 38.0);
    }
    a[6] = R(0.25) * sde[0];
    a[7] = R(0.25) * sde[2];
    a[8] = R(0.25) * sde[1];
}

// octant sub-stencil M of S', signs in the printed order (+++), (-++), (+-+),
// (--+), (++-), (-+-), (+--), (---)
template <int M, typename R> HK_HD void sub_stencil_sp(const Stencil<R> &st, R b[3])
{
    constexpr int sx = (M & 1) ? 0 : 1, sy = (M & 2) ? 0 : 1, sz = (M & 4) ? 0 : 1;
    b[0] = sx ? st.f[0][1] : -st.f[0][0];
    b[1] = sy ? st.f[1][1] : -st.f[1][0];
    b[2] = sz ? st.f[2][1] : -st.f[2][0];
}

#define HK_FOR_SUBSTENCILS_SP(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7)

template <typename R> HK_HD void sub_stencil_sp_rt(const Stencil<R> &st, int m, R b[3])
{
    switch (m) {
#define HK_CASE_SP(M)                   \
    case M:                             \
        sub_stencil_sp<M, R>(st, b);    \
        break;
        HK_FOR_SUBSTENCILS_SP(HK_CASE_SP)
#undef HK_CASE_SP
    default:
        b[0] = b[1] = b[2] = R(0);
    }
}

// One-pass form of the WENO-AO combination (Sec. 2, eqs. (para) and
// (nonlinear)).  With x_m = 1/(beta_m + eps), y0 = 1/(beta0 + eps), the
// exponent p of tau/(beta + eps) and t = tau^p, the weights are
// w_m = g_m (1 + t x_m^p) and w_0 = g_0 (1 + t y0^p), so the coefficient of
// P_m in P~ = (w0/g0) P0 + sum (w_m - w0 g_m/g0) P_m (before normalising by
// the weight sum) is
//   g_m t (x_m^p - y0^p) = g_m t y0 (beta0 - beta_m) x_m k_m,
// k_m = 1 (p = 1) or x_m + y0 (p = 2), and the weight sum is
// w_0 + g_m (n + t sum x_m^p).  Both are linear in t, so a single pass over
// the n sub-stencils gathers every sum before tau is known; the difference
// beta0 - beta_m that tau needs also carries the coefficients, so no
// cancellation between nearly equal weights enters them.
template <typename R> struct AoSums {
    R y0, dsum, xs, T[3];
    bool pow2;
    HK_HD void init(R beta0, R eps, bool p2)
    {
        y0 = R(1) / (beta0 + eps);
        dsum = xs = T[0] = T[1] = T[2] = R(0);
        pow2 = p2;
    }
    // linear polynomial with coefficients b (indicator bm = |b|^2), given
    // x = 1/(bm + eps)
    HK_HD void add_x(R beta0, const R b[3], R bm, R x)
    {
        const R d = beta0 - bm;
        dsum += m_abs(d);
        xs += pow2 ? x * x : x;
        const R f = d * x * (pow2 ? x + y0 : R(1));
        T[0] += f * b[0];
        T[1] += f * b[1];
        T[2] += f * b[2];
    }
    HK_HD void add(R beta0, R eps, const R b[3])
    {
        const R bm = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        add_x(beta0, b, bm, R(1) / (bm + eps));
    }
    // P~ - Q_c = iw (f0 (P0 - Q_c) + lin . X) for NSUB sub-stencils with
    // linear weights g0 and gm each
    template <int NSUB> HK_HD void combine(R g0, R gm, R &iw, R &f0, R lin[3]) const
    {
        const R tau = dsum * R(1.0 / NSUB);
        const R t = pow2 ? tau * tau : tau;
        f0 = R(1) + t * (pow2 ? y0 * y0 : y0);
        iw = R(1) / (g0 * f0 + gm * (R(NSUB) + t * xs));
        const R cl = gm * t * y0;
        lin[0] = cl * T[0];
        lin[1] = cl * T[1];
        lin[2] = cl * T[2];
    }
};

// x_q = 1/d_q for four nonzero d_q.  In FP64, where a division costs
// several FP64-pipe operations, one division of the product and nine
// multiplications; in other precisions four divisions.
template <typename R> HK_HD void recip4(const R d[4], R x[4])
{
    if constexpr (sizeof(R) == 8) {
        const R p01 = d[0] * d[1], p23 = d[2] * d[3];
        const R r = R(1) / (p01 * p23);
        const R r01 = r * p23, r23 = r * p01;
        x[0] = r01 * d[1];
        x[1] = r01 * d[0];
        x[2] = r23 * d[3];
        x[3] = r23 * d[2];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = R(1) / d[q];
    }
}

// the sub-stencils in groups of four (m = 0..23 and the 8 of S')
#define HK_FOR_SUBSTENCIL_QUADS(X) X(0, 1, 2, 3) X(4, 5, 6, 7) X(8, 9, 10, 11) X(12, 13, 14, 15) \
    X(16, 17, 18, 19) X(20, 21, 22, 23)
#define HK_FOR_SUBSTENCIL_QUADS_SP(X) X(0, 1, 2, 3) X(4, 5, 6, 7)

// WENO-AO combination for one conserved variable (Sec. 2): P0, the 24
// linear P_m, their indicators, tau of eq. (para), the nonlinear weights of
// eq. (nonlinear) and P~ = (w0/g0) P0 + sum (w_m - w0 g_m/g0) P_m, returned
// as the 9 coefficients of one quadratic; rad receives a rigorous bound of
// |P_m(X) - Q_c| at the cell's 24 face Gauss points for all 25 polynomials.
template <typename R>
HK_HD void weno_ao(const Stencil<R> &st, const Scheme &S, R out[9], R &rad)
{
    const R g0 = R(1.0 - 24.0 * S.Gamma_lin), gm = R(S.Gamma_lin), eps = R(S.weno_eps);
    R a[9];
    big_stencil_P0(st, a);
    const R beta0 = beta_quadratic(a);
    R bmax = R(0);
    AoSums<R> acc;
    acc.init(beta0, eps, S.weno_pow == 2);
#define HK_PASS(M0, M1, M2, M3)                                                \
    {                                                                          \
        R b[4][3], bm[4], den[4], x[4];                                        \
        sub_stencil<M0>(st, b[0]);                                             \
        sub_stencil<M1>(st, b[1]);                                             \
        sub_stencil<M2>(st, b[2]);                                             \
        sub_stencil<M3>(st, b[3]);                                             \
        for (int q = 0; q < 4; ++q) {                                          \
            bm[q] = b[q][0] * b[q][0] + b[q][1] * b[q][1] + b[q][2] * b[q][2]; \
            den[q] = bm[q] + eps;                                              \
            bmax = m_max(bmax, bm[q]);                                         \
        }                                                                      \
        recip4(den, x);                                                        \
        for (int q = 0; q < 4; ++q) acc.add_x(beta0, b[q], bm[q], x[q]);      \
    }
    HK_FOR_SUBSTENCIL_QUADS(HK_PASS)
#undef HK_PASS
    rad = m_max(bound_quadratic(a), bound_linear_gauss(bmax));
    R iw, f0, lin[3];
    acc.template combine<24>(g0, gm, iw, f0, lin);
#pragma unroll
    for (int n = 0; n < 9; ++n) out[n] = iw * (f0 * a[n] + (n < 3 ? lin[n] : R(0)));
}

// WENO-AO with S' and its 8 sub-stencils: linear weights gamma_0 = 1 - 8
// Gamma, gamma_m = Gamma (reading), tau the mean of |beta_0 - beta_m| over
// the 8; otherwise as weno_ao
template <typename R>
HK_HD void weno_ao_sp(const Stencil<R> &st, const Scheme &S, R out[9], R &rad)
{
    const R g0 = R(1.0 - 8.0 * S.Gamma_lin), gm = R(S.Gamma_lin), eps = R(S.weno_eps);
    R a[9];
    big_stencil_P0_sp(st, a);
    const R beta0 = beta_quadratic(a);
    R bmax = R(0);
    AoSums<R> acc;
    acc.init(beta0, eps, S.weno_pow == 2);
#define HK_PASS_SP(M0, M1, M2, M3)                                             \
    {                                                                          \
        R b[4][3], bm[4], den[4], x[4];                                        \
        sub_stencil_sp<M0>(st, b[0]);                                          \
        sub_stencil_sp<M1>(st, b[1]);                                          \
        sub_stencil_sp<M2>(st, b[2]);                                          \
        sub_stencil_sp<M3>(st, b[3]);                                          \
        for (int q = 0; q < 4; ++q) {                                          \
            bm[q] = b[q][0] * b[q][0] + b[q][1] * b[q][1] + b[q][2] * b[q][2]; \
            den[q] = bm[q] + eps;                                              \
            bmax = m_max(bmax, bm[q]);                                         \
        }                                                                      \
        recip4(den, x);                                                        \
        for (int q = 0; q < 4; ++q) acc.add_x(beta0, b[q], bm[q], x[q]);      \
    }
    HK_FOR_SUBSTENCIL_QUADS_SP(HK_PASS_SP)
#undef HK_PASS_SP
    rad = m_max(bound_quadratic(a), bound_linear_gauss(bmax));
    R iw, f0, lin[3];
    acc.template combine<8>(g0, gm, iw, f0, lin);
#pragma unroll
    for (int n = 0; n < 9; ++n) out[n] = iw * (f0 * a[n] + (n < 3 ? lin[n] : R(0)));
}

// The sign test of the pressure p = (gamma - 1)(rho E - |rho U|^2/(2 rho))
// of a point state W, for rho >= 0 (a negative rho has failed already):
// p < 0 exactly when 2 rho (rho E) - |rho U|^2 < 0, since gamma > 1; no
// division.  (rho = 0 with rho U = 0 is not negative, as p is then NaN.)
template <typename R> HK_HD bool pressure_negative(const R W[5])
{
    R q = R(2) * W[0] * W[4];
    q -= W[1] * W[1];
    q -= W[2] * W[2];
    q -= W[3] * W[3];
    return q < R(0);
}

// Sufficient test that no P_m gives negative density or pressure at the
// cell's Gauss points, from the cell averages and the bounds rad[v]; when it fails the
// literal check of the fallback (Sec. 4) decides.
template <typename R> HK_HD bool positivity_certain(const R qc[5], const R rad[5], R gamma)
{
    const R rho_min = qc[0] - rad[0];
    if (!(rho_min > R(0))) return false;
    R m2 = R(0);
#pragma unroll
    for (int d = 1; d <= 3; ++d) {
        const R mm = m_abs(qc[d]) + rad[d];
        m2 += mm * mm;
    }
    const R e_min = qc[4] - rad[4];
    const R p_low = (gamma - R(1)) * (e_min - R(0.5) * m2 / rho_min);
    const R margin = R(sizeof(R) == 8 ? 1e-10 : 1e-4) * (m_abs(qc[4]) + rad[4] + R(0.5) * m2 / rho_min);
    return p_low > margin;
}

}  // namespace hk
