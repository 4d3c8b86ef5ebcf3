// Reconstruction in characteristic variables (Sec. 4) on a uniform mesh:
// for every face normal to axis D the characteristic variables are L Q,
// L = R^{-1}, R the right eigenvectors of the Euler flux Jacobian along e_D
// at the mean of the face's two cell averages (reading of "at the Gaussian
// quadrature point").  Each side of the face is reconstructed by WENO-AO
// field by field in those variables and mapped back with R; the face flux
// then reads per-(face, side) polynomials instead of per-cell ones.
#pragma once
#include "hgks_items.cuh"

namespace hk {

// layout of the per-axis coefficient array: [side][slot(v, n)][face], 50
// slots per side (Q_c and the 9 coefficients of each variable)
constexpr int CHAR_SLOTS = 50;
static_assert(CHAR_SLOTS == NCOEF, "one (face, side) holds the per-cell record");

// the eigenbasis along e_D at the conservative state W
template <typename R> struct CharBasis {
    R u[3], c, b1, b2, H, k;
};

template <typename R, int D> __device__ __forceinline__ CharBasis<R> char_basis(const double W[5], double gamma)
{
    const double rho = W[0], ir = 1.0 / rho;
    const double u[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double p = (gamma - 1.0) * (W[4] - rho * k);
    const double c2 = gamma * p * ir;
    CharBasis<R> B;
#pragma unroll
    for (int e = 0; e < 3; ++e) B.u[e] = R(u[e]);
    B.c = R(sqrt(c2));
    B.b1 = R((gamma - 1.0) / c2);
    B.b2 = R((gamma - 1.0) / c2 * k);
    B.H = R((W[4] + p) * ir);
    B.k = R(k);
    return B;
}

// row f of L = R^{-1}: acoustic (u_D - c), entropy, shear along e_A and e_B,
// acoustic (u_D + c)
template <typename R, int D> __device__ __forceinline__ void char_left_row(const CharBasis<R> &B, int f, R l[5])
{
    constexpr int A = (D + 1) % 3, Bx = (D + 2) % 3;
    const R ic = R(1) / B.c;
    switch (f) {
    case 0:
    case 4: {
        const R s = f == 0 ? R(1) : R(-1);
        l[0] = R(0.5) * (B.b2 + s * B.u[D] * ic);
#pragma unroll
        for (int e = 0; e < 3; ++e) l[1 + e] = R(-0.5) * (B.b1 * B.u[e] + (e == D ? s * ic : R(0)));
        l[4] = R(0.5) * B.b1;
        break;
    }
    case 1:
        l[0] = R(1) - B.b2;
#pragma unroll
        for (int e = 0; e < 3; ++e) l[1 + e] = B.b1 * B.u[e];
        l[4] = -B.b1;
        break;
    default: {
        const int t = f == 2 ? A : Bx;
        l[0] = -B.u[t];
#pragma unroll
        for (int e = 0; e < 3; ++e) l[1 + e] = e == t ? R(1) : R(0);
        l[4] = R(0);
    }
    }
}

// column f of R
template <typename R, int D> __device__ __forceinline__ void char_right_col(const CharBasis<R> &B, int f, R r[5])
{
    constexpr int A = (D + 1) % 3, Bx = (D + 2) % 3;
    switch (f) {
    case 0:
    case 4: {
        const R s = f == 0 ? R(-1) : R(1);
        r[0] = R(1);
#pragma unroll
        for (int e = 0; e < 3; ++e) r[1 + e] = B.u[e] + (e == D ? s * B.c : R(0));
        r[4] = B.H + s * B.c * B.u[D];
        break;
    }
    case 1:
        r[0] = R(1);
#pragma unroll
        for (int e = 0; e < 3; ++e) r[1 + e] = B.u[e];
        r[4] = B.k;
        break;
    default: {
        const int t = f == 2 ? A : Bx;
        r[0] = R(0);
#pragma unroll
        for (int e = 0; e < 3; ++e) r[1 + e] = e == t ? R(1) : R(0);
        r[4] = B.u[t];
    }
    }
}

// the projected differences l . (Q_nb - Q_c) of the 18 big-stencil
// neighbours of cell (i,j,k) (differences formed in FP64)
template <typename R>
__device__ __forceinline__ void load_stencil_proj(const double *__restrict__ Q, const Geo &g, int i, int j, int k,
                                                  const double qc[5], const R l[5], Stencil<R> &st)
{
    const long long sd[3] = {1, g.px, (long long)g.px * g.py};
    const long long c = pidx(g, i, j, k);
    auto proj = [&](long long at) {
        R s = R(0);
#pragma unroll
        for (int v = 0; v < 5; ++v) s += l[v] * R(Q[v * g.pstride + at] - qc[v]);
        return s;
    };
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.f[d][0] = proj(c - sd[d]);
        st.f[d][1] = proj(c + sd[d]);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const long long a = sd[p], b = sd[(p + 1) % 3];
#pragma unroll
        for (int sa = 0; sa < 2; ++sa)
#pragma unroll
            for (int sb = 0; sb < 2; ++sb) st.e[p][sa][sb] = proj(c + (sa ? a : -a) + (sb ? b : -b));
    }
}

// face index -> the reconstructed cell of this side and the face's two cells
template <int D>
__device__ __forceinline__ void char_face_cells(const Geo &g, long long face, int side, int cell[3], int lc[3],
                                                int rc[3])
{
    const int ex = g.nx + (D == 0), ey = g.ny + (D == 1);
    split3(face, ex, ey, rc[0], rc[1], rc[2]);
#pragma unroll
    for (int e = 0; e < 3; ++e) lc[e] = rc[e] - (e == D);
#pragma unroll
    for (int e = 0; e < 3; ++e) cell[e] = side ? rc[e] : lc[e];
}

template <typename R, int D>
__device__ __forceinline__ CharBasis<R> char_face_basis(const double *__restrict__ Q, const Geo &g, const int lc[3],
                                                        const int rc[3], double gamma)
{
    const long long pl = pidx(g, lc[0], lc[1], lc[2]), pr = pidx(g, rc[0], rc[1], rc[2]);
    double Wm[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Wm[v] = 0.5 * (Q[v * g.pstride + pl] + Q[v * g.pstride + pr]);
    return char_basis<R, D>(Wm, gamma);
}

// one (face, side) of axis D; t in [0, 2 nface): side = t / nface.  Writes
// Q_c and the 9 coefficients of each conservative variable, and the flag
// (0, or 2 when the positivity bound is inconclusive: literal check next)
template <typename R, int D>
__device__ __forceinline__ void recon_char_item(const double *__restrict__ Q, R *__restrict__ coefc,
                                                unsigned char *__restrict__ flagc, const Geo &g, const Scheme &S,
                                                long long t)
{
    const long long nface = face_count<D>(g);
    if (t >= 2 * nface) return;
    const int side = t >= nface;
    const long long face = side ? t - nface : t;
    int cell[3], lc[3], rc[3];
    char_face_cells<D>(g, face, side, cell, lc, rc);
    const CharBasis<R> B = char_face_basis<R, D>(Q, g, lc, rc, S.gamma);
    const long long pc = pidx(g, cell[0], cell[1], cell[2]);
    double qc[5];
    R qcv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        qc[v] = Q[v * g.pstride + pc];
        qcv[v] = R(qc[v]);
    }
    R cf[5][9], rad[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        rad[v] = R(0);
#pragma unroll
        for (int n = 0; n < 9; ++n) cf[v][n] = R(0);
    }
#pragma unroll 1
    for (int f = 0; f < 5; ++f) {
        R l[5], r[5];
        char_left_row<R, D>(B, f, l);
        Stencil<R> st;
        load_stencil_proj(Q, g, cell[0], cell[1], cell[2], qc, l, st);
        R out[9], radf;
        weno_ao(st, S, out, radf);
        char_right_col<R, D>(B, f, r);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
#pragma unroll
            for (int n = 0; n < 9; ++n) cf[v][n] += r[v] * out[n];
            rad[v] += m_abs(r[v]) * radf;
        }
    }
    R *base = coefc + (long long)side * CHAR_SLOTS * nface + face;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        base[coef_slot(v, 0) * nface] = qcv[v];
#pragma unroll
        for (int n = 0; n < 9; ++n) base[coef_slot(v, 1 + n) * nface] = cf[v][n];
        rad[v] *= R(1.0000001);
    }
    flagc[t] = (S.limiter && !positivity_certain(qcv, rad, fluxk<R>(S).gamma)) ? 2 : 0;
}

// literal positivity check (Sec. 4) of the items marked 2: all 25
// polynomials, built field by field in the face's characteristic variables
// and mapped back, at the cell's 24 face Gauss points; a violation sets
// the polynomial of this (face, side) to the cell average
template <typename R, int D>
__device__ __forceinline__ void positivity_char_item(const double *__restrict__ Q, R *__restrict__ coefc,
                                                     unsigned char *__restrict__ flagc, const Geo &g, const Scheme &S,
                                                     Ctl *ctl, long long t)
{
    const long long nface = face_count<D>(g);
    if (t >= 2 * nface || flagc[t] != 2) return;
    const int side = t >= nface;
    const long long face = side ? t - nface : t;
    int cell[3], lc[3], rc[3];
    char_face_cells<D>(g, face, side, cell, lc, rc);
    const CharBasis<R> B = char_face_basis<R, D>(Q, g, lc, rc, S.gamma);
    const long long pc = pidx(g, cell[0], cell[1], cell[2]);
    double qc[5];
    R qcv[5];
    for (int v = 0; v < 5; ++v) {
        qc[v] = Q[v * g.pstride + pc];
        qcv[v] = R(qc[v]);
    }
    const R gamma = fluxk<R>(S).gamma;
    bool bad = false;
    for (int m = 0; m <= 24 && !bad; ++m) {
        R cf[5][9];
        for (int v = 0; v < 5; ++v)
            for (int n = 0; n < 9; ++n) cf[v][n] = R(0);
        for (int f = 0; f < 5; ++f) {
            R l[5], r[5], p[9];
            char_left_row<R, D>(B, f, l);
            Stencil<R> st;
            load_stencil_proj(Q, g, cell[0], cell[1], cell[2], qc, l, st);
            if (m == 0) {
                big_stencil_P0(st, p);
            } else {
                R b[3];
                sub_stencil_rt(st, m - 1, b);
                for (int n = 0; n < 9; ++n) p[n] = n < 3 ? b[n] : R(0);
            }
            char_right_col<R, D>(B, f, r);
            for (int v = 0; v < 5; ++v)
                for (int n = 0; n < 9; ++n) cf[v][n] += r[v] * p[n];
        }
        for (int gq = 0; gq < 24 && !bad; ++gq) {
            const int d = gq / 8, sd = (gq / 4) & 1, ga = (gq >> 1) & 1, gb = gq & 1;
            R X[3];
            X[d] = sd ? R(0.5) : R(-0.5);
            X[(d + 1) % 3] = ga ? R(GAUSS_S) : R(-GAUSS_S);
            X[(d + 2) % 3] = gb ? R(GAUSS_S) : R(-GAUSS_S);
            R W[5];
            for (int v = 0; v < 5; ++v) W[v] = qcv[v] + poly9(cf[v], X);
            if (W[0] < R(0) || pressure_negative(W)) bad = true;
        }
    }
    if (bad) {
        R *base = coefc + (long long)side * CHAR_SLOTS * nface + face;
        for (int v = 0; v < 5; ++v)
            for (int n = 1; n < 10; ++n) base[coef_slot(v, n) * nface] = R(0);
        atomicAdd(&ctl->flagged, 1);
    }
    flagc[t] = bad ? 1 : 0;
}

}  // namespace hk
