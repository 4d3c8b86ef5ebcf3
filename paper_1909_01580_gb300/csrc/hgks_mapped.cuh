// Mapped and moving meshes of trilinear hexahedra (Sec. 2 trilinear cells,
// Sec. 3 bilinear faces, Remark 2 moving mesh): per-cell geometry, the
// WENO-AO reconstruction with per-cell least squares, and the face flux in
// the frame moving with the grid.  Per-item bodies for hgks_mapped.cu.
#pragma once
#include "hgks_items.cuh"

namespace hk {

// The mesh map: x_d = xi_d + amp S(t) prod_e sin(2 pi (xi_e - lo_e)/L_e)
// with S = 1 (static) or sin(omega t) (moving); xi on a uniform reference
// grid.  sx/sy/sz hold the sine factor at vertex indices -GHOST..n+GHOST
// (offset GHOST).
struct MapGeo {
    double lo[3], hi[3];
    int n[3];
    double h[3], ih[3];  // reference spacing (hi - lo)/n and its inverse
    double amp, omega;
    int moving;
    const double *sx, *sy, *sz;
    // FP32 copies for the mixed path's face geometry: lo, the reference
    // spacing (hi - lo)/n, and the sine factors
    float lof[3], hf[3], ihf[3];
    const float *sxf, *syf, *szf;
    // mixed path (null otherwise): an FP32 copy of the cells' central second
    // moments and of their centroid offsets from the reference centres,
    // [GEOF][pstride], written by the geometry kernel, and the split state
    // of the stage's Q (Q_hi + Q_lo in FP32, [2][5][pstride])
    float *geof;
    const float *qsplit;
};

// per-cell geometry record (FP64, over the padded cell box): volume,
// centroid, central second moments (xx, yy, zz, xy, xz, yz)
constexpr int NGEO = 10;
// FP32 copy of the mixed path: the six central moments, then the centroid
// minus the reference centre lo + (idx + 1/2) h (3)
constexpr int GEOF = 9;

// one 16-byte-aligned part of a mapped record (the frame, or one
// variable: MRec<R>::VS values) by vector loads and stores
__device__ __forceinline__ void load_mrec_part(const float *__restrict__ p, float x[12])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    x[8] = c.x; x[9] = c.y; x[10] = c.z; x[11] = c.w;
}
__device__ __forceinline__ void load_mrec_part(const double *__restrict__ p, double x[10])
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int e = 0; e < 5; ++e) {
        const double2 a = __ldg(q + e);
        x[2 * e] = a.x;
        x[2 * e + 1] = a.y;
    }
}
__device__ __forceinline__ void store_mrec_part(float *__restrict__ p, const float x[12])
{
    float4 *q = reinterpret_cast<float4 *>(p);
    q[0] = make_float4(x[0], x[1], x[2], x[3]);
    q[1] = make_float4(x[4], x[5], x[6], x[7]);
    q[2] = make_float4(x[8], x[9], x[10], x[11]);
}
__device__ __forceinline__ void store_mrec_part(double *__restrict__ p, const double x[10])
{
    double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int e = 0; e < 5; ++e) q[e] = make_double2(x[2 * e], x[2 * e + 1]);
}

HK_HD double map_factor(const MapGeo &m, double t) { return m.moving ? sin(m.omega * t) : 1.0; }

HK_HD void vertex_pos(const MapGeo &m, int i, int j, int k, double S, double x[3])
{
    const int idx[3] = {i, j, k};
    const double s = m.sx[i + GHOST] * m.sy[j + GHOST] * m.sz[k + GHOST];
    const double disp = m.amp * S * s;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[d] = (m.lo[d] + (m.hi[d] - m.lo[d]) * (double)idx[d] / (double)m.n[d]) + disp;
}

// volume, centroid and central second moments of cell (i,j,k) by the 2x2x2
// Gauss rule on its trilinear map (weights 1/8 times |det J|).  The map
// adds the same scalar D(p) = amp S sum_v psi_v(p) s_v to every coordinate
// of the reference point xi_c + p h (p in [-1/2, 1/2]^3), so
//   x - xi_c = p h + D (1,1,1),   J = diag(h) + (1,1,1) (grad_p D)^T,
//   det J = h_x h_y h_z (1 + sum_e (dD/dp_e) / h_e)
// (matrix determinant lemma); moments are taken about the reference centre
// xi_c and shifted to the centroid.
HK_HD void cell_geometry(const MapGeo &m, int i, int j, int k, double S, double out[NGEO])
{
    const int idx[3] = {i, j, k};
    double h[3], xc[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        h[e] = m.h[e];
        xc[e] = m.lo[e] + ((double)idx[e] + 0.5) * h[e];
    }
    const double aS = m.amp * S;
    double sv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        sv[q] = m.sx[i + (q & 1) + GHOST] * m.sy[j + ((q >> 1) & 1) + GHOST] * m.sz[k + (q >> 2) + GHOST];
    const double hprod = h[0] * h[1] * h[2];
    // D and its p-gradient at the 2x2x2 Gauss points, one axis at a time: at
    // the point index ia (p = -g, +g) vertex 0 of the axis weighs 1/2 - p and
    // vertex 1 weighs 1/2 + p; a derivative along an axis is the difference
    // of its two vertex values, constant along that axis.
    const double wv[2][2] = {{0.5 + GAUSS_S, 0.5 - GAUSS_S}, {0.5 - GAUSS_S, 0.5 + GAUSS_S}};
    double ax[2][4], dax[4];  // along x: [ix][b + 2c], and d/dp_x at [b + 2c]
#pragma unroll
    for (int yz = 0; yz < 4; ++yz) {
        const double v0 = sv[2 * yz], v1 = sv[2 * yz + 1];
        dax[yz] = v1 - v0;
#pragma unroll
        for (int ix = 0; ix < 2; ++ix) ax[ix][yz] = v0 * wv[ix][0] + v1 * wv[ix][1];
    }
    double axy[2][2][2], dxy[2][2], dyx[2][2];  // [ix][iy][c], d/dp_x at [iy][c], d/dp_y at [ix][c]
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int iy = 0; iy < 2; ++iy) {
#pragma unroll
            for (int ix = 0; ix < 2; ++ix)
                axy[ix][iy][c] = ax[ix][2 * c] * wv[iy][0] + ax[ix][2 * c + 1] * wv[iy][1];
            dxy[iy][c] = dax[2 * c] * wv[iy][0] + dax[2 * c + 1] * wv[iy][1];
        }
#pragma unroll
        for (int ix = 0; ix < 2; ++ix) dyx[ix][c] = ax[ix][2 * c + 1] - ax[ix][2 * c];
    }
    double Y[8][3], w[8], vol = 0.0, m1[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ix = q & 1, iy = (q >> 1) & 1, iz = q >> 2;
        const double p[3] = {ix ? GAUSS_S : -GAUSS_S, iy ? GAUSS_S : -GAUSS_S, iz ? GAUSS_S : -GAUSS_S};
        double D = axy[ix][iy][0] * wv[iz][0] + axy[ix][iy][1] * wv[iz][1];
        const double gD[3] = {dxy[iy][0] * wv[iz][0] + dxy[iy][1] * wv[iz][1],
                              dyx[ix][0] * wv[iz][0] + dyx[ix][1] * wv[iz][1], axy[ix][iy][1] - axy[ix][iy][0]};
        D *= aS;
        const double det = hprod * (1.0 + aS * (gD[0] * m.ih[0] + gD[1] * m.ih[1] + gD[2] * m.ih[2]));
        w[q] = 0.125 * fabs(det);
        for (int d = 0; d < 3; ++d) Y[q][d] = p[d] * h[d] + D;
        vol += w[q];
        for (int d = 0; d < 3; ++d) m1[d] += w[q] * Y[q][d];
    }
    const double ivol = 1.0 / vol;
    const double cy[3] = {m1[0] * ivol, m1[1] * ivol, m1[2] * ivol};
    double M[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const double dx = Y[r][0] - cy[0], dy = Y[r][1] - cy[1], dz = Y[r][2] - cy[2];
        M[0] += w[r] * dx * dx;
        M[1] += w[r] * dy * dy;
        M[2] += w[r] * dz * dz;
        M[3] += w[r] * dx * dy;
        M[4] += w[r] * dx * dz;
        M[5] += w[r] * dy * dz;
    }
    out[0] = vol;
    for (int d = 0; d < 3; ++d) out[1 + d] = xc[d] + cy[d];
    for (int e = 0; e < 6; ++e) out[4 + e] = M[e] * ivol;
}

// The same record for the mixed path, with the small quantities in FP32:
// the relative Jacobian 1 + sum_e (dD/dp_e)/h_e, the point offsets
// p h + D about the reference centre, the centroid offset and the central
// moments are all of the size of a cell (or of the displacement), so FP32
// keeps them to about 1e-7 relative, the precision of the reconstruction
// that reads them; the volume h_x h_y h_z (relative volume) and the centroid
// xi_c + offset are assembled in FP64.  fm receives the central moments in
// FP32 (the copy the FP32 reconstruction reads).
__device__ __forceinline__ void cell_geometry_mixed(const MapGeo &m, int i, int j, int k, float aS,
                                                    double out[NGEO], float fm[GEOF])
{
    const float g = float(GAUSS_S);
    float sv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        sv[q] = m.sxf[i + (q & 1) + GHOST] * m.syf[j + ((q >> 1) & 1) + GHOST] * m.szf[k + (q >> 2) + GHOST];
    const float wv[2][2] = {{0.5f + g, 0.5f - g}, {0.5f - g, 0.5f + g}};
    float ax[2][4], dax[4];
#pragma unroll
    for (int yz = 0; yz < 4; ++yz) {
        const float v0 = sv[2 * yz], v1 = sv[2 * yz + 1];
        dax[yz] = v1 - v0;
#pragma unroll
        for (int ix = 0; ix < 2; ++ix) ax[ix][yz] = v0 * wv[ix][0] + v1 * wv[ix][1];
    }
    float axy[2][2][2], dxy[2][2], dyx[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int iy = 0; iy < 2; ++iy) {
#pragma unroll
            for (int ix = 0; ix < 2; ++ix)
                axy[ix][iy][c] = ax[ix][2 * c] * wv[iy][0] + ax[ix][2 * c + 1] * wv[iy][1];
            dxy[iy][c] = dax[2 * c] * wv[iy][0] + dax[2 * c + 1] * wv[iy][1];
        }
#pragma unroll
        for (int ix = 0; ix < 2; ++ix) dyx[ix][c] = ax[ix][2 * c + 1] - ax[ix][2 * c];
    }
    float Y[8][3], w[8], vr = 0.0f, m1[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int ix = q & 1, iy = (q >> 1) & 1, iz = q >> 2;
        const float p[3] = {ix ? g : -g, iy ? g : -g, iz ? g : -g};
        const float D = aS * (axy[ix][iy][0] * wv[iz][0] + axy[ix][iy][1] * wv[iz][1]);
        const float gD[3] = {dxy[iy][0] * wv[iz][0] + dxy[iy][1] * wv[iz][1],
                             dyx[ix][0] * wv[iz][0] + dyx[ix][1] * wv[iz][1], axy[ix][iy][1] - axy[ix][iy][0]};
        // relative Jacobian times the Gauss weight 1/8
        w[q] = 0.125f * fabsf(1.0f + aS * (gD[0] * m.ihf[0] + gD[1] * m.ihf[1] + gD[2] * m.ihf[2]));
#pragma unroll
        for (int d = 0; d < 3; ++d) Y[q][d] = p[d] * m.hf[d] + D;
        vr += w[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) m1[d] += w[q] * Y[q][d];
    }
    const float ivr = 1.0f / vr;
    const float cy[3] = {m1[0] * ivr, m1[1] * ivr, m1[2] * ivr};
    float M[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float dx = Y[r][0] - cy[0], dy = Y[r][1] - cy[1], dz = Y[r][2] - cy[2];
        M[0] += w[r] * dx * dx;
        M[1] += w[r] * dy * dy;
        M[2] += w[r] * dz * dz;
        M[3] += w[r] * dx * dy;
        M[4] += w[r] * dx * dz;
        M[5] += w[r] * dy * dz;
    }
    const int idx[3] = {i, j, k};
    out[0] = m.h[0] * m.h[1] * m.h[2] * double(vr);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        out[1 + d] = (m.lo[d] + ((double)idx[d] + 0.5) * m.h[d]) + double(cy[d]);
        fm[6 + d] = cy[d];
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        fm[e] = M[e] * ivr;
        out[4 + e] = double(fm[e]);
    }
}

// ---------------------------------------------------------------------------
// reconstruction on a trilinear cell: the rows of the least squares are the
// neighbour means of the monomials in the centre cell's scaled frame minus
// the centre cell's own; with centroid c and central second moments M of
// each cell (per unit volume) they are, for Delta = c_nb - c_c:
//   linear    Delta_d / h
//   quadratic (M_nb,de - M_c,de)/h^2 + Delta_d Delta_e / h^2.
// ---------------------------------------------------------------------------
template <typename R> struct CellFrame {
    double c[3];
    double h;
    double Mh[6];   // M_c / h^2: the cell means of the quadratic monomials
};

__device__ __forceinline__ void read_geo(const double *__restrict__ geo, const Geo &g, int i, int j, int k,
                                         double rec[NGEO])
{
    const long long p = pidx(g, i, j, k);
#pragma unroll
    for (int e = 0; e < NGEO; ++e) rec[e] = geo[e * g.pstride + p];
}

// centroid, h = |Omega|^(1/3) and the scaled second moments of cell (i,j,k)
template <typename R>
__device__ __forceinline__ void make_frame(const double *__restrict__ geo, const Geo &g, int i, int j, int k,
                                           CellFrame<R> &F)
{
    double rec[NGEO];
    read_geo(geo, g, i, j, k, rec);
    F.c[0] = rec[1];
    F.c[1] = rec[2];
    F.c[2] = rec[3];
    F.h = cbrt(rec[0]);
    const double ih2 = 1.0 / (F.h * F.h);
#pragma unroll
    for (int e = 0; e < 6; ++e) F.Mh[e] = rec[4 + e] * ih2;
}

// row of the big-stencil system for the neighbour at offset o
template <typename R>
__device__ __forceinline__ void neighbour_row(const double *__restrict__ geo, const Geo &g, const CellFrame<R> &F,
                                              int i, int j, int k, R row[9])
{
    double rec[NGEO];
    read_geo(geo, g, i, j, k, rec);
    const double ih = 1.0 / F.h, ih2 = ih * ih;
    const double D[3] = {rec[1] - F.c[0], rec[2] - F.c[1], rec[3] - F.c[2]};
    row[0] = R(D[0] * ih);
    row[1] = R(D[1] * ih);
    row[2] = R(D[2] * ih);
    row[3] = R(rec[4] * ih2 - F.Mh[0] + D[0] * D[0] * ih2);
    row[4] = R(rec[5] * ih2 - F.Mh[1] + D[1] * D[1] * ih2);
    row[5] = R(rec[6] * ih2 - F.Mh[2] + D[2] * D[2] * ih2);
    row[6] = R(rec[7] * ih2 - F.Mh[3] + D[0] * D[1] * ih2);
    row[7] = R(rec[8] * ih2 - F.Mh[4] + D[0] * D[2] * ih2);
    row[8] = R(rec[9] * ih2 - F.Mh[5] + D[1] * D[2] * ih2);
}

// the 18 offsets of the big stencil (3x3x3 block minus centre and corners)
__device__ __forceinline__ void big_offset(int s, int o[3])
{
    // enumerate k0, j0, i0 in -1..1, skipping the centre and the 8 corners
    int cnt = 0;
    for (int k0 = -1; k0 <= 1; ++k0)
        for (int j0 = -1; j0 <= 1; ++j0)
            for (int i0 = -1; i0 <= 1; ++i0) {
                if ((i0 == 0 && j0 == 0 && k0 == 0) || (i0 * j0 * k0 != 0)) continue;
                if (cnt == s) {
                    o[0] = i0;
                    o[1] = j0;
                    o[2] = k0;
                }
                ++cnt;
            }
}

// in-place Cholesky of a packed symmetric n x n matrix (lower, row-major
// packed: A[i*(i+1)/2 + j], j <= i) and solve.  The diagonal slots keep the
// INVERSE of L's diagonal (1/sqrt of the pivot), so neither the factor nor
// the solves divide.
template <typename R, int N> __device__ __forceinline__ void chol_factor(R A[N * (N + 1) / 2])
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            R s = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
            if (i == j) A[i * (i + 1) / 2 + i] = m_rsqrt(s);
            else A[i * (i + 1) / 2 + j] = s * A[j * (j + 1) / 2 + j];
        }
    }
}
template <typename R, int N> __device__ __forceinline__ void chol_solve(const R L[N * (N + 1) / 2], R b[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i * (i + 1) / 2 + k] * b[k];
        b[i] = s * L[i * (i + 1) / 2 + i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        R s = b[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) s -= L[k * (k + 1) / 2 + i] * b[k];
        b[i] = s * L[i * (i + 1) / 2 + i];
    }
}

// offsets of the 4 cells of sub-stencil M (same family as on the uniform mesh)
template <int M> __device__ __forceinline__ void sub_offsets(int o[4][3])
{
    constexpr int p = M >> 3, s = M & 7;
    constexpr int sa = (s & 1) ? -1 : 1, sb = (s & 2) ? -1 : 1, sc = (s & 4) ? -1 : 1;
    constexpr int a = p, b = (p + 1) % 3, c = (p + 2) % 3;
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r][0] = o[r][1] = o[r][2] = 0;
    o[0][a] = sa;
    o[1][b] = sb;
    o[2][a] = sa;
    o[2][b] = sb;
    o[3][c] = sc;
}

// linear least squares over the 4 cells of a sub-stencil (3x3 normal
// equations): rows r (linear means in the centre frame), data dq
template <typename R> __device__ __forceinline__ void sub_lsq(const R r[4][3], const R dq[4], R bvec[3])
{
    R G[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R rhs[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        G[0] += r[q][0] * r[q][0];
        G[1] += r[q][1] * r[q][0];
        G[2] += r[q][1] * r[q][1];
        G[3] += r[q][2] * r[q][0];
        G[4] += r[q][2] * r[q][1];
        G[5] += r[q][2] * r[q][2];
#pragma unroll
        for (int d = 0; d < 3; ++d) rhs[d] += r[q][d] * dq[q];
    }
    chol_factor<R, 3>(G);
    chol_solve<R, 3>(G, rhs);
    bvec[0] = rhs[0];
    bvec[1] = rhs[1];
    bvec[2] = rhs[2];
}

// smoothness indicator of P0 on a general cell: cell means of the squared
// derivatives in the scaled frame, with the cell's second moments Mh
template <typename R> __device__ __forceinline__ R beta_quadratic_mapped(const R a[9], const R Mh[6])
{
    // grad P0 = g_d(0) + v_d . X with v_x = (2axx, axy, axz), v_y = (axy, 2ayy, ayz), v_z = (axz, ayz, 2azz)
    const R v[3][3] = {{R(2) * a[3], a[6], a[7]}, {a[6], R(2) * a[4], a[8]}, {a[7], a[8], R(2) * a[5]}};
    R s = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const R *u = v[d];
        const R quad = u[0] * u[0] * Mh[0] + u[1] * u[1] * Mh[1] + u[2] * u[2] * Mh[2] +
                       R(2) * (u[0] * u[1] * Mh[3] + u[0] * u[2] * Mh[4] + u[1] * u[2] * Mh[5]);
        s += a[d] * a[d] + quad;
    }
    const R d2 = R(4) * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5]);
    const R m2 = a[6] * a[6] + a[7] * a[7] + a[8] * a[8];
    return s + d2 + m2;
}

template <typename R>
__device__ __forceinline__ R poly9_mapped(const R c[9], const R X[3], const R Mh[6])
{
    return c[0] * X[0] + c[1] * X[1] + c[2] * X[2] + c[3] * (X[0] * X[0] - Mh[0]) + c[4] * (X[1] * X[1] - Mh[1]) +
           c[5] * (X[2] * X[2] - Mh[2]) + c[6] * (X[0] * X[1] - Mh[3]) + c[7] * (X[0] * X[2] - Mh[4]) +
           c[8] * (X[1] * X[2] - Mh[5]);
}

// the 24 face Gauss points of cell (i,j,k) in its scaled frame
__device__ __forceinline__ void cell_gauss_point(const MapGeo &m, int i, int j, int k, double S, int gq,
                                                 const double c[3], double h, double X[3])
{
    const int d = gq / 8, side = (gq / 4) & 1, ga = (gq >> 1) & 1, gb = gq & 1;
    double p[3];
    p[d] = side ? 0.5 : -0.5;
    p[(d + 1) % 3] = ga ? GAUSS_S : -GAUSS_S;
    p[(d + 2) % 3] = gb ? GAUSS_S : -GAUSS_S;
    double x[3] = {0, 0, 0};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
                double v[3];
                vertex_pos(m, i + a, j + b, k + cc, S, v);
                const double psi = 0.125 * (1.0 + 2.0 * (2 * a - 1) * p[0]) * (1.0 + 2.0 * (2 * b - 1) * p[1]) *
                                   (1.0 + 2.0 * (2 * cc - 1) * p[2]);
                for (int e = 0; e < 3; ++e) x[e] += v[e] * psi;
            }
    for (int e = 0; e < 3; ++e) X[e] = (x[e] - c[e]) / h;
}

// P0 of one variable on a trilinear cell: right-hand side A^T dQ over the
// 18 neighbours, solved with the Cholesky factor N of the normal matrix
template <typename R>
__device__ __forceinline__ void p0_mapped(const double *__restrict__ Qv, const double *__restrict__ geo, const Geo &g,
                                          const CellFrame<R> &F, const R N[45], int i, int j, int k, double qc,
                                          R a[9])
{
#pragma unroll
    for (int n = 0; n < 9; ++n) a[n] = R(0);
#pragma unroll 1
    for (int s = 0; s < 18; ++s) {
        int o[3];
        big_offset(s, o);
        R row[9];
        neighbour_row<R>(geo, g, F, i + o[0], j + o[1], k + o[2], row);
        const R dq = R(Qv[pidx(g, i + o[0], j + o[1], k + o[2])] - qc);
#pragma unroll
        for (int n = 0; n < 9; ++n) a[n] += row[n] * dq;
    }
    chol_solve<R, 9>(N, a);
}

template <typename R>
__device__ __forceinline__ void normal_matrix_mapped(const double *__restrict__ geo, const Geo &g,
                                                     const CellFrame<R> &F, int i, int j, int k, R N[45])
{
#pragma unroll
    for (int e = 0; e < 45; ++e) N[e] = R(0);
#pragma unroll 1
    for (int s = 0; s < 18; ++s) {
        int o[3];
        big_offset(s, o);
        R row[9];
        neighbour_row<R>(geo, g, F, i + o[0], j + o[1], k + o[2], row);
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) N[a * (a + 1) / 2 + b] += row[a] * row[b];
    }
    chol_factor<R, 9>(N);
}

// P_m of one variable on a trilinear cell (linear least squares over its 4
// neighbours)
template <int M, typename R>
__device__ __forceinline__ void pm_mapped(const double *__restrict__ Qv, const double *__restrict__ geo, const Geo &g,
                                          const CellFrame<R> &F, int i, int j, int k, double qc, R b[3])
{
    int o[4][3];
    sub_offsets<M>(o);
    R rows[4][3], dqs[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        R row[9];
        neighbour_row<R>(geo, g, F, i + o[r][0], j + o[r][1], k + o[r][2], row);
        rows[r][0] = row[0];
        rows[r][1] = row[1];
        rows[r][2] = row[2];
        dqs[r] = R(Qv[pidx(g, i + o[r][0], j + o[r][1], k + o[r][2])] - qc);
    }
    sub_lsq(rows, dqs, b);
}

template <typename R>
__device__ __forceinline__ void pm_mapped_rt(const double *__restrict__ Qv, const double *__restrict__ geo,
                                             const Geo &g, const CellFrame<R> &F, int i, int j, int k, double qc,
                                             int m, R b[3])
{
    switch (m) {
#define HK_PMRT(M)                                        \
    case M:                                               \
        pm_mapped<M, R>(Qv, geo, g, F, i, j, k, qc, b);   \
        break;
        HK_FOR_SUBSTENCILS(HK_PMRT)
#undef HK_PMRT
    default:
        b[0] = b[1] = b[2] = R(0);
    }
}

// literal positivity check (Sec. 4) on a trilinear cell
template <typename R>
__device__ __forceinline__ bool positivity_violated_mapped(const double *__restrict__ Q, const double *__restrict__ geo,
                                                        const Geo &g, const MapGeo &m, double S, int i, int j, int k,
                                                        const CellFrame<R> &F, R gamma)
{
    const R Mh[6] = {R(F.Mh[0]), R(F.Mh[1]), R(F.Mh[2]), R(F.Mh[3]), R(F.Mh[4]), R(F.Mh[5])};
    R N[45];
    normal_matrix_mapped<R>(geo, g, F, i, j, k, N);
    for (int mm = 0; mm <= 24; ++mm) {
        R cf[5][9], qcv[5];
        for (int v = 0; v < 5; ++v) {
            const double *Qv = Q + v * g.pstride;
            const double qc = Qv[pidx(g, i, j, k)];
            qcv[v] = R(qc);
            if (mm == 0) {
                p0_mapped<R>(Qv, geo, g, F, N, i, j, k, qc, cf[v]);
            } else {
                R b[3];
                pm_mapped_rt<R>(Qv, geo, g, F, i, j, k, qc, mm - 1, b);
                for (int n = 0; n < 9; ++n) cf[v][n] = n < 3 ? b[n] : R(0);
            }
        }
        for (int gq = 0; gq < 24; ++gq) {
            double Xd[3];
            cell_gauss_point(m, i, j, k, S, gq, F.c, F.h, Xd);
            const R X[3] = {R(Xd[0]), R(Xd[1]), R(Xd[2])};
            R W[5];
            for (int v = 0; v < 5; ++v) W[v] = qcv[v] + poly9_mapped(cf[v], X, Mh);
            if (W[0] < R(0) || pressure_negative(W)) return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Per-cell staging for the reconstruction: the 18 neighbours' centroid
// offsets in the scaled frame, (c_nb - c)/h, formed once in FP64 and kept in
// shared memory in the working precision; in the mixed path also the 90
// differences Q_nb - Q_c, formed from the split state (hi_nb - hi_c) +
// (lo_nb - lo_c) when the handle keeps one, else in FP64.  Each thread owns one column of
// the block's array (stride RM_BS), so no synchronisation is needed.
// ---------------------------------------------------------------------------
constexpr int RM_BS = 64;  // threads per block of the reconstruction kernel
template <typename R> struct RmStage {
    static constexpr bool dq = sizeof(R) == 4;
    static constexpr int n = 54 + (dq ? 90 : 0);
};

// offset of big-stencil neighbour s (0..17, the enumeration of big_offset)
__device__ __forceinline__ void big_offset_rt(int s, int o[3])
{
    // skip the centre (13) and the corners (0, 2, 6, 8, 18, 20, 24, 26)
    int p = s + 1;
    p += p >= 2;
    p += p >= 6;
    p += p >= 8;
    p += p >= 13;
    p += p >= 18;
    p += p >= 20;
    p += p >= 24;
    o[0] = p % 3 - 1;
    o[1] = (p / 3) % 3 - 1;
    o[2] = p / 9 - 1;
}


// row of the big-stencil system for neighbour s from the staged offsets and
// the neighbour's second moments
template <typename R>
__device__ __forceinline__ void staged_row(const R *sh, const double *__restrict__ geo, const Geo &g, R ih2,
                                           const R Mh[6], int s, long long pn, R row[9],
                                           const float *__restrict__ geof = nullptr)
{
    const R D0 = sh[(3 * s + 0) * RM_BS], D1 = sh[(3 * s + 1) * RM_BS], D2 = sh[(3 * s + 2) * RM_BS];
    R mm[6];
    if constexpr (sizeof(R) == 4) {
        if (geof) {
#pragma unroll
            for (int e = 0; e < 6; ++e) mm[e] = geof[e * g.pstride + pn] * ih2;
        } else {
#pragma unroll
            for (int e = 0; e < 6; ++e) mm[e] = R(geo[(4 + e) * g.pstride + pn]) * ih2;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) mm[e] = R(geo[(4 + e) * g.pstride + pn]) * ih2;
    }
    row[0] = D0;
    row[1] = D1;
    row[2] = D2;
    row[3] = mm[0] - Mh[0] + D0 * D0;
    row[4] = mm[1] - Mh[1] + D1 * D1;
    row[5] = mm[2] - Mh[2] + D2 * D2;
    row[6] = mm[3] - Mh[3] + D0 * D1;
    row[7] = mm[4] - Mh[4] + D0 * D2;
    row[8] = mm[5] - Mh[5] + D1 * D2;
}

// Q_nb - Q_c of variable v at big-stencil neighbour s
template <typename R>
__device__ __forceinline__ R staged_dq(const R *sh, const double *__restrict__ Q, const Geo &g, int v, int s,
                                       long long pn, double qc)
{
    if constexpr (RmStage<R>::dq) return sh[(54 + 18 * v + s) * RM_BS];
    else return R(Q[v * g.pstride + pn] - qc);
}

// least-squares operator of sub-stencil M on a trilinear cell: b = P dq for
// the data dq of its 4 cells, P = (R^T R)^{-1} R^T with R the 4 x 3 linear
// rows; formed once per cell and applied to the five variables
// offsets of the 4 cells of sub-stencil M for a run-time M, by selects
// only (no run-time indexing of a local array)
__device__ __forceinline__ void sub_offsets_rt(int M, int o[4][3])
{
    const int p = M >> 3, s = M & 7;
    const int sa = (s & 1) ? -1 : 1, sb = (s & 2) ? -1 : 1, sc = (s & 4) ? -1 : 1;
    // unit vectors of the axes a = p, b = p + 1, c = p + 2 (mod 3)
    const int ea[3] = {p == 0, p == 1, p == 2};
    const int eb[3] = {p == 2, p == 0, p == 1};
    const int ec[3] = {p == 1, p == 2, p == 0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        o[0][d] = sa * ea[d];
        o[1][d] = sb * eb[d];
        o[2][d] = sa * ea[d] + sb * eb[d];
        o[3][d] = sc * ec[d];
    }
}

// big-stencil indices (0..17) of the 4 cells of each sub-stencil, 5 bits
// each, built at compile time from the same enumerations as
// sub_offsets_rt and the big-stencil enumeration; read from constant memory by the run-time
// sub-stencil loop (the index is uniform over the warp)
struct SubIdxTable {
    unsigned w[24];
};
constexpr int big_index_c(int x, int y, int z)
{
    const int p = (z + 1) * 9 + (y + 1) * 3 + (x + 1);
    return p - (p > 0) - (p > 2) - (p > 6) - (p > 8) - (p > 13) - (p > 18) - (p > 20) - (p > 24);
}
constexpr SubIdxTable make_sub_idx()
{
    SubIdxTable t{};
    for (int M = 0; M < 24; ++M) {
        const int p = M >> 3, s = M & 7;
        const int sa = (s & 1) ? -1 : 1, sb = (s & 2) ? -1 : 1, sc = (s & 4) ? -1 : 1;
        const int ea[3] = {p == 0, p == 1, p == 2}, eb[3] = {p == 2, p == 0, p == 1}, ec[3] = {p == 1, p == 2, p == 0};
        const int o[4][3] = {{sa * ea[0], sa * ea[1], sa * ea[2]},
                             {sb * eb[0], sb * eb[1], sb * eb[2]},
                             {sa * ea[0] + sb * eb[0], sa * ea[1] + sb * eb[1], sa * ea[2] + sb * eb[2]},
                             {sc * ec[0], sc * ec[1], sc * ec[2]}};
        unsigned w = 0;
        for (int q = 0; q < 4; ++q) w |= unsigned(big_index_c(o[q][0], o[q][1], o[q][2])) << (5 * q);
        t.w[M] = w;
    }
    return t;
}
// every sub-stencil names 4 distinct neighbours of the 18, and the 24
// sub-stencils are distinct
constexpr bool sub_idx_valid(const SubIdxTable &t)
{
    for (int M = 0; M < 24; ++M) {
        for (int q = 0; q < 4; ++q) {
            const unsigned a = (t.w[M] >> (5 * q)) & 31u;
            if (a >= 18u) return false;
            for (int r = 0; r < q; ++r)
                if (((t.w[M] >> (5 * r)) & 31u) == a) return false;
        }
        for (int N = 0; N < M; ++N)
            if (t.w[N] == t.w[M]) return false;
    }
    return (t.w[0] >> 20) == 0u;
}
static_assert(sub_idx_valid(make_sub_idx()), "sub-stencil index table");
static __constant__ SubIdxTable kSubIdx = make_sub_idx();
__device__ __forceinline__ int sub_cell(unsigned w, int q) { return (int)((w >> (5 * q)) & 31u); }

template <typename R>
__device__ __forceinline__ void sub_pinv(const R *sh, unsigned w, R P[3][4])
{
    R r[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R *rs = sh + 3 * sub_cell(w, q) * RM_BS;
#pragma unroll
        for (int d = 0; d < 3; ++d) r[q][d] = rs[d * RM_BS];
    }
    R G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            R sum = R(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) sum += r[q][a] * r[q][b];
            G[a][b] = sum;
        }
    // inverse of the symmetric 3 x 3 matrix by cofactors
    const R c00 = G[1][1] * G[2][2] - G[1][2] * G[2][1];
    const R c01 = G[1][2] * G[2][0] - G[1][0] * G[2][2];
    const R c02 = G[1][0] * G[2][1] - G[1][1] * G[2][0];
    const R c11 = G[0][0] * G[2][2] - G[0][2] * G[2][0];
    const R c12 = G[0][2] * G[1][0] - G[0][0] * G[1][2];
    const R c22 = G[0][0] * G[1][1] - G[0][1] * G[1][0];
    const R idet = R(1) / (G[0][0] * c00 + G[0][1] * c01 + G[0][2] * c02);
    const R Gi[3][3] = {{c00 * idet, c01 * idet, c02 * idet},
                        {c01 * idet, c11 * idet, c12 * idet},
                        {c02 * idet, c12 * idet, c22 * idet}};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) P[d][q] = Gi[d][0] * r[q][0] + Gi[d][1] * r[q][1] + Gi[d][2] * r[q][2];
}

// differences Q_nb - Q_c of variable v over the 4 cells of a sub-stencil
// (cells w of kSubIdx; offsets o for the FP64 path, which reads Q)
template <typename R>
__device__ __forceinline__ void sub_dq(const R *sh, const double *__restrict__ Q, const Geo &g, int v, int i, int j,
                                       int k, double qc, unsigned w, const int o[4][3], R dq[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if constexpr (RmStage<R>::dq) dq[q] = sh[(54 + 18 * v + sub_cell(w, q)) * RM_BS];
        else dq[q] = R(Q[v * g.pstride + pidx(g, i + o[q][0], j + o[q][1], k + o[q][2])] - qc);
    }
}

// sh: this thread's column of the block's staging array (RmStage<R>::n
// entries, stride RM_BS)
template <typename R>
__device__ __forceinline__ void recon_mapped_item(const double *__restrict__ Q, const double *__restrict__ geo,
                                                  R *__restrict__ coef, unsigned char *__restrict__ flag,
                                                  const Geo &g, const MapGeo &m, double S, const Scheme &Sch, Ctl *ctl,
                                                  R *sh, long long t)
{
    // FP32: the records are staged in the block's shared memory for a
    // coalesced copy (k_recon_mapped), so every thread takes part in the
    // stage's barrier; a thread past the box reconstructs the last cell
    // again and writes nothing
    const bool valid = t < g.cstride;
    if constexpr (!RmStage<R>::dq) {
        if (!valid) return;
    }
    if (!valid) t = g.cstride - 1;
    int i, j, k;
    split3(t, g.cx, g.cy, i, j, k);
    i -= 1;
    j -= 1;
    k -= 1;
    CellFrame<R> F;
    make_frame(geo, g, i, j, k, F);
    const double ih = 1.0 / F.h;
    const R ih2 = R(ih * ih);
    const R Mh[6] = {R(F.Mh[0]), R(F.Mh[1]), R(F.Mh[2]), R(F.Mh[3]), R(F.Mh[4]), R(F.Mh[5])};
    const R g0 = R(1.0 - 24.0 * Sch.Gamma_lin), gm = R(Sch.Gamma_lin), eps = R(Sch.weno_eps);
    const bool pow2 = Sch.weno_pow == 2;
    const long long pc = pidx(g, i, j, k);
    double qcd[5];
    R qcv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        qcd[v] = Q[v * g.pstride + pc];
        qcv[v] = R(qcd[v]);
    }
    // the centre's split state (mixed path with a split copy of Q)
    float hc[5] = {}, lc[5] = {};
    if constexpr (RmStage<R>::dq) {
        if (m.qsplit) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                hc[v] = m.qsplit[v * g.pstride + pc];
                lc[v] = m.qsplit[(5 + v) * g.pstride + pc];
            }
        }
    }
    // stage the neighbours' scaled centroid offsets (and, mixed, the data
    // differences).  Mixed: c_nb - c_c = o h + (off_nb - off_c) with off the
    // FP32 centroid offsets from the reference centres, all in FP32 (the
    // terms are of the size of a cell, so this keeps the FP32 rounding of
    // the FP64 difference)
    float offc[3] = {0.0f, 0.0f, 0.0f};
    const float ihf = float(ih);
    if constexpr (RmStage<R>::dq) {
        if (m.geof) {
#pragma unroll
            for (int d = 0; d < 3; ++d) offc[d] = m.geof[(6 + d) * g.pstride + pc];
        }
    }
#pragma unroll 1
    for (int s = 0; s < 18; ++s) {
        int o[3];
        big_offset_rt(s, o);
        const long long pn = pidx(g, i + o[0], j + o[1], k + o[2]);
        if (RmStage<R>::dq && m.geof) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                sh[(3 * s + d) * RM_BS] =
                    R((float(o[d]) * m.hf[d] + (m.geof[(6 + d) * g.pstride + pn] - offc[d])) * ihf);
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) sh[(3 * s + d) * RM_BS] = R((geo[(1 + d) * g.pstride + pn] - F.c[d]) * ih);
        }
        if constexpr (RmStage<R>::dq) {
            if (m.qsplit) {
                // from the split state: (hi_nb - hi_c) + (lo_nb - lo_c)
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    sh[(54 + 18 * v + s) * RM_BS] = (m.qsplit[v * g.pstride + pn] - hc[v]) +
                                                     (m.qsplit[(5 + v) * g.pstride + pn] - lc[v]);
            } else {
#pragma unroll
                for (int v = 0; v < 5; ++v) sh[(54 + 18 * v + s) * RM_BS] = R(Q[v * g.pstride + pn] - qcd[v]);
            }
        }
    }

    // P0 of every variable with the big stencil's normal matrix, factored
    // once.  FP32: P0 and beta0 stay in registers until the weights are
    // known; FP64 (more registers per value) parks them in the output slots
    // (0 and 1..9 of each variable)
    constexpr bool fold = RmStage<R>::dq;
    R p0[5][9], beta0[5];
    if constexpr (!fold) {
        // FP64: the five right-hand sides A^T dQ in one sweep over the 18
        // rows (each row formed once for all five), parked in the output
        // slots; the normal matrix takes a second sweep, since its 45
        // accumulators and these 45 do not fit in registers together
        R rhs[5][9];
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int n = 0; n < 9; ++n) rhs[v][n] = R(0);
#pragma unroll 1
        for (int s = 0; s < 18; ++s) {
            int o[3];
            big_offset_rt(s, o);
            const long long pn = pidx(g, i + o[0], j + o[1], k + o[2]);
            R row[9];
            staged_row<R>(sh, geo, g, ih2, Mh, s, pn, row, m.geof);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const R dq = staged_dq<R>(sh, Q, g, v, s, pn, qcd[v]);
#pragma unroll
                for (int n = 0; n < 9; ++n) rhs[v][n] += row[n] * dq;
            }
        }
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int n = 0; n < 9; ++n) coef[mrec_idx<R>(t, v, 1 + n)] = rhs[v][n];
    }
    {
        R N[45];
#pragma unroll
        for (int e = 0; e < 45; ++e) N[e] = R(0);
        // FP32: the five right-hand sides A^T dQ gathered in the same sweep
        // over the 18 rows as the normal matrix (each row, and the
        // neighbour's second moments it reads, formed once)
        R rhs[5][9];
#pragma unroll
        for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int n = 0; n < 9; ++n) rhs[v][n] = R(0);
#pragma unroll 1
        for (int s = 0; s < 18; ++s) {
            int o[3];
            big_offset_rt(s, o);
            R row[9];
            staged_row<R>(sh, geo, g, ih2, Mh, s, pidx(g, i + o[0], j + o[1], k + o[2]), row, m.geof);
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = 0; b <= a; ++b) N[a * (a + 1) / 2 + b] += row[a] * row[b];
            if constexpr (fold) {
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const R dq = sh[(54 + 18 * v + s) * RM_BS];
#pragma unroll
                    for (int n = 0; n < 9; ++n) rhs[v][n] += row[n] * dq;
                }
            }
        }
        chol_factor<R, 9>(N);
        if constexpr (fold) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                chol_solve<R, 9>(N, rhs[v]);
                beta0[v] = beta_quadratic_mapped(rhs[v], Mh);
#pragma unroll
                for (int n = 0; n < 9; ++n) p0[v][n] = rhs[v][n];
            }
        }
#pragma unroll 1
        for (int v = 0; v < (fold ? 0 : 5); ++v) {
            R a[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) a[n] = coef[mrec_idx<R>(t, v, 1 + n)];
            chol_solve<R, 9>(N, a);
            coef[mrec_idx<R>(t, v, 0)] = beta_quadratic_mapped(a, Mh);
#pragma unroll
            for (int n = 0; n < 9; ++n) coef[mrec_idx<R>(t, v, 1 + n)] = a[n];
        }
    }
    if constexpr (!fold) {
#pragma unroll
        for (int v = 0; v < 5; ++v) beta0[v] = coef[mrec_idx<R>(t, v, 0)];
    }
    // one pass over the sub-stencils (AoSums): the sums of the nonlinear
    // weights and of the linear part of P~, and the largest
    // |b_x| + |b_y| + |b_z| over the P_m (positivity bound)
    AoSums<R> acc[5];
    R bsum[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        acc[v].init(beta0[v], eps, pow2);
        bsum[v] = R(0);
    }
#pragma unroll 1
    for (int M = 0; M < 24; ++M) {
        const unsigned w = kSubIdx.w[M];
        int o[4][3] = {};
        if constexpr (!RmStage<R>::dq) sub_offsets_rt(M, o);
        R P[3][4];
        sub_pinv<R>(sh, w, P);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            R dq[4];
            sub_dq<R>(sh, Q, g, v, i, j, k, qcd[v], w, o, dq);
            R b[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) b[d] = P[d][0] * dq[0] + P[d][1] * dq[1] + P[d][2] * dq[2] + P[d][3] * dq[3];
            acc[v].add(beta0[v], eps, b);
            bsum[v] = m_max(bsum[v], m_abs(b[0]) + m_abs(b[1]) + m_abs(b[2]));
        }
    }
    // extents of X and of the monomials over the cell's 24 face Gauss
    // points, for the positivity bound.  Every coordinate of a point is
    // displaced by the same amp S sum_v psi_v s_v (trilinear weights psi_v,
    // vertex sine products s_v), so in the scaled frame
    //   X_e = (xi_centre,e - c_e)/h + p_e h_e/h + (amp S/h) sum_v psi_v s_v
    // for the point's reference offset p in [-1/2, 1/2]^3.
    R ext[9];
    {
        R sv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            sv[q] = R(m.sx[i + (q & 1) + GHOST]) * R(m.sy[j + ((q >> 1) & 1) + GHOST]) * R(m.sz[k + (q >> 2) + GHOST]);
        const int idx[3] = {i, j, k};
        R x0[3], hr[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const double he = m.h[e];
            x0[e] = R((m.lo[e] + ((double)idx[e] + 0.5) * he - F.c[e]) * ih);
            hr[e] = R(he * ih);
        }
        const R aSh = R(m.amp * S * ih);
#pragma unroll
        for (int n = 0; n < 9; ++n) ext[n] = R(0);
#pragma unroll 1
        for (int gq = 0; gq < 24; ++gq) {
            const int d = gq / 8, side = (gq / 4) & 1, ga = (gq >> 1) & 1, gb = gq & 1;
            R p[3];
            p[0] = p[1] = p[2] = R(0);
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int rel = (e - d + 3) % 3;  // 0: face normal, 1: first tangent, 2: second
                p[e] = rel == 0 ? (side ? R(0.5) : R(-0.5))
                                : (rel == 1 ? (ga ? R(GAUSS_S) : R(-GAUSS_S)) : (gb ? R(GAUSS_S) : R(-GAUSS_S)));
            }
            R wlo[3], whi[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                wlo[e] = R(0.5) - p[e];
                whi[e] = R(0.5) + p[e];
            }
            R dsum = R(0);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dsum += ((q & 1) ? whi[0] : wlo[0]) * (((q >> 1) & 1) ? whi[1] : wlo[1]) *
                        ((q >> 2) ? whi[2] : wlo[2]) * sv[q];
            const R dd = aSh * dsum;
            const R X[3] = {x0[0] + p[0] * hr[0] + dd, x0[1] + p[1] * hr[1] + dd, x0[2] + p[2] * hr[2] + dd};
            const R pn[9] = {X[0], X[1], X[2], X[0] * X[0] - Mh[0], X[1] * X[1] - Mh[1], X[2] * X[2] - Mh[2],
                             X[0] * X[1] - Mh[3], X[0] * X[2] - Mh[4], X[1] * X[2] - Mh[5]};
#pragma unroll
            for (int n = 0; n < 9; ++n) ext[n] = m_max(ext[n], m_abs(pn[n]));
        }
    }
    const R xmax = m_max(ext[0], m_max(ext[1], ext[2]));
    // the cell's record: FP32 into its slot of the block's stage (the staged
    // stencil data is no longer read once every thread is past this
    // barrier), FP64 straight to global memory
    R *rec = coef + t * MRec<R>::N;
    if constexpr (fold) {
        __syncthreads();
        rec = (sh - threadIdx.x) + threadIdx.x * MRec<R>::N;
    }
    R rad[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        R iw, f0, lin[3];
        acc[v].template combine<24>(g0, gm, iw, f0, lin);
        R out[MRec<R>::VS];
        out[0] = qcv[v];
        R r0 = R(0);
#pragma unroll
        for (int n = 0; n < 9; ++n) {
            const R a = fold ? p0[v][n] : coef[mrec_idx<R>(t, v, 1 + n)];
            r0 += m_abs(a) * ext[n];
            out[1 + n] = iw * (f0 * a + (n < 3 ? lin[n] : R(0)));
        }
#pragma unroll
        for (int n = 10; n < MRec<R>::VS; ++n) out[n] = R(0);
        store_mrec_part(rec + MRec<R>::VS * (1 + v), out);
        // bound of |P_m - Q_c| at the Gauss points for all 25 P_m
        rad[v] = m_max(r0, bsum[v] * xmax) * R(1.0000001);
    }
    // a cell whose bound does not certify positivity is marked 2 and gets
    // the literal check in positivity_mapped_item (a kernel of its own, so
    // that its registers do not weigh on this one)
    if (valid) flag[t] = (Sch.limiter && !positivity_certain(qcv, rad, R(Sch.gamma))) ? 2 : 0;
    // the cell frame for the flux kernels
    {
        R fr[MRec<R>::VS];
        fr[0] = R(F.c[0]);
        fr[1] = R(F.c[1]);
        fr[2] = R(F.c[2]);
        fr[3] = R(ih);
#pragma unroll
        for (int e = 0; e < 6; ++e) fr[4 + e] = Mh[e];
#pragma unroll
        for (int n = 10; n < MRec<R>::VS; ++n) fr[n] = R(0);
        store_mrec_part(rec, fr);
    }
}

// literal positivity check of the cells marked 2 by recon_mapped_item: all
// 25 polynomials at the cell's 24 face Gauss points; a violation sets P~ to
// the cell average (Sec. 4)
template <typename R>
__device__ __forceinline__ void positivity_mapped_item(const double *__restrict__ Q, const double *__restrict__ geo,
                                                       R *__restrict__ coef, unsigned char *__restrict__ flag,
                                                       const Geo &g, const MapGeo &m, double S, const Scheme &Sch,
                                                       Ctl *ctl, long long t)
{
    if (t >= g.cstride || flag[t] != 2) return;
    int i, j, k;
    split3(t, g.cx, g.cy, i, j, k);
    i -= 1;
    j -= 1;
    k -= 1;
    CellFrame<R> F;
    make_frame(geo, g, i, j, k, F);
    const bool bad = positivity_violated_mapped<R>(Q, geo, g, m, S, i, j, k, F, R(Sch.gamma));
    if (bad) {
        for (int v = 0; v < 5; ++v)
            for (int n = 1; n < 10; ++n) coef[mrec_idx<R>(t, v, n)] = R(0);
        atomicAdd(&ctl->flagged, 1);
    }
    flag[t] = bad ? 1 : 0;
}

// ---------------------------------------------------------------------------
// face flux on a bilinear face moving with the grid: one Gauss point per
// call, 4 lanes per face; stores the face-integrated flux (weight 1/4 times
// |X_a x X_b|), its time derivative and the swept volume rate
// (1/4 |X_a x X_b| U_g . n) -- 11 FP64 values per face.
// ---------------------------------------------------------------------------
constexpr int NFACE_M = 11;

template <typename R>
__device__ __forceinline__ void eval_cell_mapped(const R *__restrict__ coef, const Geo &g, long long ci,
                                                 const R xg[3], R val[5], R grad[5][3])
{
    R fr[MRec<R>::VS];
    load_mrec_part(coef + ci * MRec<R>::N, fr);
    const R c[3] = {fr[0], fr[1], fr[2]}, ih = fr[3];
    const R Mh[6] = {fr[4], fr[5], fr[6], fr[7], fr[8], fr[9]};
    const R X[3] = {(xg[0] - c[0]) * ih, (xg[1] - c[1]) * ih, (xg[2] - c[2]) * ih};
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        R part[MRec<R>::VS], a[9];
        load_mrec_part(coef + mrec_idx<R>(ci, v, 0), part);
#pragma unroll
        for (int n = 0; n < 9; ++n) a[n] = part[1 + n];
        val[v] = part[0] + poly9_mapped(a, X, Mh);
        grad[v][0] = (a[0] + R(2) * a[3] * X[0] + a[6] * X[1] + a[7] * X[2]) * ih;
        grad[v][1] = (a[1] + R(2) * a[4] * X[1] + a[6] * X[0] + a[8] * X[2]) * ih;
        grad[v][2] = (a[2] + R(2) * a[5] * X[2] + a[7] * X[0] + a[8] * X[1]) * ih;
    }
}

// The map displaces every coordinate of a vertex by the same scalar
// amp S(t) s_v (s_v the product of the vertex's sine factors) and moves it
// with velocity amp omega C(t) s_v in every coordinate.  On the bilinear face
// spanned by the reference edges h_A e_A and h_B e_B this gives, at face
// parameters (1/2 + ea, 1/2 + eb):
//   X   = xi + d (1,1,1),          d  = amp S sum_v phi_v s_v
//   X_a = h_A e_A + dA (1,1,1),    dA = amp S sum_v dphi_v/da s_v
//   X_b = h_B e_B + dB (1,1,1),    dB = amp S sum_v dphi_v/db s_v
//   U_g = ug (1,1,1),              ug = amp omega C sum_v phi_v s_v
// so the face geometry needs only the 4 sine products, in the working
// precision.
template <typename R, int D>
__device__ __forceinline__ void flux_mapped_item(const R *__restrict__ coef, double *__restrict__ Fout, const Geo &g,
                                                 const MapGeo &m, double Sf, double Cf, float aSf, float aUCf,
                                                 const Scheme &S, double dt, long long t)
{
    constexpr bool F32 = sizeof(R) == 4;  // mixed path: face geometry from the FP32 copies
    const int ex = g.nx + (D == 0), ey = g.ny + (D == 1);
    const long long nface = face_count<D>(g);
    long long face = t >> 2;
    const int gp = (int)(t & 3);
    const bool valid = face < nface;
    if (!valid) face = nface - 1;
    int i, j, k;
    {
        // the face index decoded with the precomputed divisors of ex and ey
        const unsigned u = (unsigned)face;
        const unsigned r = div32(u, g.dv[D == 0 ? 1 : 0]);
        i = (int)(u - r * (unsigned)ex);
        k = (int)div32(r, g.dv[D == 1 ? 3 : 2]);
        j = (int)(r - (unsigned)k * (unsigned)ey);
    }
    const int il = i - (D == 0), jl = j - (D == 1), kl = k - (D == 2);
    constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
    const R ea = (gp & 2) ? R(GAUSS_S) : R(-GAUSS_S), eb = (gp & 1) ? R(GAUSS_S) : R(-GAUSS_S);
    R sphi = R(0), spa = R(0), spb = R(0);
#pragma unroll
    for (int sa = 0; sa < 2; ++sa)
#pragma unroll
        for (int sb = 0; sb < 2; ++sb) {
            int o[3] = {i, j, k};
            o[A] += sa;
            o[B] += sb;
            R sv;
            if constexpr (F32) sv = m.sxf[o[0] + GHOST] * m.syf[o[1] + GHOST] * m.szf[o[2] + GHOST];
            else sv = R(m.sx[o[0] + GHOST]) * R(m.sy[o[1] + GHOST]) * R(m.sz[o[2] + GHOST]);
            const R qa = R(2 * sa - 1), qb = R(2 * sb - 1);
            sphi += R(0.25) * (R(1) + R(2) * qa * ea) * (R(1) + R(2) * qb * eb) * sv;
            spa += R(0.5) * qa * (R(1) + R(2) * qb * eb) * sv;
            spb += R(0.5) * qb * (R(1) + R(2) * qa * ea) * sv;
        }
    const R aS = F32 ? R(aSf) : R(m.amp * Sf);
    const R d = aS * sphi, dA = aS * spa, dB = aS * spb;
    const R ug = m.moving ? (F32 ? R(aUCf) : R(m.amp * m.omega * Cf)) * sphi : R(0);
    const int idx[3] = {i, j, k};
    R X[3], Xa[3], Xb[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if constexpr (F32) {
            const float he = m.hf[e];
            const float par = e == D ? 0.0f : (e == A ? 0.5f + float(ea) : 0.5f + float(eb));
            X[e] = R(m.lof[e] + (float(idx[e]) + par) * he) + d;
            Xa[e] = (e == A ? R(he) : R(0)) + dA;
            Xb[e] = (e == B ? R(he) : R(0)) + dB;
        } else {
            const double he = m.h[e];
            const double par = e == D ? 0.0 : (e == A ? 0.5 + (double)ea : 0.5 + (double)eb);
            X[e] = R(m.lo[e] + ((double)idx[e] + par) * he) + d;
            Xa[e] = (e == A ? R(he) : R(0)) + dA;
            Xb[e] = (e == B ? R(he) : R(0)) + dB;
        }
    }
    const R nrm[3] = {Xa[1] * Xb[2] - Xa[2] * Xb[1], Xa[2] * Xb[0] - Xa[0] * Xb[2], Xa[0] * Xb[1] - Xa[1] * Xb[0]};
    // |n| and 1/|n| from one reciprocal square root (no division)
    const R nn = nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2];
    const R iarea = m_rsqrt(nn), area = nn * iarea;
    const R ilb = m_rsqrt(Xb[0] * Xb[0] + Xb[1] * Xb[1] + Xb[2] * Xb[2]);
    R fr[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        fr[0][e] = nrm[e] * iarea;
        fr[2][e] = Xb[e] * ilb;
    }
    fr[1][0] = fr[2][1] * fr[0][2] - fr[2][2] * fr[0][1];
    fr[1][1] = fr[2][2] * fr[0][0] - fr[2][0] * fr[0][2];
    fr[1][2] = fr[2][0] * fr[0][1] - fr[2][1] * fr[0][0];
    // both cells' values and gradients, rotated to the face frame
    R Wc[2][5], dWc[2][3][5];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        R val[5], grad[5][3];
        eval_cell_mapped<R>(coef, g, s ? cidx(g, i, j, k) : cidx(g, il, jl, kl), X, val, grad);
        const R(&f)[3][3] = fr;
        Wc[s][0] = val[0];
        Wc[s][4] = val[4];
#pragma unroll
        for (int l = 0; l < 3; ++l) Wc[s][1 + l] = val[1] * f[l][0] + val[2] * f[l][1] + val[3] * f[l][2];
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            R dd[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) dd[v] = grad[v][0] * f[di][0] + grad[v][1] * f[di][1] + grad[v][2] * f[di][2];
            dWc[s][di][0] = dd[0];
            dWc[s][di][4] = dd[4];
#pragma unroll
            for (int l = 0; l < 3; ++l) dWc[s][di][1 + l] = dd[1] * f[l][0] + dd[2] * f[l][1] + dd[3] * f[l][2];
        }
    }
    // the frame moving with the grid (Remark 2): shift the states by U_g
    R Ug[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) Ug[l] = ug * (fr[l][0] + fr[l][1] + fr[l][2]);
    const R u2 = Ug[0] * Ug[0] + Ug[1] * Ug[1] + Ug[2] * Ug[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        R *W = Wc[s];
        W[4] = W[4] - (Ug[0] * W[1] + Ug[1] * W[2] + Ug[2] * W[3]) + R(0.5) * u2 * W[0];
#pragma unroll
        for (int l = 0; l < 3; ++l) W[1 + l] = W[1 + l] - Ug[l] * W[0];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            R *dW = dWc[s][e];
            dW[4] = dW[4] - (Ug[0] * dW[1] + Ug[1] * dW[2] + Ug[2] * dW[3]) + R(0.5) * u2 * dW[0];
#pragma unroll
            for (int l = 0; l < 3; ++l) dW[1 + l] = dW[1 + l] - Ug[l] * dW[0];
        }
    }
    R Fl[5], dFl[5];
    gks_flux<R>(Wc[0], dWc[0], Wc[1], dWc[1], S, R(dt), Fl, dFl);
    // back from the grid frame (u = u_rel + U_g), then to the global frame
    R Fb[5], dFb[5];
    Fb[0] = Fl[0];
    dFb[0] = dFl[0];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        Fb[1 + l] = Fl[1 + l] + Ug[l] * Fl[0];
        dFb[1 + l] = dFl[1 + l] + Ug[l] * dFl[0];
    }
    Fb[4] = Fl[4] + Ug[0] * Fl[1] + Ug[1] * Fl[2] + Ug[2] * Fl[3] + R(0.5) * u2 * Fl[0];
    dFb[4] = dFl[4] + Ug[0] * dFl[1] + Ug[1] * dFl[2] + Ug[2] * dFl[3] + R(0.5) * u2 * dFl[0];
    const R wgt = R(0.25) * area;
    R f[NFACE_M];
    f[0] = wgt * Fb[0];
    f[4] = wgt * Fb[4];
    f[5] = wgt * dFb[0];
    f[9] = wgt * dFb[4];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        // the frame is orthonormal: its inverse is its transpose
        f[1 + e] = wgt * (fr[0][e] * Fb[1] + fr[1][e] * Fb[2] + fr[2][e] * Fb[3]);
        f[6 + e] = wgt * (fr[0][e] * dFb[1] + fr[1][e] * dFb[2] + fr[2][e] * dFb[3]);
    }
    f[10] = R(0.25) * ug * (nrm[0] + nrm[1] + nrm[2]);
#pragma unroll
    for (int q = 0; q < NFACE_M; ++q) {
        f[q] += __shfl_xor_sync(0xffffffffu, f[q], 1);
        f[q] += __shfl_xor_sync(0xffffffffu, f[q], 2);
    }
    // lane gp stores the sums q = gp, gp + 4, gp + 8, so the FP64
    // conversions are spread over the face's 4 lanes
    static_assert(NFACE_M == 11, "the selection below covers 11 sums");
    if (valid) {
        const bool b0 = gp & 1, b1 = gp & 2;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const R v = b1 ? (b0 ? f[4 * r + 3] : f[4 * r + 2]) : (b0 ? f[4 * r + 1] : f[4 * r]);
            Fout[(gp + 4 * r) * nface + face] = double(v);
        }
        if (gp < 3) Fout[(gp + 8) * nface + face] = double(b1 ? f[10] : (b0 ? f[9] : f[8]));
    }
}

// residual R = -sum of the outward face-integrated fluxes, dR/dt, and the
// swept volume rate V of cell (i,j,k)
__device__ __forceinline__ void cell_residual_mapped(const double *__restrict__ Fx, const double *__restrict__ Fy,
                                                     const double *__restrict__ Fz, const Geo &g, int i, int j, int k,
                                                     double Rr[5], double dR[5], double &V)
{
    const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
    const long long nfy = (long long)g.nx * (g.ny + 1) * g.nz;
    const long long nfz = (long long)g.nx * g.ny * (g.nz + 1);
    const long long fx0 = ((long long)k * g.ny + j) * (g.nx + 1) + i;
    const long long fy0 = ((long long)k * (g.ny + 1) + j) * g.nx + i;
    const long long fz0 = ((long long)k * g.ny + j) * g.nx + i;
    const long long fzs = (long long)g.nx * g.ny;
#pragma unroll
    for (int v = 0; v < NFACE_M; ++v) {
        const double sx = Fx[v * nfx + fx0 + 1] - Fx[v * nfx + fx0];
        const double sy = Fy[v * nfy + fy0 + g.nx] - Fy[v * nfy + fy0];
        const double sz = Fz[v * nfz + fz0 + fzs] - Fz[v * nfz + fz0];
        const double r = -(sx + sy + sz);
        if (v < 5) Rr[v] = r;
        else if (v < 10) dR[v - 5] = r;
        else V = -r;
    }
}

// two-stage update of |Omega| Q with the volume advanced by the same
// formula from the swept rate (discrete geometric conservation law); vol is
// that volume at t_n, vnext receives it at t_{n+1}
template <int STAGE>
__device__ __forceinline__ void update_mapped_item(double *__restrict__ Qn, double *__restrict__ Qs,
                                                   double *__restrict__ Wacc, double *__restrict__ vol,
                                                   double *__restrict__ vnext, const double *__restrict__ Fx,
                                                   const double *__restrict__ Fy, const double *__restrict__ Fz,
                                                   const Geo &g, double gamma, Ctl *ctl, double dt, long long t)
{
    if (STAGE == 2 && t == 0) {
        ctl->t += dt;
        ctl->steps_done += 1;
    }
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    double Rr[5], dR[5], V;
    cell_residual_mapped(Fx, Fy, Fz, g, i, j, k, Rr, dR, V);
    const long long pi = pidx(g, i, j, k);
    if (STAGE == 1) {
        const double v0 = vol[t];
        const double vs = v0 + 0.5 * dt * V;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double x = v0 * Qn[q * g.pstride + pi];
            Qs[q * g.pstride + pi] = (x + 0.5 * dt * Rr[q] + 0.125 * dt * dt * dR[q]) / vs;
            Wacc[q * g.ncell + t] = x + dt * Rr[q] + (dt * dt / 6.0) * dR[q];
        }
        vnext[t] = v0 + dt * V;
    } else {
        const double vn = vnext[t];
        double W[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            W[q] = (Wacc[q * g.ncell + t] + (dt * dt / 3.0) * dR[q]) / vn;
            Qn[q * g.pstride + pi] = W[q];
        }
        vol[t] = vn;
        const double p = (gamma - 1.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0]);
        if (!(W[0] > 0.0) || !(p > 0.0)) atomicOr(&ctl->status, 1);
    }
}

}  // namespace hk
