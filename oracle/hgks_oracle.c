/*
 * HGKS oracle -- a plain, slow FP64 CPU implementation of the third-order
 * WENO-AO reconstruction and two-stage gas-kinetic scheme of Pan & Xu,
 * "High-order gas-kinetic scheme with three-dimensional WENO reconstruction
 * for the Euler and Navier-Stokes solutions" (arXiv 1909.01580).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only code allowed to load this
 * library; the product path never calls it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Style: every routine follows the paper's definitions in the paper's order
 * with generic numerics -- Householder least squares for the WENO stencils,
 * Gauss quadrature over trilinear hexahedra for every cell integral,
 * Gaussian elimination for the 5x5 moment systems, and a small sparse
 * polynomial integrator for every velocity-space moment -- so that a reader
 * can check it against the paper by eye.  Nothing is fused or reordered for
 * speed.  Readings of passages the paper leaves open are marked "Reading:".
 *
 * Pins of the two parts the paper's printed values do not reach: the
 * positivity fallback (Sec. 4 limiter) by hand-built cells whose candidate
 * polynomials go negative at exactly one of the 24 Gauss points, or only
 * between them; the Prandtl-number heat-flux correction (a reading: the
 * paper is silent on it) by its Pr = 1 no-op and by the Navier-Stokes limit
 * of the heat flux, -kappa dT/dx with kappa = mu gamma/((gamma - 1) Pr).
 *
 * Layout of every state array crossing this file's interface:
 * conservative cell averages (rho, rho U, rho V, rho W, rho E), SoA
 * [5][nz][ny][nx], x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define NV 5
#define GH 3 /* ghost layers: the big stencil S' reaches two cells, and the
                reconstruction of the first ghost cell reaches one more */

/* ------------------------------------------------------------------------ */
/* configuration (mirrored field by field by the Python loader)              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n[3];          /* cells in x, y, z                                   */
    double lo[3];      /* physical box, reference coordinates xi            */
    double hi[3];
    int mesh;          /* 0 uniform, 1 static mapped, 2 moving mapped        */
    double amp;        /* mapped mesh: x_d = xi_d + amp*S(t)*prod sin(...)   */
    double omega;      /* moving mesh: S(t) = sin(omega t); static: S = 1    */
    double gamma, mu, Pr;
    int bc[6];         /* -x,+x,-y,+y,-z,+z : 0 periodic, 1 reflective,
                          2 non-reflecting (outflow)                          */
    double Gamma_lin;  /* linear weight of each sub-stencil (Sec. 2)         */
    double weno_eps;   /* epsilon of the nonlinear weights                   */
    int weno_pow;      /* exponent on tau/(beta+eps); 1 as printed           */
    double tau_eps, tau_C; /* collision-time constants (Sec. 4)              */
    int limiter;       /* positivity fallback on/off                         */
    int nthreads;      /* OpenMP threads (0 = runtime default)               */
    int charvar;       /* 1: reconstruct characteristic variables (Sec. 4)   */
    double mu_pow;     /* mu = mu (T/T_ref)^mu_pow (isotropic turbulence,
                          Sec. 4: 0.76); 0 keeps mu constant                   */
    double T_ref;      /* reference temperature p/rho of that law            */
    int stencil;       /* 0: big stencil S and 24 sub-stencils (Sec. 2);
                          1: S' and its 8 sub-stencils (Remark of Sec. 2)    */
} orc_cfg;

#ifdef _OPENMP
#include <omp.h>
#define ORC_THREADS(cfg) ((cfg)->nthreads > 0 ? (cfg)->nthreads : omp_get_max_threads())
#else
#define ORC_THREADS(cfg) 1
#endif

int orc_threads_used(const orc_cfg *cfg) { (void)cfg; return ORC_THREADS(cfg); }

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                               */
/* ------------------------------------------------------------------------ */

/* Least squares min ||A x - b|| for each of nrhs right-hand sides by
 * Householder QR (A is m x n row-major, m >= n; A and B are overwritten).
 * Returns 0, or -1 when A is rank deficient. */
static int lsq_householder(int m, int n, double *A, int nrhs, double *B, double *X)
{
    for (int k = 0; k < n; ++k) {
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
        norm = sqrt(norm);
        if (norm == 0.0) return -1;
        double alpha = A[k * n + k] > 0 ? -norm : norm;
        double v0 = A[k * n + k] - alpha;
        /* v = (v0, A[k+1..m-1][k]); H = I - 2 v v^T / (v^T v) */
        double vtv = v0 * v0;
        for (int i = k + 1; i < m; ++i) vtv += A[i * n + k] * A[i * n + k];
        for (int j = k + 1; j < n; ++j) {
            double s = v0 * A[k * n + j];
            for (int i = k + 1; i < m; ++i) s += A[i * n + k] * A[i * n + j];
            s = 2.0 * s / vtv;
            A[k * n + j] -= s * v0;
            for (int i = k + 1; i < m; ++i) A[i * n + j] -= s * A[i * n + k];
        }
        for (int r = 0; r < nrhs; ++r) {
            double s = v0 * B[k * nrhs + r];
            for (int i = k + 1; i < m; ++i) s += A[i * n + k] * B[i * nrhs + r];
            s = 2.0 * s / vtv;
            B[k * nrhs + r] -= s * v0;
            for (int i = k + 1; i < m; ++i) B[i * nrhs + r] -= s * A[i * n + k];
        }
        A[k * n + k] = alpha;
    }
    for (int r = 0; r < nrhs; ++r) {
        for (int k = n - 1; k >= 0; --k) {
            double s = B[k * nrhs + r];
            for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * X[j * nrhs + r];
            X[k * nrhs + r] = s / A[k * n + k];
        }
    }
    return 0;
}

/* Solve the n x n system M x = b by Gaussian elimination with partial
 * pivoting (M, b copied).  Returns 0 or -1 on a zero pivot. */
static int gauss_solve(int n, const double *M, const double *b, double *x)
{
    double a[8][9];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) a[i][j] = M[i * n + j];
        a[i][n] = b[i];
    }
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(a[i][k]) > fabs(a[p][k])) p = i;
        if (a[p][k] == 0.0) return -1;
        if (p != k)
            for (int j = 0; j <= n; ++j) { double t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double f = a[i][k] / a[k][k];
            for (int j = k; j <= n; ++j) a[i][j] -= f * a[k][j];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = a[i][n];
        for (int j = i + 1; j < n; ++j) s -= a[i][j] * x[j];
        x[i] = s / a[i][i];
    }
    return 0;
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* ------------------------------------------------------------------------ */
/* mesh: vertices of the (mapped) hexahedral mesh at time t                  */
/* ------------------------------------------------------------------------ */

/* Mapped mesh of the accuracy and moving-mesh tests (Sec. 4): each
 * coordinate is shifted by amp * S(t) * prod_d sin(2 pi (xi_d - lo_d)/L_d);
 * on [0,2]^3 the sine argument is pi*xi as printed.  S(t) = 1 for the
 * static mapped mesh and sin(omega t) for the moving mesh. */
static double mesh_shape(const orc_cfg *c, const double *xi)
{
    double s = 1.0;
    for (int d = 0; d < 3; ++d) s *= sin(2.0 * M_PI * (xi[d] - c->lo[d]) / (c->hi[d] - c->lo[d]));
    return s;
}

static void mesh_vertex(const orc_cfg *c, int i, int j, int k, double t, double *x, double *xdot)
{
    int idx[3] = {i, j, k};
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = c->lo[d] + (c->hi[d] - c->lo[d]) * (double)idx[d] / (double)c->n[d];
    double disp = 0.0, vel = 0.0;
    if (c->mesh == 1) disp = c->amp * mesh_shape(c, xi);
    if (c->mesh == 2) {
        double s = mesh_shape(c, xi);
        disp = c->amp * sin(c->omega * t) * s;
        vel = c->amp * c->omega * cos(c->omega * t) * s;
    }
    for (int d = 0; d < 3; ++d) {
        x[d] = xi[d] + disp;
        if (xdot) xdot[d] = vel;
    }
}

/* padded cell / vertex indexing: cells -GH..n+GH-1, vertices -GH..n+GH */
typedef struct {
    int n[3];
    int cn[3];   /* padded cell extents  */
    int vn[3];   /* padded vertex extents */
    size_t ncell, nvert;
} orc_dims;

static orc_dims make_dims(const orc_cfg *c)
{
    orc_dims D;
    for (int d = 0; d < 3; ++d) {
        D.n[d] = c->n[d];
        D.cn[d] = c->n[d] + 2 * GH;
        D.vn[d] = c->n[d] + 2 * GH + 1;
    }
    D.ncell = (size_t)D.cn[0] * D.cn[1] * D.cn[2];
    D.nvert = (size_t)D.vn[0] * D.vn[1] * D.vn[2];
    return D;
}
static inline size_t cid(const orc_dims *D, int i, int j, int k)
{
    return ((size_t)(k + GH) * D->cn[1] + (size_t)(j + GH)) * D->cn[0] + (size_t)(i + GH);
}
static inline size_t vid(const orc_dims *D, int i, int j, int k)
{
    return ((size_t)(k + GH) * D->vn[1] + (size_t)(j + GH)) * D->vn[0] + (size_t)(i + GH);
}

/* 2-point Gauss-Legendre on [-1/2, 1/2]: nodes +-sqrt(3)/6, weights 1/2. */
static const double GNODE[2] = {-0.28867513459481288225, 0.28867513459481288225};

/* trilinear map of a hexahedron (Sec. 2): X = sum_i x_i psi_i with
 * psi = prod_d (1 + 2 s_d xi_d)/2, s_d = -1/+1 for the two vertex layers. */
static void trilinear(const double hv[2][2][2][3], const double *p, double *X, double J[3][3])
{
    for (int d = 0; d < 3; ++d) {
        X[d] = 0.0;
        for (int e = 0; e < 3; ++e) J[d][e] = 0.0;
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double s[3] = {2.0 * a - 1.0, 2.0 * b - 1.0, 2.0 * c - 1.0};
                double f[3], df[3];
                for (int e = 0; e < 3; ++e) {
                    f[e] = 0.5 * (1.0 + 2.0 * s[e] * p[e]);
                    df[e] = s[e];
                }
                double psi = f[0] * f[1] * f[2];
                double dpsi[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
                for (int d = 0; d < 3; ++d) {
                    X[d] += hv[a][b][c][d] * psi;
                    for (int e = 0; e < 3; ++e) J[d][e] += hv[a][b][c][d] * dpsi[e];
                }
            }
}

static double det3(double J[3][3])
{
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* per-cell geometry */
typedef struct {
    double vol;        /* |Omega| by 2x2x2 Gauss quadrature (Sec. 2)         */
    double cen[3];     /* centroid                                           */
    double h;          /* |Omega|^(1/3)                                      */
    double qx[8][3];   /* quadrature points                                  */
    double qw[8];      /* quadrature weights times |det J|                   */
} cell_geom;

typedef struct {
    orc_dims D;
    double *vx;        /* [nvert][3] vertex positions   */
    double *vv;        /* [nvert][3] vertex velocities  */
} orc_geom;

static void cell_vertices(const orc_geom *G, int i, int j, int k, double hv[2][2][2][3])
{
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                for (int d = 0; d < 3; ++d)
                    hv[a][b][c][d] = G->vx[vid(&G->D, i + a, j + b, k + c) * 3 + d];
}

/* volume, centroid and quadrature points of cell (i,j,k) by the 2x2x2
 * Gauss rule on its trilinear map (Sec. 2) */
static void cell_geometry(const orc_geom *G, int i, int j, int k, cell_geom *cg)
{
    double hv[2][2][2][3];
    cell_vertices(G, i, j, k, hv);
    double vol = 0.0, m1[3] = {0, 0, 0};
    int q = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc, ++q) {
                double p[3] = {GNODE[a], GNODE[b], GNODE[cc]}, X[3], J[3][3];
                trilinear(hv, p, X, J);
                double w = 0.125 * fabs(det3(J));
                cg->qw[q] = w;
                for (int d = 0; d < 3; ++d) cg->qx[q][d] = X[d];
                vol += w;
                for (int d = 0; d < 3; ++d) m1[d] += w * X[d];
            }
    cg->vol = vol;
    for (int d = 0; d < 3; ++d) cg->cen[d] = m1[d] / vol;
    cg->h = cbrt(vol);
}

static int geom_build(const orc_cfg *c, double t, orc_geom *G)
{
    G->D = make_dims(c);
    const orc_dims *D = &G->D;
    G->vx = (double *)malloc(D->nvert * 3 * sizeof(double));
    G->vv = (double *)malloc(D->nvert * 3 * sizeof(double));
    if (!G->vx || !G->vv) return -1;
    for (int k = -GH; k <= c->n[2] + GH; ++k)
        for (int j = -GH; j <= c->n[1] + GH; ++j)
            for (int i = -GH; i <= c->n[0] + GH; ++i) {
                size_t v = vid(D, i, j, k);
                mesh_vertex(c, i, j, k, t, &G->vx[v * 3], &G->vv[v * 3]);
            }
    return 0;
}

static void geom_free(orc_geom *G)
{
    free(G->vx); free(G->vv);
    G->vx = G->vv = NULL;
}

/* ------------------------------------------------------------------------ */
/* ghost cells                                                               */
/* ------------------------------------------------------------------------ */

/* Copy the interior state into the padded array and fill GH ghost layers.
 * Periodic boundaries wrap; reflective ("symmetric") boundaries mirror the
 * cell order and negate the momentum normal to that boundary; non-reflecting
 * (outflow) boundaries repeat the boundary cell in every ghost layer
 * (zero-gradient extrapolation, the reading of the non-reflecting condition
 * of the Riemann problems of Sec. 4).  Edge and corner ghosts take every
 * applicable wrap, mirror or repeat, since the big stencil reaches the edge
 * neighbours. */
static int fill_ghosts(const orc_cfg *c, const orc_dims *D, const double *q, double *Qp)
{
    /* a mirror reaches GH cells into the grid */
    for (int d = 0; d < 3; ++d)
        if (c->n[d] < GH && (c->bc[2 * d] == 1 || c->bc[2 * d + 1] == 1)) return -1;
    size_t ncint = (size_t)c->n[0] * c->n[1] * c->n[2];
    for (int k = -GH; k < c->n[2] + GH; ++k)
        for (int j = -GH; j < c->n[1] + GH; ++j)
            for (int i = -GH; i < c->n[0] + GH; ++i) {
                int idx[3] = {i, j, k}, src[3], flip[3] = {0, 0, 0};
                for (int d = 0; d < 3; ++d) {
                    int n = c->n[d], s = idx[d];
                    if (s < 0) {
                        if (c->bc[2 * d] == 0) s = ((s % n) + n) % n;
                        else if (c->bc[2 * d] == 2) s = 0;
                        else { s = -1 - s; flip[d] = 1; }
                    } else if (s >= n) {
                        if (c->bc[2 * d + 1] == 0) s = s % n;
                        else if (c->bc[2 * d + 1] == 2) s = n - 1;
                        else { s = 2 * n - 1 - s; flip[d] = 1; }
                    }
                    src[d] = s;
                }
                size_t from = ((size_t)src[2] * c->n[1] + src[1]) * c->n[0] + src[0];
                size_t to = cid(D, i, j, k);
                for (int v = 0; v < NV; ++v) {
                    double val = q[(size_t)v * ncint + from];
                    if (v >= 1 && v <= 3 && flip[v - 1]) val = -val;
                    Qp[(size_t)v * D->ncell + to] = val;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* WENO-AO reconstruction (Sec. 2)                                           */
/* ------------------------------------------------------------------------ */

/* The nine monomials x^n1 y^n2 z^n3 with 1 <= |n| <= 2 of eq. (qua-def). */
static const int MONO[9][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* D^l of the monomial X^n at X (scaled coordinates) */
static double dmono(const int *n, const int *l, const double *X)
{
    double r = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (l[d] > n[d]) return 0.0;
        for (int f = 0; f < l[d]; ++f) r *= (double)(n[d] - f);
        r *= ipow(X[d], n[d] - l[d]);
    }
    return r;
}

/* The reconstruction of one cell.  All polynomials are written in the
 * scaled coordinates X = (x - centroid)/h, h = |Omega|^(1/3); the least
 * squares solution is the same function in any coordinates. */
typedef struct {
    double cen[3], h;
    double mean[9];          /* cell mean of each monomial                       */
    double Qc[NV];           /* cell average                                     */
    double coef[NV][9];      /* coefficients of the final polynomial P~          */
    double a[NV][9];         /* P0 coefficients                                  */
    double b[24][NV][3];     /* P_m coefficients                                 */
    double beta[NV][25];     /* smoothness indicators beta_0..beta_24            */
    double wbar[NV][25];     /* normalised nonlinear weights                     */
    int flag;                /* 1 when the positivity fallback fired             */
} cell_rec;

/* cell mean of X^n over cell g, in the frame (cen, h) */
static void cell_monomial_means(const cell_geom *g, const double *cen, double h, double *out)
{
    for (int m = 0; m < 9; ++m) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) {
            double X[3];
            for (int d = 0; d < 3; ++d) X[d] = (g->qx[q][d] - cen[d]) / h;
            s += g->qw[q] * ipow(X[0], MONO[m][0]) * ipow(X[1], MONO[m][1]) * ipow(X[2], MONO[m][2]);
        }
        out[m] = s / g->vol;
    }
}

/* The big stencil S: the 3x3x3 block minus the centre and the 8 corners;
 * S' (sprime) adds the six cells two steps away along the axes. */
static int big_stencil(int off[24][3], int sprime)
{
    int n = 0;
    for (int k0 = -1; k0 <= 1; ++k0)
        for (int j0 = -1; j0 <= 1; ++j0)
            for (int i0 = -1; i0 <= 1; ++i0) {
                if (i0 == 0 && j0 == 0 && k0 == 0) continue;
                if (i0 * j0 * k0 == 1 || i0 * j0 * k0 == -1) continue;
                off[n][0] = i0; off[n][1] = j0; off[n][2] = k0;
                ++n;
            }
    if (sprime)
        for (int d = 0; d < 3; ++d)
            for (int sg = -2; sg <= 2; sg += 4) {
                off[n][0] = off[n][1] = off[n][2] = 0;
                off[n][d] = sg;
                ++n;
            }
    return n;
}

/* The 24 sub-stencils.  Reading of the printed S1..S8 (the printed S4 and
 * S8 mix quadrants): S = {c, s_a e_a, s_b e_b, s_a e_a + s_b e_b, s_c e_c}
 * for the plane (a,b) with out-of-plane axis c, signs (s_a, s_b, s_c) in
 * the printed order (+++), (-++), (+-+), (--+), (++-), (-+-), (+--), (---),
 * for the planes xy, yz, zx in turn ("symmetrically"). */
/* The 8 sub-stencils of S' (sprime): the centre and one face neighbour along
 * each axis, {s_x e_x, s_y e_y, s_z e_z}, signs in the printed order S'_1..S'_8:
 * (+++), (-++), (+-+), (--+), (++-), (-+-), (+--), (---).  Reading: the
 * printed S'_4 and S'_8 repeat S'_2 and S'_6; they are read as the two
 * remaining octants (--+) and (---).  Returns the number of sub-stencils
 * and sets the cells per sub-stencil (besides the centre) in *nrow. */
static int sub_stencils_sel(int off[24][4][3], int *nrow, int sprime);

static void sub_stencils(int off[24][4][3])
{
    static const int SG[8][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {-1, -1, 1},
                                 {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    static const int PL[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
    int m = 0;
    for (int p = 0; p < 3; ++p)
        for (int s = 0; s < 8; ++s, ++m) {
            int a = PL[p][0], b = PL[p][1], cc = PL[p][2];
            for (int r = 0; r < 4; ++r)
                for (int d = 0; d < 3; ++d) off[m][r][d] = 0;
            off[m][0][a] = SG[s][0];
            off[m][1][b] = SG[s][1];
            off[m][2][a] = SG[s][0]; off[m][2][b] = SG[s][1];
            off[m][3][cc] = SG[s][2];
        }
}

static int sub_stencils_sel(int off[24][4][3], int *nrow, int sprime)
{
    if (!sprime) {
        sub_stencils(off);
        *nrow = 4;
        return 24;
    }
    static const int SG[8][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {-1, -1, 1},
                                 {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    for (int m = 0; m < 8; ++m)
        for (int r = 0; r < 3; ++r) {
            for (int d = 0; d < 3; ++d) off[m][r][d] = 0;
            off[m][r][r] = SG[m][r];
        }
    *nrow = 3;
    return 8;
}

/* the 24 face Gauss points of a cell (6 faces x 2 x 2) in physical space */
static void cell_face_gauss_points(const orc_geom *G, int i, int j, int k, double xg[24][3])
{
    double hv[2][2][2][3];
    cell_vertices(G, i, j, k, hv);
    int q = 0;
    for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
            int a = (d + 1) % 3, b = (d + 2) % 3;
            for (int ga = 0; ga < 2; ++ga)
                for (int gb = 0; gb < 2; ++gb, ++q) {
                    double p[3], X[3], J[3][3];
                    p[d] = side ? 0.5 : -0.5;
                    p[a] = GNODE[ga];
                    p[b] = GNODE[gb];
                    trilinear(hv, p, X, J);
                    for (int e = 0; e < 3; ++e) xg[q][e] = X[e];
                }
        }
}

static double pressure_of(const orc_cfg *c, const double *W)
{
    return (c->gamma - 1.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0]);
}

/* value of a polynomial Qc + sum coef_n (X^n - mean_n) at physical x */
static double poly_value(const cell_rec *r, const double *coef, double qc, int nterm, const double *x)
{
    double X[3];
    for (int d = 0; d < 3; ++d) X[d] = (x[d] - r->cen[d]) / r->h;
    double v = qc;
    for (int m = 0; m < nterm; ++m)
        v += coef[m] * (ipow(X[0], MONO[m][0]) * ipow(X[1], MONO[m][1]) * ipow(X[2], MONO[m][2]) - r->mean[m]);
    return v;
}

/* Reconstruction of cell (i,j,k).  With P (5x5, row-major) the data are
 * the projected variables P Q of every cell of the stencil (the
 * characteristic variables of Sec. 4, P = R^{-1}); the polynomials are then
 * built, weighted and combined per projected variable and mapped back with
 * Rb (= R) before the positivity check, so that r holds conservative
 * polynomials and the indicators and weights of the projected ones. */
static void reconstruct_cell_proj(const orc_cfg *c, const orc_geom *G, const double *Qp, int i, int j, int k,
                                  const double *P, const double *Rb, cell_rec *r);

static void reconstruct_cell(const orc_cfg *c, const orc_geom *G, const double *Qp, int i, int j, int k, cell_rec *r)
{
    reconstruct_cell_proj(c, G, Qp, i, j, k, NULL, NULL, r);
}

/* value of variable v of cell id, projected by P when given */
static double data_value(const orc_dims *D, const double *Qp, const double *P, int v, size_t id)
{
    if (!P) return Qp[(size_t)v * D->ncell + id];
    double s = 0.0;
    for (int u = 0; u < NV; ++u) s += P[v * NV + u] * Qp[(size_t)u * D->ncell + id];
    return s;
}

static void reconstruct_cell_proj(const orc_cfg *c, const orc_geom *G, const double *Qp, int i, int j, int k,
                                  const double *P, const double *Rb, cell_rec *r)
{
    const orc_dims *D = &G->D;
    /* geometry of the cells of the big stencil around the cell: the 3x3x3
     * block without its corners, and for S' the axis cells two steps away */
    static cell_geom zero_geom;
    cell_geom blk[5][5][5];
    for (int c2 = -2; c2 <= 2; ++c2)
        for (int b2 = -2; b2 <= 2; ++b2)
            for (int a2 = -2; a2 <= 2; ++a2) {
                const int in3 = abs(a2) <= 1 && abs(b2) <= 1 && abs(c2) <= 1 && a2 * b2 * c2 == 0;
                const int axis2 = c->stencil && abs(a2) + abs(b2) + abs(c2) == 2 &&
                                  (abs(a2) == 2 || abs(b2) == 2 || abs(c2) == 2);
                if (in3 || axis2) cell_geometry(G, i + a2, j + b2, k + c2, &blk[c2 + 2][b2 + 2][a2 + 2]);
                else blk[c2 + 2][b2 + 2][a2 + 2] = zero_geom;
            }
#define BLK(o0, o1, o2) (&blk[(o2) + 2][(o1) + 2][(o0) + 2])
    const cell_geom *gc = BLK(0, 0, 0);
    for (int d = 0; d < 3; ++d) r->cen[d] = gc->cen[d];
    r->h = gc->h;
    cell_monomial_means(gc, r->cen, r->h, r->mean);
    for (int v = 0; v < NV; ++v) r->Qc[v] = data_value(D, Qp, P, v, cid(D, i, j, k));

    /* P0: least squares over the 18 neighbours of the big stencil; the
     * centre constraint holds exactly because every p_n has zero mean. */
    int off[24][3];
    int ns = big_stencil(off, c->stencil);
    double A[24 * 9], B[24 * NV], X[9 * NV];
    for (int s = 0; s < ns; ++s) {
        int ii = i + off[s][0], jj = j + off[s][1], kk = k + off[s][2];
        double mn[9];
        cell_monomial_means(BLK(off[s][0], off[s][1], off[s][2]), r->cen, r->h, mn);
        for (int m = 0; m < 9; ++m) A[s * 9 + m] = mn[m] - r->mean[m];
        for (int v = 0; v < NV; ++v) B[s * NV + v] = data_value(D, Qp, P, v, cid(D, ii, jj, kk)) - r->Qc[v];
    }
    lsq_householder(ns, 9, A, NV, B, X);
    for (int v = 0; v < NV; ++v)
        for (int m = 0; m < 9; ++m) r->a[v][m] = X[m * NV + v];

    /* P_m, m = 1..nsub: linear least squares over the neighbours of S_m
     * (4 for S, 3 for S', where the system is square) */
    int so[24][4][3], nrow;
    const int nsub = sub_stencils_sel(so, &nrow, c->stencil);
    for (int s = 0; s < nsub; ++s) {
        double As[4 * 3], Bs[4 * NV], Xs[3 * NV];
        for (int rr = 0; rr < nrow; ++rr) {
            int ii = i + so[s][rr][0], jj = j + so[s][rr][1], kk = k + so[s][rr][2];
            double mn[9];
            cell_monomial_means(BLK(so[s][rr][0], so[s][rr][1], so[s][rr][2]), r->cen, r->h, mn);
            for (int m = 0; m < 3; ++m) As[rr * 3 + m] = mn[m] - r->mean[m];
            for (int v = 0; v < NV; ++v) Bs[rr * NV + v] = data_value(D, Qp, P, v, cid(D, ii, jj, kk)) - r->Qc[v];
        }
        lsq_householder(nrow, 3, As, NV, Bs, Xs);
        for (int v = 0; v < NV; ++v)
            for (int m = 0; m < 3; ++m) r->b[s][v][m] = Xs[m * NV + v];
    }

    /* linear weights: gamma_0 = 1 - nsub Gamma, gamma_m = Gamma (reading for
     * S': the same Gamma for each of its 8 sub-stencils) */
    double gam[25];
    gam[0] = 1.0 - nsub * c->Gamma_lin;
    for (int s = 1; s <= nsub; ++s) gam[s] = c->Gamma_lin;

    /* multi-indices l with 1 <= |l| <= 2, each counted once (Reading) */
    static const int LIDX[9][3] = {
        {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};

    for (int v = 0; v < NV; ++v) {
        /* smoothness indicators, eq. (indicator), integrals by the cell's
         * 2x2x2 Gauss rule in physical coordinates */
        double beta[25];
        for (int s = 0; s <= nsub; ++s) {
            int nl = (s == 0) ? 9 : 3;
            int nt = (s == 0) ? 9 : 3;
            const double *cf = (s == 0) ? r->a[v] : r->b[s - 1][v];
            double bsum = 0.0;
            for (int l = 0; l < nl; ++l) {
                int ord = LIDX[l][0] + LIDX[l][1] + LIDX[l][2];
                double integral = 0.0;
                for (int q = 0; q < 8; ++q) {
                    double Xq[3];
                    for (int d = 0; d < 3; ++d) Xq[d] = (gc->qx[q][d] - r->cen[d]) / r->h;
                    double dv = 0.0;
                    for (int m = 0; m < nt; ++m) dv += cf[m] * dmono(MONO[m], LIDX[l], Xq);
                    dv /= ipow(r->h, ord); /* physical derivative */
                    integral += gc->qw[q] * dv * dv;
                }
                bsum += pow(gc->vol, 2.0 * ord / 3.0 - 1.0) * integral;
            }
            beta[s] = bsum;
        }
        /* global indicator, eq. (para) */
        double tau = 0.0;
        for (int s = 1; s <= nsub; ++s) tau += fabs(beta[0] - beta[s]) / nsub;
        /* nonlinear weights, eq. (nonlinear) */
        double w[25], wsum = 0.0;
        for (int s = 0; s <= nsub; ++s) {
            double ratio = tau / (beta[s] + c->weno_eps);
            w[s] = gam[s] * (1.0 + (c->weno_pow == 2 ? ratio * ratio : ratio));
            wsum += w[s];
        }
        double wb[25];
        for (int s = 0; s <= nsub; ++s) wb[s] = w[s] / wsum;
        for (int s = 0; s <= 24; ++s) {
            r->beta[v][s] = s <= nsub ? beta[s] : 0.0;
            r->wbar[v][s] = s <= nsub ? wb[s] : 0.0;
        }
        /* P~ = wb0 (P0/g0 - sum g_m/g0 P_m) + sum wb_m P_m */
        for (int m = 0; m < 9; ++m) r->coef[v][m] = (wb[0] / gam[0]) * r->a[v][m];
        for (int s = 1; s <= nsub; ++s)
            for (int m = 0; m < 3; ++m)
                r->coef[v][m] += (wb[s] - wb[0] * gam[s] / gam[0]) * r->b[s - 1][v][m];
    }

    /* back to the conservative variables: every polynomial is linear in
     * the data, so the map acts on the averages and coefficients */
    if (P) {
        double t0[NV], t9[NV][9], ta[NV][9], tb[24][NV][3];
        for (int v = 0; v < NV; ++v) {
            t0[v] = 0.0;
            for (int m = 0; m < 9; ++m) t9[v][m] = ta[v][m] = 0.0;
            for (int s2 = 0; s2 < 24; ++s2)
                for (int m = 0; m < 3; ++m) tb[s2][v][m] = 0.0;
            for (int u = 0; u < NV; ++u) {
                double rv = Rb[v * NV + u];
                t0[v] += rv * r->Qc[u];
                for (int m = 0; m < 9; ++m) {
                    t9[v][m] += rv * r->coef[u][m];
                    ta[v][m] += rv * r->a[u][m];
                }
                for (int s2 = 0; s2 < 24; ++s2)
                    for (int m = 0; m < 3; ++m) tb[s2][v][m] += rv * r->b[s2][u][m];
            }
        }
        memcpy(r->coef, t9, sizeof t9);
        memcpy(r->a, ta, sizeof ta);
        memcpy(r->b, tb, sizeof tb);
        /* the cell average itself, exactly as stored */
        for (int v = 0; v < NV; ++v) r->Qc[v] = Qp[(size_t)v * D->ncell + cid(D, i, j, k)];
        (void)t0;
    }

    /* positivity fallback (Sec. 4): if rho or p of any P_m, m = 0..24, is
     * negative at any of the cell's 24 Gauss points, drop to first order. */
    r->flag = 0;
    if (c->limiter) {
        double xg[24][3];
        cell_face_gauss_points(G, i, j, k, xg);
        for (int s = 0; s <= nsub && !r->flag; ++s)
            for (int g = 0; g < 24 && !r->flag; ++g) {
                double W[NV];
                for (int v = 0; v < NV; ++v)
                    W[v] = (s == 0) ? poly_value(r, r->a[v], r->Qc[v], 9, xg[g])
                                    : poly_value(r, r->b[s - 1][v], r->Qc[v], 3, xg[g]);
                if (W[0] < 0.0 || pressure_of(c, W) < 0.0) r->flag = 1;
            }
        if (r->flag)
            for (int v = 0; v < NV; ++v)
                for (int m = 0; m < 9; ++m) r->coef[v][m] = 0.0;
    }
#undef BLK
}

/* what the flux needs of a reconstructed cell */
typedef struct {
    double cen[3], h;
    double mean[9];
    double Qc[NV];
    double coef[NV][9];
    int flag;
} slim_rec;

static void slim_from(const cell_rec *r, slim_rec *o)
{
    for (int d = 0; d < 3; ++d) o->cen[d] = r->cen[d];
    o->h = r->h;
    memcpy(o->mean, r->mean, sizeof o->mean);
    memcpy(o->Qc, r->Qc, sizeof o->Qc);
    memcpy(o->coef, r->coef, sizeof o->coef);
    o->flag = r->flag;
}

/* value and physical gradient of P~ at x */
static void rec_eval(const slim_rec *r, const double *x, double W[NV], double dW[NV][3])
{
    double X[3];
    for (int d = 0; d < 3; ++d) X[d] = (x[d] - r->cen[d]) / r->h;
    static const int L1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int L0[3] = {0, 0, 0};
    for (int v = 0; v < NV; ++v) {
        W[v] = r->Qc[v];
        for (int e = 0; e < 3; ++e) dW[v][e] = 0.0;
        for (int m = 0; m < 9; ++m) {
            W[v] += r->coef[v][m] * (dmono(MONO[m], L0, X) - r->mean[m]);
            for (int e = 0; e < 3; ++e) dW[v][e] += r->coef[v][m] * dmono(MONO[m], L1[e], X) / r->h;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* velocity-space moments of a Maxwellian (Sec. 3)                           */
/* ------------------------------------------------------------------------ */

/* One-dimensional moments <c^k> of sqrt(lambda/pi) exp(-lambda (u-U)^2)
 * over u in the whole line (side 0), u > 0 (side +1) or u < 0 (side -1),
 * written in the peculiar velocity c = u - U.  Whole line: (k-1)!!/(2 lambda)^(k/2)
 * for even k.  Half line u > 0 (c > -U): I0 = erfc(-sqrt(lambda) U)/2,
 * I1 = exp(-lambda U^2)/(2 sqrt(pi lambda)), and by parts
 * I_k = (k-1)/(2 lambda) I_{k-2} + (-U)^(k-1) exp(-lambda U^2)/(2 sqrt(pi lambda)). */
#define MAXE 10
typedef struct { double m[MAXE + 1]; } mom1d;

static void central_moments(double U, double lam, int side, double *I)
{
    double e = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
    if (side == 0) {
        I[0] = 1.0; I[1] = 0.0;
        for (int k = 2; k <= MAXE; ++k) I[k] = (k - 1) / (2.0 * lam) * I[k - 2];
        return;
    }
    /* u > 0: c from -U to inf; u < 0: c from -inf to -U */
    double lower = -U;
    if (side > 0) {
        I[0] = 0.5 * erfc(sqrt(lam) * lower);
        I[1] = e;
        for (int k = 2; k <= MAXE; ++k) I[k] = (k - 1) / (2.0 * lam) * I[k - 2] + ipow(lower, k - 1) * e;
    } else {
        I[0] = 0.5 * erfc(-sqrt(lam) * lower);
        I[1] = -e;
        for (int k = 2; k <= MAXE; ++k) I[k] = (k - 1) / (2.0 * lam) * I[k - 2] - ipow(lower, k - 1) * e;
    }
}

/* <u^n> = sum_k C(n,k) U^(n-k) <c^k> */
static void moments_1d(double U, double lam, int side, mom1d *M)
{
    double I[MAXE + 1];
    central_moments(U, lam, side, I);
    for (int n = 0; n <= MAXE; ++n) {
        double s = 0.0, binom = 1.0;
        for (int k = 0; k <= n; ++k) {
            s += binom * ipow(U, n - k) * I[k];
            binom = binom * (double)(n - k) / (double)(k + 1);
        }
        M->m[n] = s;
    }
}

/* Maxwellian of one state: primitive variables and moment tables */
typedef struct {
    double rho, U[3], lam;
    mom1d full[3];     /* <u^n>, <v^n>, <w^n> over all velocities           */
    mom1d half[3];     /* same with u restricted to one half-space          */
    double xi[4];      /* <xi^(2d)> of the K internal degrees of freedom    */
} maxwellian;

static void make_maxwellian(const orc_cfg *c, const double *W, int side, maxwellian *g)
{
    double K = (5.0 - 3.0 * c->gamma) / (c->gamma - 1.0);
    g->rho = W[0];
    for (int d = 0; d < 3; ++d) g->U[d] = W[1 + d] / W[0];
    double kin = 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0];
    /* rho E = rho |U|^2/2 + (K+3) rho/(4 lambda) */
    g->lam = (K + 3.0) * W[0] / (4.0 * (W[4] - kin));
    for (int d = 0; d < 3; ++d) {
        moments_1d(g->U[d], g->lam, 0, &g->full[d]);
        moments_1d(g->U[d], g->lam, d == 0 ? side : 0, &g->half[d]);
    }
    /* internal DOF: isotropic Gaussian in K dimensions */
    g->xi[0] = 1.0;
    g->xi[1] = K / (2.0 * g->lam);
    g->xi[2] = K * (K + 2.0) / (4.0 * g->lam * g->lam);
    g->xi[3] = K * (K + 2.0) * (K + 4.0) / (8.0 * g->lam * g->lam * g->lam);
}

/* sparse polynomials in (u, v, w, xi^2); exponents of u, v, w up to 8 and
 * of xi^2 up to 3 cover every product formed below */
#define MAXT 700
#define EU 9
#define EX 4
typedef struct { double c; unsigned char e[4]; } mono_t;
typedef struct { int n; mono_t t[MAXT]; } poly_t;

static void poly_zero(poly_t *p) { p->n = 0; }
static void poly_add_term(poly_t *p, double c, int a, int b, int cc, int d)
{
    if (c == 0.0) return;
    for (int i = 0; i < p->n; ++i)
        if (p->t[i].e[0] == a && p->t[i].e[1] == b && p->t[i].e[2] == cc && p->t[i].e[3] == d) {
            p->t[i].c += c;
            return;
        }
    if (p->n >= MAXT || a >= EU || b >= EU || cc >= EU || d >= EX) abort();
    p->t[p->n].c = c;
    p->t[p->n].e[0] = (unsigned char)a; p->t[p->n].e[1] = (unsigned char)b;
    p->t[p->n].e[2] = (unsigned char)cc; p->t[p->n].e[3] = (unsigned char)d;
    p->n++;
}

/* psi_i: (1, u, v, w, (u^2+v^2+w^2+xi^2)/2) */
static void poly_psi(int i, poly_t *p)
{
    poly_zero(p);
    switch (i) {
    case 0: poly_add_term(p, 1.0, 0, 0, 0, 0); break;
    case 1: poly_add_term(p, 1.0, 1, 0, 0, 0); break;
    case 2: poly_add_term(p, 1.0, 0, 1, 0, 0); break;
    case 3: poly_add_term(p, 1.0, 0, 0, 1, 0); break;
    default:
        poly_add_term(p, 0.5, 2, 0, 0, 0); poly_add_term(p, 0.5, 0, 2, 0, 0);
        poly_add_term(p, 0.5, 0, 0, 2, 0); poly_add_term(p, 0.5, 0, 0, 0, 1);
    }
}

/* a . psi for a coefficient vector a[5] */
static void poly_apsi(const double *a, poly_t *p)
{
    poly_zero(p);
    for (int i = 0; i < NV; ++i) {
        poly_t q;
        poly_psi(i, &q);
        for (int t = 0; t < q.n; ++t)
            poly_add_term(p, a[i] * q.t[t].c, q.t[t].e[0], q.t[t].e[1], q.t[t].e[2], q.t[t].e[3]);
    }
}

static void poly_mul(const poly_t *a, const poly_t *b, poly_t *out)
{
    /* dense accumulator over the exponent box, compacted in first-touch order */
    static __thread double acc[EU * EU * EU * EX];
    static __thread int used[EU * EU * EU * EX];
    static __thread int touched[EU * EU * EU * EX];
    int nt = 0;
    for (int i = 0; i < a->n; ++i)
        for (int j = 0; j < b->n; ++j) {
            int e0 = a->t[i].e[0] + b->t[j].e[0], e1 = a->t[i].e[1] + b->t[j].e[1];
            int e2 = a->t[i].e[2] + b->t[j].e[2], e3 = a->t[i].e[3] + b->t[j].e[3];
            if (e0 >= EU || e1 >= EU || e2 >= EU || e3 >= EX) abort();
            int id = ((e0 * EU + e1) * EU + e2) * EX + e3;
            if (!used[id]) { used[id] = 1; acc[id] = 0.0; touched[nt++] = id; }
            acc[id] += a->t[i].c * b->t[j].c;
        }
    poly_t r;
    r.n = 0;
    for (int k = 0; k < nt; ++k) {
        int id = touched[k];
        used[id] = 0;
        if (acc[id] == 0.0) continue;
        if (r.n >= MAXT) abort();
        r.t[r.n].c = acc[id];
        r.t[r.n].e[3] = (unsigned char)(id % EX);
        r.t[r.n].e[2] = (unsigned char)((id / EX) % EU);
        r.t[r.n].e[1] = (unsigned char)((id / (EX * EU)) % EU);
        r.t[r.n].e[0] = (unsigned char)(id / (EX * EU * EU));
        r.n++;
    }
    *out = r;
}

/* integral of poly * g over the chosen velocity domain, g normalised so
 * that its zeroth moment is rho (half-space tables when half != 0) */
static double integrate(const maxwellian *g, int half, const poly_t *p)
{
    const mom1d *T = half ? g->half : g->full;
    double s = 0.0;
    for (int t = 0; t < p->n; ++t) {
        const unsigned char *e = p->t[t].e;
        s += p->t[t].c * T[0].m[e[0]] * T[1].m[e[1]] * T[2].m[e[2]] * g->xi[e[3]];
    }
    return g->rho * s;
}

/* 5-vector int w(u) psi g dXi for a weight polynomial w */
static void integrate_psi(const maxwellian *g, int half, const poly_t *w, double *out)
{
    for (int i = 0; i < NV; ++i) {
        poly_t pi, prod;
        poly_psi(i, &pi);
        poly_mul(w, &pi, &prod);
        out[i] = integrate(g, half, &prod);
    }
}

/* the moment matrix int psi psi^T g dXi */
static void moment_matrix(const maxwellian *g, double *M)
{
    for (int i = 0; i < NV; ++i)
        for (int j = 0; j < NV; ++j) {
            poly_t pi, pj, prod;
            poly_psi(i, &pi);
            poly_psi(j, &pj);
            poly_mul(&pi, &pj, &prod);
            M[i * NV + j] = integrate(g, 0, &prod);
        }
}

/* sum_i u_i (a_i . psi): the spatial part of the first-order expansion */
static void poly_a_dot_u(const double a[3][NV], poly_t *p)
{
    poly_zero(p);
    for (int d = 0; d < 3; ++d) {
        poly_t ap, ud, prod;
        poly_apsi(a[d], &ap);
        poly_zero(&ud);
        poly_add_term(&ud, 1.0, d == 0, d == 1, d == 2, 0);
        poly_mul(&ap, &ud, &prod);
        for (int t = 0; t < prod.n; ++t)
            poly_add_term(p, prod.t[t].c, prod.t[t].e[0], prod.t[t].e[1], prod.t[t].e[2], prod.t[t].e[3]);
    }
}

/* Slopes of one Maxwellian: a_i = M^-1 dW/dn_i, and the time slope A from
 * <a_1 u + a_2 v + a_3 w + A> = 0, i.e. M A = -int (a.u) psi g. */
static int micro_slopes(const maxwellian *g, const double dW[3][NV], double a[3][NV], double *A)
{
    double M[NV * NV];
    moment_matrix(g, M);
    for (int d = 0; d < 3; ++d)
        if (gauss_solve(NV, M, dW[d], a[d])) return -1;
    poly_t au;
    poly_a_dot_u(a, &au);
    double rhs[NV];
    integrate_psi(g, 0, &au, rhs);
    for (int i = 0; i < NV; ++i) rhs[i] = -rhs[i];
    return gauss_solve(NV, M, rhs, A);
}

/* Exact time integrals over [0, delta] of the factors of eq. (flux):
 * q[0]: 1 - e^{-t/tau}                   q[3]: e^{-t/tau}
 * q[1]: (t + tau) e^{-t/tau} - tau       q[4]: -(t + tau) e^{-t/tau}
 * q[2]: t - tau + tau e^{-t/tau}         q[5]: -tau e^{-t/tau}          */
void orc_time_integrals(double delta, double tau, double *q)
{
    double e = exp(-delta / tau);
    q[0] = delta - tau * (1.0 - e);
    q[1] = -tau * delta * (1.0 + e) + 2.0 * tau * tau * (1.0 - e);
    q[2] = 0.5 * delta * delta - tau * delta + tau * tau * (1.0 - e);
    q[3] = tau * (1.0 - e);
    q[4] = tau * delta * e - 2.0 * tau * tau * (1.0 - e);
    q[5] = -tau * tau * (1.0 - e);
}

/* ------------------------------------------------------------------------ */
/* gas-kinetic flux at one Gauss point (Sec. 3)                              */
/* ------------------------------------------------------------------------ */

/* Inputs, all in the local frame (n_x, n_y, n_z) of the Gauss point, with
 * n_x pointing from the left cell to the right cell:
 *   in[0..4]   W_l (conservative),  in[5..19]  dW_l/dn_x, dW_l/dn_y, dW_l/dn_z
 *   in[20..24] W_r,                 in[25..39] dW_r/dn_x, dW_r/dn_y, dW_r/dn_z
 *   ug[3]      grid velocity in the local frame (zero on a fixed mesh)
 * Outputs: F[5] and dF[5], the flux through the face per unit area and its
 * time derivative, in the same frame.
 *
 * On a moving mesh (Remark 2) the flux is computed in the frame moving with
 * the grid: the states are shifted by the grid velocity, the standard flux
 * is taken, and the moments are mapped back (u = u_rel + U_g).
 *
 * Reading: eq. (flux) pairs g_r with H(u) and g_l with 1-H(u), at odds with
 * the half-space split of Q0 printed right below it; the split of Q0 is
 * followed (g_l carries u > 0).
 * Reading (Prandtl number; the paper is silent): the energy flux takes the
 * usual correction F_E += (1/Pr - 1) q with q the time-integrated heat flux
 * about the velocity of g0, when mu > 0 and Pr != 1. */
int orc_point_flux(const orc_cfg *c, const double *in, const double *ug, double dt, double *F, double *dF)
{
    double W[2][NV], dW[2][3][NV];
    for (int s = 0; s < 2; ++s)
        for (int v = 0; v < NV; ++v) {
            W[s][v] = in[s * 20 + v];
            for (int d = 0; d < 3; ++d) dW[s][d][v] = in[s * 20 + 5 + d * 5 + v];
        }
    double Ug[3] = {ug ? ug[0] : 0.0, ug ? ug[1] : 0.0, ug ? ug[2] : 0.0};
    double ug2 = Ug[0] * Ug[0] + Ug[1] * Ug[1] + Ug[2] * Ug[2];
    /* states relative to the grid */
    for (int s = 0; s < 2; ++s) {
        double Wa[NV];
        memcpy(Wa, W[s], sizeof Wa);
        W[s][4] = Wa[4] - (Ug[0] * Wa[1] + Ug[1] * Wa[2] + Ug[2] * Wa[3]) + 0.5 * ug2 * Wa[0];
        for (int d = 0; d < 3; ++d) W[s][1 + d] = Wa[1 + d] - Ug[d] * Wa[0];
        for (int e = 0; e < 3; ++e) {
            double da[NV];
            memcpy(da, dW[s][e], sizeof da);
            dW[s][e][4] = da[4] - (Ug[0] * da[1] + Ug[1] * da[2] + Ug[2] * da[3]) + 0.5 * ug2 * da[0];
            for (int d = 0; d < 3; ++d) dW[s][e][1 + d] = da[1 + d] - Ug[d] * da[0];
        }
    }

    /* g_l with the u > 0 half space, g_r with u < 0 */
    maxwellian g[2];
    make_maxwellian(c, W[0], +1, &g[0]);
    make_maxwellian(c, W[1], -1, &g[1]);
    double a[2][3][NV], A[2][NV];
    for (int s = 0; s < 2; ++s)
        if (micro_slopes(&g[s], dW[s], a[s], A[s])) return -1;

    /* equilibrium at the interface from the colliding half spaces */
    poly_t one;
    poly_zero(&one);
    poly_add_term(&one, 1.0, 0, 0, 0, 0);
    double W0[NV], dW0[3][NV];
    {
        double wl[NV], wr[NV];
        integrate_psi(&g[0], 1, &one, wl);
        integrate_psi(&g[1], 1, &one, wr);
        for (int v = 0; v < NV; ++v) W0[v] = wl[v] + wr[v];
        for (int d = 0; d < 3; ++d) {
            poly_t pl, pr;
            poly_apsi(a[0][d], &pl);
            poly_apsi(a[1][d], &pr);
            integrate_psi(&g[0], 1, &pl, wl);
            integrate_psi(&g[1], 1, &pr, wr);
            for (int v = 0; v < NV; ++v) dW0[d][v] = wl[v] + wr[v];
        }
    }
    maxwellian g0;
    make_maxwellian(c, W0, 0, &g0);
    double abar[3][NV], Abar[NV];
    if (micro_slopes(&g0, dW0, abar, Abar)) return -1;

    /* collision time (Sec. 4) */
    double pl = pressure_of(c, W[0]), pr = pressure_of(c, W[1]);
    double jump = fabs((pl - pr) / (pl + pr));
    double tau;
    /* viscosity at the interface: mu, or mu (T0/T_ref)^mu_pow with T0 = p0/rho0
     * = 1/(2 lam0) the temperature of g0 */
    double mu_eff = c->mu;
    if (c->mu_pow != 0.0) mu_eff = c->mu * pow(1.0 / (2.0 * g0.lam) / c->T_ref, c->mu_pow);
    if (c->mu > 0.0) tau = mu_eff / (g0.rho / (2.0 * g0.lam)) + c->tau_C * jump * dt;
    else tau = c->tau_eps * dt + c->tau_C * jump * dt;

    /* weight polynomials of the time-integrated distribution (kept on the
     * heap: they are too large for worker-thread stacks) */
    enum { P_U1, P_HEAT, P_CX, P_CS, P_TMP, P_CD, P_SQ, P_AU0, P_A0, P_AUL, P_AUR, P_AL, P_AR, P_W2, P_W3, P_COUNT };
    poly_t *P = (poly_t *)malloc(P_COUNT * sizeof(poly_t));
    if (!P) return -1;
    poly_zero(&P[P_U1]);
    poly_add_term(&P[P_U1], 1.0, 1, 0, 0, 0);
    /* heat-flux weight (u - U0)((u-U0)^2 + (v-V0)^2 + (w-W0)^2 + xi^2)/2 */
    poly_zero(&P[P_CX]);
    poly_add_term(&P[P_CX], 1.0, 1, 0, 0, 0);
    poly_add_term(&P[P_CX], -g0.U[0], 0, 0, 0, 0);
    poly_zero(&P[P_CS]);
    for (int d = 0; d < 3; ++d) {
        poly_zero(&P[P_CD]);
        poly_add_term(&P[P_CD], 1.0, d == 0, d == 1, d == 2, 0);
        poly_add_term(&P[P_CD], -g0.U[d], 0, 0, 0, 0);
        poly_mul(&P[P_CD], &P[P_CD], &P[P_SQ]);
        for (int t = 0; t < P[P_SQ].n; ++t)
            poly_add_term(&P[P_CS], P[P_SQ].t[t].c, P[P_SQ].t[t].e[0], P[P_SQ].t[t].e[1], P[P_SQ].t[t].e[2],
                          P[P_SQ].t[t].e[3]);
    }
    poly_add_term(&P[P_CS], 1.0, 0, 0, 0, 1);
    poly_mul(&P[P_CX], &P[P_CS], &P[P_TMP]);
    poly_zero(&P[P_HEAT]);
    for (int t = 0; t < P[P_TMP].n; ++t)
        poly_add_term(&P[P_HEAT], 0.5 * P[P_TMP].t[t].c, P[P_TMP].t[t].e[0], P[P_TMP].t[t].e[1], P[P_TMP].t[t].e[2],
                      P[P_TMP].t[t].e[3]);

    /* the pieces of eq. (flux) as weight polynomials */
    poly_a_dot_u(abar, &P[P_AU0]);
    poly_apsi(Abar, &P[P_A0]);
    poly_a_dot_u(a[0], &P[P_AUL]);
    poly_a_dot_u(a[1], &P[P_AUR]);
    poly_apsi(A[0], &P[P_AL]);
    poly_apsi(A[1], &P[P_AR]);

    int pr_fix = (c->mu > 0.0 && c->Pr != 1.0);
    double Fh[2][NV];
    const double deltas[2] = {dt, 0.5 * dt};
    for (int h = 0; h < 2; ++h) {
        double q[6];
        orc_time_integrals(deltas[h], tau, q);
        /* moments of u psi (and of the heat-flux weight) against every term */
        double acc[2][NV];
        for (int k = 0; k < 2; ++k) {
            double m1[NV], m2[NV], m3[NV];
            const poly_t *w = k ? &P[P_HEAT] : &P[P_U1];
            for (int v = 0; v < NV; ++v) acc[k][v] = 0.0;
            if (k == 1 && !pr_fix) continue;
            /* g0 terms */
            integrate_psi(&g0, 0, w, m1);
            poly_mul(w, &P[P_AU0], &P[P_W2]);
            integrate_psi(&g0, 0, &P[P_W2], m2);
            poly_mul(w, &P[P_A0], &P[P_W3]);
            integrate_psi(&g0, 0, &P[P_W3], m3);
            for (int v = 0; v < NV; ++v) acc[k][v] += q[0] * m1[v] + q[1] * m2[v] + q[2] * m3[v];
            /* half-space terms of the initial distribution */
            for (int s = 0; s < 2; ++s) {
                integrate_psi(&g[s], 1, w, m1);
                poly_mul(w, &P[s ? P_AUR : P_AUL], &P[P_W2]);
                integrate_psi(&g[s], 1, &P[P_W2], m2);
                poly_mul(w, &P[s ? P_AR : P_AL], &P[P_W3]);
                integrate_psi(&g[s], 1, &P[P_W3], m3);
                for (int v = 0; v < NV; ++v) acc[k][v] += q[3] * m1[v] + q[4] * m2[v] + q[5] * m3[v];
            }
        }
        for (int v = 0; v < NV; ++v) Fh[h][v] = acc[0][v];
        /* the heat-flux weight times psi_0 = 1 is the heat flux itself */
        if (pr_fix) Fh[h][4] += (1.0 / c->Pr - 1.0) * acc[1][0];
    }
    free(P);

    /* F dt + dF dt^2/2 = Fh(dt);  F dt/2 + dF dt^2/8 = Fh(dt/2) */
    double M2[4] = {dt, 0.5 * dt * dt, 0.5 * dt, 0.125 * dt * dt};
    double Fr[NV], dFr[NV];
    for (int v = 0; v < NV; ++v) {
        double rhs[2] = {Fh[0][v], Fh[1][v]}, x[2];
        if (gauss_solve(2, M2, rhs, x)) return -1;
        Fr[v] = x[0];
        dFr[v] = x[1];
    }
    /* back from the grid frame: u = u_rel + U_g */
    F[0] = Fr[0];
    dF[0] = dFr[0];
    for (int d = 0; d < 3; ++d) {
        F[1 + d] = Fr[1 + d] + Ug[d] * Fr[0];
        dF[1 + d] = dFr[1 + d] + Ug[d] * dFr[0];
    }
    F[4] = Fr[4] + Ug[0] * Fr[1] + Ug[1] * Fr[2] + Ug[2] * Fr[3] + 0.5 * ug2 * Fr[0];
    dF[4] = dFr[4] + Ug[0] * dFr[1] + Ug[1] * dFr[2] + Ug[2] * dFr[3] + 0.5 * ug2 * dFr[0];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the operator L and its time derivative (eq. finite)                      */
/* ------------------------------------------------------------------------ */

/* Face of axis d with index f (between cells f-1 and f along d) and
 * transverse indices (t1, t2): its bilinear map (eq. bilinear) is
 * parameterised by (eta_a, eta_b), a = d+1, b = d+2 (mod 3), so that for
 * d = x this is the printed (eta, zeta). */
static void face_vertices(const orc_geom *G, int d, int i, int j, int k, double fv[2][2][3])
{
    int a = (d + 1) % 3, b = (d + 2) % 3;
    for (int sa = 0; sa < 2; ++sa)
        for (int sb = 0; sb < 2; ++sb) {
            int o[3] = {0, 0, 0};
            o[a] = sa;
            o[b] = sb;
            size_t v = vid(&G->D, i + o[0], j + o[1], k + o[2]);
            for (int e = 0; e < 3; ++e) fv[sa][sb][e] = G->vx[v * 3 + e];
        }
}
static void face_vertex_velocity(const orc_geom *G, int d, int i, int j, int k, double fv[2][2][3])
{
    int a = (d + 1) % 3, b = (d + 2) % 3;
    for (int sa = 0; sa < 2; ++sa)
        for (int sb = 0; sb < 2; ++sb) {
            int o[3] = {0, 0, 0};
            o[a] = sa;
            o[b] = sb;
            size_t v = vid(&G->D, i + o[0], j + o[1], k + o[2]);
            for (int e = 0; e < 3; ++e) fv[sa][sb][e] = G->vv[v * 3 + e];
        }
}

/* invert a 3x3 matrix by Gauss-Jordan elimination */
static int inv3(const double *R, double *Ri)
{
    double e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int col = 0; col < 3; ++col) {
        double x[3];
        if (gauss_solve(3, R, e[col], x)) return -1;
        for (int row = 0; row < 3; ++row) Ri[row * 3 + col] = x[row];
    }
    return 0;
}

/* face flux integrated over the face (eq. flux-x), both time levels, in
 * the global frame, for the face whose left cell is (i,j,k)-e_d */
static int face_flux(const orc_cfg *c, const orc_geom *G, const slim_rec *rl, const slim_rec *rr,
                     int d, int i, int j, int k, double dt, double *FF, double *dFF)
{
    double fv[2][2][3], fu[2][2][3];
    face_vertices(G, d, i, j, k, fv);
    face_vertex_velocity(G, d, i, j, k, fu);
    for (int v = 0; v < NV; ++v) FF[v] = dFF[v] = 0.0;
    for (int ga = 0; ga < 2; ++ga)
        for (int gb = 0; gb < 2; ++gb) {
            double ea = GNODE[ga], eb = GNODE[gb];
            double X[3] = {0, 0, 0}, Xa[3] = {0, 0, 0}, Xb[3] = {0, 0, 0}, Vg[3] = {0, 0, 0};
            for (int sa = 0; sa < 2; ++sa)
                for (int sb = 0; sb < 2; ++sb) {
                    double qa = 2.0 * sa - 1.0, qb = 2.0 * sb - 1.0;
                    double phi = 0.25 * (1.0 + 2.0 * qa * ea) * (1.0 + 2.0 * qb * eb);
                    double pa = 0.5 * qa * (1.0 + 2.0 * qb * eb);
                    double pb = 0.5 * qb * (1.0 + 2.0 * qa * ea);
                    for (int e = 0; e < 3; ++e) {
                        X[e] += fv[sa][sb][e] * phi;
                        Xa[e] += fv[sa][sb][e] * pa;
                        Xb[e] += fv[sa][sb][e] * pb;
                        Vg[e] += fu[sa][sb][e] * phi;
                    }
                }
            double nrm[3], nx[3], ny[3], nz[3];
            cross3(Xa, Xb, nrm);
            double area = norm3(nrm);
            for (int e = 0; e < 3; ++e) nx[e] = nrm[e] / area;
            double lb = norm3(Xb);
            for (int e = 0; e < 3; ++e) nz[e] = Xb[e] / lb;
            cross3(nz, nx, ny);
            const double *fr[3] = {nx, ny, nz};

            /* reconstructed states and gradients on both sides */
            double in[40], Wl[NV], Wr[NV], dWl[NV][3], dWr[NV][3];
            rec_eval(rl, X, Wl, dWl);
            rec_eval(rr, X, Wr, dWr);
            for (int s = 0; s < 2; ++s) {
                const double *Wg = s ? Wr : Wl;
                double(*dWg)[3] = s ? dWr : dWl;
                double *o = in + 20 * s;
                o[0] = Wg[0];
                for (int m = 0; m < 3; ++m)
                    o[1 + m] = Wg[1] * fr[m][0] + Wg[2] * fr[m][1] + Wg[3] * fr[m][2];
                o[4] = Wg[4];
                for (int di = 0; di < 3; ++di) {
                    /* directional derivatives along n_di, momentum rotated */
                    double dd[NV];
                    for (int v = 0; v < NV; ++v)
                        dd[v] = dWg[v][0] * fr[di][0] + dWg[v][1] * fr[di][1] + dWg[v][2] * fr[di][2];
                    double *od = o + 5 + 5 * di;
                    od[0] = dd[0];
                    for (int m = 0; m < 3; ++m) od[1 + m] = dd[1] * fr[m][0] + dd[2] * fr[m][1] + dd[3] * fr[m][2];
                    od[4] = dd[4];
                }
            }
            double ugl[3];
            for (int m = 0; m < 3; ++m) ugl[m] = Vg[0] * fr[m][0] + Vg[1] * fr[m][1] + Vg[2] * fr[m][2];
            double Fl[NV], dFl[NV];
            if (orc_point_flux(c, in, ugl, dt, Fl, dFl)) return -1;

            /* back to the global frame with (a_ij), the inverse of the
             * matrix whose rows are n_x, n_y, n_z (eq. trans) */
            double R[9], Ri[9];
            for (int m = 0; m < 3; ++m)
                for (int e = 0; e < 3; ++e) R[m * 3 + e] = fr[m][e];
            if (inv3(R, Ri)) return -1;
            double Fg[NV], dFg[NV];
            Fg[0] = Fl[0];
            dFg[0] = dFl[0];
            Fg[4] = Fl[4];
            dFg[4] = dFl[4];
            for (int e = 0; e < 3; ++e) {
                Fg[1 + e] = Ri[e * 3 + 0] * Fl[1] + Ri[e * 3 + 1] * Fl[2] + Ri[e * 3 + 2] * Fl[3];
                dFg[1 + e] = Ri[e * 3 + 0] * dFl[1] + Ri[e * 3 + 1] * dFl[2] + Ri[e * 3 + 2] * dFl[3];
            }
            /* 2x2 Gauss rule on [-1/2,1/2]^2: weights 1/4 */
            for (int v = 0; v < NV; ++v) {
                FF[v] += 0.25 * area * Fg[v];
                dFF[v] += 0.25 * area * dFg[v];
            }
        }
    return 0;
}

/* grid-velocity flux of the face: the volume swept per unit time,
 * sum over Gauss points of w * area * U_g . n (discrete GCL) */
static double face_swept_rate(const orc_geom *G, int d, int i, int j, int k)
{
    double fv[2][2][3], fu[2][2][3];
    face_vertices(G, d, i, j, k, fv);
    face_vertex_velocity(G, d, i, j, k, fu);
    double s = 0.0;
    for (int ga = 0; ga < 2; ++ga)
        for (int gb = 0; gb < 2; ++gb) {
            double ea = GNODE[ga], eb = GNODE[gb];
            double Xa[3] = {0, 0, 0}, Xb[3] = {0, 0, 0}, Vg[3] = {0, 0, 0};
            for (int sa = 0; sa < 2; ++sa)
                for (int sb = 0; sb < 2; ++sb) {
                    double qa = 2.0 * sa - 1.0, qb = 2.0 * sb - 1.0;
                    double phi = 0.25 * (1.0 + 2.0 * qa * ea) * (1.0 + 2.0 * qb * eb);
                    double pa = 0.5 * qa * (1.0 + 2.0 * qb * eb);
                    double pb = 0.5 * qb * (1.0 + 2.0 * qa * ea);
                    for (int e = 0; e < 3; ++e) {
                        Xa[e] += fv[sa][sb][e] * pa;
                        Xb[e] += fv[sa][sb][e] * pb;
                        Vg[e] += fu[sa][sb][e] * phi;
                    }
                }
            double nrm[3];
            cross3(Xa, Xb, nrm); /* = area * n_x */
            s += 0.25 * (Vg[0] * nrm[0] + Vg[1] * nrm[1] + Vg[2] * nrm[2]);
        }
    return s;
}

/* Residuals R = -sum_faces F (the face-integrated flux leaving the cell)
 * and dR/dt for every interior cell, plus the grid's volume rate V = sum
 * of swept rates (zero on a fixed mesh).  L = R/|Omega| on a fixed mesh.
 * Only the cells listed in `cells` are computed when ncells >= 0. */
/* Right eigenvectors of the Euler flux Jacobian n . dF/dQ for n = e_d at
 * the state W (columns of R, row-major 5x5): the acoustic waves u_n -+ c,
 * the entropy wave and the two shear waves along the tangents e_{d+1},
 * e_{d+2}; L = R^{-1} by Gaussian elimination.  Characteristic variables
 * are L Q (Sec. 4). */
int orc_char_basis(const orc_cfg *c, const double *W, int d, double *Rm, double *Lm)
{
    double rho = W[0], u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    double p = pressure_of(c, W);
    if (!(rho > 0.0) || !(p > 0.0)) return -1;
    double cs = sqrt(c->gamma * p / rho), H = (W[4] + p) / rho, k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    int a = (d + 1) % 3, b = (d + 2) % 3;
    double col[NV][NV];
    for (int m = 0; m < NV; ++m)
        for (int v = 0; v < NV; ++v) col[m][v] = 0.0;
    /* u_n - c */
    col[0][0] = 1.0;
    for (int e = 0; e < 3; ++e) col[0][1 + e] = u[e] - (e == d ? cs : 0.0);
    col[0][4] = H - cs * u[d];
    /* entropy */
    col[1][0] = 1.0;
    for (int e = 0; e < 3; ++e) col[1][1 + e] = u[e];
    col[1][4] = k;
    /* shear along e_a and e_b */
    col[2][1 + a] = 1.0;
    col[2][4] = u[a];
    col[3][1 + b] = 1.0;
    col[3][4] = u[b];
    /* u_n + c */
    col[4][0] = 1.0;
    for (int e = 0; e < 3; ++e) col[4][1 + e] = u[e] + (e == d ? cs : 0.0);
    col[4][4] = H + cs * u[d];
    for (int v = 0; v < NV; ++v)
        for (int m = 0; m < NV; ++m) Rm[v * NV + m] = col[m][v];
    for (int m = 0; m < NV; ++m) {
        double e[NV] = {0, 0, 0, 0, 0}, x[NV];
        e[m] = 1.0;
        if (gauss_solve(NV, Rm, e, x)) return -1;
        for (int v = 0; v < NV; ++v) Lm[v * NV + m] = x[v];
    }
    return 0;
}

static int residuals(const orc_cfg *c, const orc_geom *G, const double *q, double dt,
                     double *R, double *dR, double *V, long ncells, const long *cells)
{
    const orc_dims *D = &G->D;
    /* characteristic variables along the face normal: axis-aligned faces */
    if (c->charvar && c->mesh != 0) return -1;
    size_t nint = (size_t)c->n[0] * c->n[1] * c->n[2];
    double *Qp = (double *)malloc(D->ncell * NV * sizeof(double));
    long *slot = (long *)malloc(D->ncell * sizeof(long));
    unsigned char *need = (unsigned char *)calloc(D->ncell, 1);
    slim_rec *rec = NULL;
    if (!Qp || !slot || !need) { free(Qp); free(slot); free(need); return -1; }
    if (fill_ghosts(c, D, q, Qp)) { free(Qp); free(slot); free(need); return -1; }

    /* which cells must be reconstructed: a requested cell and its 6 face neighbours */
    size_t nout = ncells >= 0 ? (size_t)ncells : nint;
    for (size_t o = 0; o < nout; ++o) {
        long lin = ncells >= 0 ? cells[o] : (long)o;
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
        need[cid(D, i, j, k)] = 1;
        for (int d = 0; d < 3; ++d)
            for (int s = -1; s <= 1; s += 2) {
                int o3[3] = {i, j, k};
                o3[d] += s;
                need[cid(D, o3[0], o3[1], o3[2])] = 1;
            }
    }
    int err = 0;
    int nx1 = c->n[0] + 2, ny1 = c->n[1] + 2, nz1 = c->n[2] + 2;
    long nrec = (long)nx1 * ny1 * nz1, nslot = 0;
    for (size_t id = 0; id < D->ncell; ++id) slot[id] = need[id] ? nslot++ : -1;
    rec = (slim_rec *)malloc((size_t)(nslot > 0 ? nslot : 1) * sizeof(slim_rec));
    if (!rec) { free(Qp); free(slot); free(need); return -1; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(ORC_THREADS(c))
    for (long lin = 0; lin < nrec; ++lin) {
        int i = (int)(lin % nx1) - 1, j = (int)((lin / nx1) % ny1) - 1, k = (int)(lin / ((long)nx1 * ny1)) - 1;
        size_t id = cid(D, i, j, k);
        if (need[id] && !c->charvar) {
            cell_rec full;
            reconstruct_cell(c, G, Qp, i, j, k, &full);
            slim_from(&full, &rec[slot[id]]);
        }
    }

    /* every face once: axis d, index f in [0, n_d] along d, transverse
     * indices in range; the face lies between cells f-1 and f along d */
    long nf[3], fbase[3], ftot = 0;
    for (int d = 0; d < 3; ++d) {
        nf[d] = 1;
        for (int e = 0; e < 3; ++e) nf[d] *= (e == d) ? c->n[e] + 1 : c->n[e];
        fbase[d] = ftot;
        ftot += nf[d];
    }
    double *FF = (double *)malloc((size_t)ftot * 2 * NV * sizeof(double));
    double *SW = (double *)malloc((size_t)ftot * sizeof(double));
    unsigned char *fneed = (unsigned char *)calloc((size_t)ftot, 1);
    if (!FF || !SW || !fneed) { free(FF); free(SW); free(fneed); free(Qp); free(rec); free(need); return -1; }
#define FACE_ID(d, f3) (fbase[d] + (((long)(f3)[2] * ((d) == 1 ? c->n[1] + 1 : c->n[1]) + (f3)[1]) \
                                    * ((d) == 0 ? c->n[0] + 1 : c->n[0]) + (f3)[0]))
    for (size_t o = 0; o < nout; ++o) {
        long lin = ncells >= 0 ? cells[o] : (long)o;
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                int o3[3] = {i, j, k};
                o3[d] += s;
                fneed[FACE_ID(d, o3)] = 1;
            }
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(ORC_THREADS(c))
    for (long fid = 0; fid < ftot; ++fid) {
        if (!fneed[fid]) continue;
        int d = fid >= fbase[2] ? 2 : (fid >= fbase[1] ? 1 : 0);
        long r0 = fid - fbase[d];
        int ext[3] = {c->n[0], c->n[1], c->n[2]};
        ext[d] += 1;
        int o3[3] = {(int)(r0 % ext[0]), (int)((r0 / ext[0]) % ext[1]), (int)(r0 / ((long)ext[0] * ext[1]))};
        int l3[3] = {o3[0], o3[1], o3[2]};
        l3[d] -= 1;
        if (c->charvar) {
            /* characteristic variables of this face (Sec. 4): the basis of
             * the Jacobian along the face normal at the mean of the two
             * cell averages (reading), both sides reconstructed in it */
            size_t idl = cid(D, l3[0], l3[1], l3[2]), idr = cid(D, o3[0], o3[1], o3[2]);
            double Wm[NV], Rm[NV * NV], Lm[NV * NV];
            for (int v = 0; v < NV; ++v) Wm[v] = 0.5 * (Qp[(size_t)v * D->ncell + idl] + Qp[(size_t)v * D->ncell + idr]);
            slim_rec sl, sr;
            if (orc_char_basis(c, Wm, d, Rm, Lm)) {
                err = 1;
            } else {
                cell_rec full;
                reconstruct_cell_proj(c, G, Qp, l3[0], l3[1], l3[2], Lm, Rm, &full);
                slim_from(&full, &sl);
                reconstruct_cell_proj(c, G, Qp, o3[0], o3[1], o3[2], Lm, Rm, &full);
                slim_from(&full, &sr);
                if (face_flux(c, G, &sl, &sr, d, o3[0], o3[1], o3[2], dt, &FF[fid * 2 * NV], &FF[fid * 2 * NV + NV]))
                    err = 1;
            }
        } else if (face_flux(c, G, &rec[slot[cid(D, l3[0], l3[1], l3[2])]], &rec[slot[cid(D, o3[0], o3[1], o3[2])]], d,
                             o3[0], o3[1], o3[2], dt, &FF[fid * 2 * NV], &FF[fid * 2 * NV + NV]))
            err = 1;
        SW[fid] = face_swept_rate(G, d, o3[0], o3[1], o3[2]);
    }
    for (size_t o = 0; o < nout; ++o) {
        long lin = ncells >= 0 ? cells[o] : (long)o;
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
        double r[NV] = {0, 0, 0, 0, 0}, dr[NV] = {0, 0, 0, 0, 0}, vr = 0.0;
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                /* face between (cell - e_d, cell) for s = 0, (cell, cell + e_d) for s = 1 */
                int o3[3] = {i, j, k};
                o3[d] += s;
                long fid = FACE_ID(d, o3);
                double sg = s ? -1.0 : 1.0; /* flux along n_x leaves through the upper face */
                for (int v = 0; v < NV; ++v) {
                    r[v] += sg * FF[fid * 2 * NV + v];
                    dr[v] += sg * FF[fid * 2 * NV + NV + v];
                }
                vr -= sg * SW[fid];
            }
        for (int v = 0; v < NV; ++v) {
            R[(size_t)v * nout + o] = r[v];
            dR[(size_t)v * nout + o] = dr[v];
        }
        if (V) V[o] = vr;
    }
#undef FACE_ID
    free(FF);
    free(SW);
    free(fneed);
    free(Qp);
    free(rec);
    free(slot);
    free(need);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* exported API                                                              */
/* ------------------------------------------------------------------------ */

/* L(Q) and dL/dt(Q) on a fixed mesh at time t, for all cells (ncells < 0)
 * or for the listed linear cell indices; outputs [5][ncells]. */
int orc_operator(const orc_cfg *c, const double *q, double t, double dt, long ncells, const long *cells,
                 double *L, double *dL)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1;
    size_t nout = ncells >= 0 ? (size_t)ncells : (size_t)c->n[0] * c->n[1] * c->n[2];
    int rc = residuals(c, &G, q, dt, L, dL, NULL, ncells, cells);
    for (size_t o = 0; o < nout && rc == 0; ++o) {
        long lin = ncells >= 0 ? cells[o] : (long)o;
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
        cell_geom cg;
        cell_geometry(&G, i, j, k, &cg);
        double vol = cg.vol;
        for (int v = 0; v < NV; ++v) {
            L[(size_t)v * nout + o] /= vol;
            dL[(size_t)v * nout + o] /= vol;
        }
    }
    geom_free(&G);
    return rc;
}

/* P~ of every interior cell: coef[cell][5][10] = (Q_c, 9 coefficients in
 * the scaled frame), flag[cell], and P0's coefficients a0[cell][5][9] */
int orc_reconstruct(const orc_cfg *c, const double *q, double t, double *coef, int *flag, double *a0)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1;
    const orc_dims *D = &G.D;
    double *Qp = (double *)malloc(D->ncell * NV * sizeof(double));
    if (!Qp) { geom_free(&G); return -1; }
    if (fill_ghosts(c, D, q, Qp)) { free(Qp); geom_free(&G); return -1; }
    long nint = (long)c->n[0] * c->n[1] * c->n[2];
#pragma omp parallel for schedule(dynamic, 64) num_threads(ORC_THREADS(c))
    for (long lin = 0; lin < nint; ++lin) {
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
        cell_rec r;
        reconstruct_cell(c, &G, Qp, i, j, k, &r);
        for (int v = 0; v < NV; ++v) {
            coef[(lin * NV + v) * 10] = r.Qc[v];
            for (int m = 0; m < 9; ++m) {
                coef[(lin * NV + v) * 10 + 1 + m] = r.coef[v][m];
                if (a0) a0[(lin * NV + v) * 9 + m] = r.a[v][m];
            }
        }
        if (flag) flag[lin] = r.flag;
    }
    free(Qp);
    geom_free(&G);
    return 0;
}

/* Smoothness indicators and normalised weights of cell `lin`:
 * beta[5][25], wbar[5][25] (index 0 = big stencil) */
int orc_weno_weights(const orc_cfg *c, const double *q, double t, long lin, double *beta, double *wbar)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1;
    const orc_dims *D = &G.D;
    double *Qp = (double *)malloc(D->ncell * NV * sizeof(double));
    if (!Qp) { geom_free(&G); return -1; }
    if (fill_ghosts(c, D, q, Qp)) { free(Qp); geom_free(&G); return -1; }
    int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
    cell_rec r;
    reconstruct_cell(c, &G, Qp, i, j, k, &r);
    for (int v = 0; v < NV; ++v)
        for (int s = 0; s <= 24; ++s) {
            beta[v * 25 + s] = r.beta[v][s];
            wbar[v * 25 + s] = r.wbar[v][s];
        }
    free(Qp);
    geom_free(&G);
    return 0;
}

/* Values and physical gradients of P~ of cell `lin` at nx physical points:
 * out[p][5][4] = (value, d/dx, d/dy, d/dz) */
int orc_eval_reconstruction(const orc_cfg *c, const double *q, double t, long lin, int np, const double *x,
                            double *out)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1;
    const orc_dims *D = &G.D;
    double *Qp = (double *)malloc(D->ncell * NV * sizeof(double));
    if (!Qp) { geom_free(&G); return -1; }
    if (fill_ghosts(c, D, q, Qp)) { free(Qp); geom_free(&G); return -1; }
    int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((long)c->n[0] * c->n[1]));
    cell_rec r;
    slim_rec sr;
    reconstruct_cell(c, &G, Qp, i, j, k, &r);
    slim_from(&r, &sr);
    for (int p = 0; p < np; ++p) {
        double W[NV], dW[NV][3];
        rec_eval(&sr, &x[p * 3], W, dW);
        for (int v = 0; v < NV; ++v) {
            out[(p * NV + v) * 4] = W[v];
            for (int e = 0; e < 3; ++e) out[(p * NV + v) * 4 + 1 + e] = dW[v][e];
        }
    }
    free(Qp);
    geom_free(&G);
    return 0;
}

/* Time step from the CFL condition (Sec. 4 uses CFL = 0.35).
 * Reading: dt = CFL * min_cells h/(|U| + c), h = |Omega|^(1/3). */
double orc_cfl_dt(const orc_cfg *c, const double *q, double t, double cfl)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1.0;
    size_t nint = (size_t)c->n[0] * c->n[1] * c->n[2];
    double best = INFINITY;
    for (size_t lin = 0; lin < nint; ++lin) {
        int i = (int)(lin % c->n[0]), j = (int)((lin / c->n[0]) % c->n[1]), k = (int)(lin / ((size_t)c->n[0] * c->n[1]));
        double W[NV];
        for (int v = 0; v < NV; ++v) W[v] = q[v * nint + lin];
        double rho = W[0];
        double speed = sqrt(W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / rho;
        double snd = sqrt(c->gamma * pressure_of(c, W) / rho);
        cell_geom cg;
        cell_geometry(&G, i, j, k, &cg);
        double hloc = cg.h;
        double v = hloc / (speed + snd);
        if (v < best) best = v;
    }
    geom_free(&G);
    return cfl * best;
}

/* Cell volumes |Omega| of the interior cells at time t (2x2x2 Gauss). */
int orc_volumes(const orc_cfg *c, double t, double *vol)
{
    orc_geom G;
    if (geom_build(c, t, &G)) return -1;
    for (int k = 0; k < c->n[2]; ++k)
        for (int j = 0; j < c->n[1]; ++j)
            for (int i = 0; i < c->n[0]; ++i)
            {
                cell_geom cg;
                cell_geometry(&G, i, j, k, &cg);
                vol[((size_t)k * c->n[1] + j) * c->n[0] + i] = cg.vol;
            }
    geom_free(&G);
    return 0;
}

/* One step of the two-stage fourth-order method (Sec. 3) for
 * dy/dt = L(y) with the rate pair (L, dL/dt) supplied by `rate`:
 *   y*      = y^n + dt/2 L(y^n) + dt^2/8 dL/dt(y^n)
 *   y^{n+1} = y^n + dt L(y^n) + dt^2/6 (dL/dt(y^n) + 2 dL/dt(y*))
 * rate(ctx, stage, y, L, dL) evaluates the pair at y^n (stage 0) and at y*
 * (stage 1); the intermediate stage reuses the same dt. */
typedef int (*orc_rate_fn)(void *ctx, int stage, const double *y, double *L, double *dL);

int orc_two_stage(long n, double *y, double dt, orc_rate_fn rate, void *ctx)
{
    double *L1 = malloc(n * sizeof(double)), *dL1 = malloc(n * sizeof(double));
    double *L2 = malloc(n * sizeof(double)), *dL2 = malloc(n * sizeof(double));
    double *ys = malloc(n * sizeof(double));
    int rc = -1;
    if (!L1 || !dL1 || !L2 || !dL2 || !ys) goto out;
    if ((rc = rate(ctx, 0, y, L1, dL1))) goto out;
    for (long i = 0; i < n; ++i) ys[i] = y[i] + 0.5 * dt * L1[i] + 0.125 * dt * dt * dL1[i];
    if ((rc = rate(ctx, 1, ys, L2, dL2))) goto out;
    for (long i = 0; i < n; ++i) y[i] = y[i] + dt * L1[i] + dt * dt / 6.0 * (dL1[i] + 2.0 * dL2[i]);
out:
    free(L1); free(dL1); free(L2); free(dL2); free(ys);
    return rc;
}

/* The scheme's rate pair for orc_two_stage.  y = (|Omega| Q [5][N], |Omega| [N]);
 * L = (-sum of face fluxes, swept-volume rate), dL/dt = (its time derivative, 0):
 * the geometry of a stage is frozen at its start (Remark 2), so the volume
 * rate has no time derivative within a stage. */
typedef struct {
    const orc_cfg *c;
    size_t nint;
    double t, dt;
    const double *q0;  /* Q^n itself, used at stage 0 */
    double *qs;        /* the intermediate state Q* = (|Omega| Q)* / |Omega|* */
} step_ctx;

static int scheme_rate(void *vctx, int stage, const double *y, double *L, double *dL)
{
    step_ctx *x = (step_ctx *)vctx;
    const size_t nint = x->nint;
    const double *q = x->q0;
    if (stage == 1) {
        for (size_t i = 0; i < nint; ++i)
            for (int v = 0; v < NV; ++v) x->qs[(size_t)v * nint + i] = y[(size_t)v * nint + i] / y[NV * nint + i];
        q = x->qs;
    }
    orc_geom G;
    if (geom_build(x->c, x->t + (stage ? 0.5 * x->dt : 0.0), &G)) return -1;
    int rc = residuals(x->c, &G, q, x->dt, L, dL, L + NV * nint, -1, NULL);
    geom_free(&G);
    for (size_t i = 0; i < nint; ++i) dL[NV * nint + i] = 0.0;
    return rc;
}

/* Time stepping of the scheme (Sec. 3): each step is orc_two_stage on
 * (|Omega| Q, |Omega|).  Reading: the intermediate stage reuses the same
 * dt, with tau from the pressures of Q*.  On a moving mesh (Remark 2) the
 * two-stage formula advances |Omega| Q with geometry frozen at the start of
 * each stage (t_n, then t_n + dt/2), and the volume that divides it is
 * advanced by the same formula from the grid's swept-volume rate (discrete
 * geometric conservation law); on a fixed mesh that rate is zero.
 * dt_fixed > 0 fixes dt; otherwise the CFL step is clipped to t_end.
 * vol (optional, in/out) carries those volumes. */
int orc_step(const orc_cfg *c, double *q, double *t, int nsteps, double cfl, double dt_fixed, double t_end,
             double *vol_io, int *steps_done)
{
    size_t nint = (size_t)c->n[0] * c->n[1] * c->n[2];
    double *y = malloc(nint * (NV + 1) * sizeof(double));
    double *qs = malloc(nint * NV * sizeof(double));
    double *vol = y ? y + NV * nint : NULL;
    int rc = 0, done = 0;
    if (!y || !qs) { rc = -1; goto out; }
    if (vol_io && c->mesh == 2) memcpy(vol, vol_io, nint * sizeof(double));
    else if (orc_volumes(c, *t, vol)) { rc = -1; goto out; }
    for (int n = 0; n < nsteps; ++n) {
        double dt = dt_fixed > 0.0 ? dt_fixed : orc_cfl_dt(c, q, *t, cfl);
        if (dt_fixed <= 0.0 && *t + dt > t_end) dt = t_end - *t;
        if (!(dt > 0.0)) break;
        for (size_t i = 0; i < nint; ++i)
            for (int v = 0; v < NV; ++v) y[(size_t)v * nint + i] = vol[i] * q[(size_t)v * nint + i];
        step_ctx x = {c, nint, *t, dt, q, qs};
        if ((rc = orc_two_stage((long)(nint * (NV + 1)), y, dt, scheme_rate, &x))) goto out;
        for (size_t i = 0; i < nint; ++i)
            for (int v = 0; v < NV; ++v) q[(size_t)v * nint + i] = y[(size_t)v * nint + i] / vol[i];
        *t += dt;
        ++done;
    }
    if (vol_io) memcpy(vol_io, vol, nint * sizeof(double));
out:
    if (steps_done) *steps_done = done;
    free(y); free(qs);
    return rc;
}

/* moment tables for the tests: out[0..MAXE] = <u^n> of the normalised
 * Maxwellian over the chosen domain (side 0, +1, -1) */
void orc_moments_1d(double U, double lam, int side, double *out)
{
    mom1d M;
    moments_1d(U, lam, side, &M);
    for (int n = 0; n <= MAXE; ++n) out[n] = M.m[n];
}

/* the 5x5 moment matrix int psi psi^T g for a conservative state W */
void orc_moment_matrix(const orc_cfg *c, const double *W, double *M)
{
    maxwellian g;
    make_maxwellian(c, W, 0, &g);
    moment_matrix(&g, M);
}

/* geometry of the big stencil and sub-stencils, for the tests */
/* the stencil tables of S' (Remark of Sec. 2): big[24][3], sub[8][3][3] */
void orc_stencils_sprime(int *big, int *sub)
{
    int off[24][3], so[24][4][3], nrow;
    big_stencil(off, 1);
    for (int s = 0; s < 24; ++s)
        for (int d = 0; d < 3; ++d) big[s * 3 + d] = off[s][d];
    int ns = sub_stencils_sel(so, &nrow, 1);
    for (int m = 0; m < ns; ++m)
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) sub[(m * 3 + r) * 3 + d] = so[m][r][d];
}

void orc_stencils(int *big, int *sub)
{
    int off[24][3], so[24][4][3];
    big_stencil(off, 0);
    sub_stencils(so);
    memcpy(big, off, 18 * sizeof off[0]);
    memcpy(sub, so, sizeof so);
}
