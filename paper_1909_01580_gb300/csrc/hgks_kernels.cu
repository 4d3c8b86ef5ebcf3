// Kernels of the HGKS stage sweep on sm_103a (uniform mesh of cubes):
// ghost fill, WENO-AO reconstruction (Sec. 2), Gauss-point gas-kinetic
// face flux (Sec. 3), two-stage update and CFL reduction.
#include "hgks_kernels.cuh"

namespace hk {

// the 2-point Gauss-Legendre node on [-1/2, 1/2]
#define GAUSS_S 0.28867513459481288225

// ---------------------------------------------------------------------------
// ghost cells: periodic wrap or reflective mirror (normal momentum negated),
// width 2 including edge and corner ghosts; every ghost reads its interior
// source directly, so one launch fills all of them.
// ---------------------------------------------------------------------------
__global__ void k_halo(double *__restrict__ Q, Geo g)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = g.pstride;
    if (t >= tot) return;
    int ip = (int)(t % g.px), jp = (int)((t / g.px) % g.py), kp = (int)(t / ((long long)g.px * g.py));
    int idx[3] = {ip - 2, jp - 2, kp - 2};
    int n[3] = {g.nx, g.ny, g.nz};
    int src[3];
    int flip[3] = {0, 0, 0};
    bool ghost = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int s = idx[d];
        if (s < 0) {
            ghost = true;
            if (g.bc[2 * d] == 0) s += n[d];
            else { s = -1 - s; flip[d] = 1; }
        } else if (s >= n[d]) {
            ghost = true;
            if (g.bc[2 * d + 1] == 0) s -= n[d];
            else { s = 2 * n[d] - 1 - s; flip[d] = 1; }
        }
        src[d] = s;
    }
    if (!ghost) return;
    long long from = pidx(g, src[0], src[1], src[2]);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        double val = Q[v * g.pstride + from];
        if (v >= 1 && v <= 3 && flip[v - 1]) val = -val;
        Q[v * g.pstride + t] = val;
    }
}

template <typename R>
__device__ __forceinline__ void load_stencil(const double *__restrict__ Qv, const Geo &g, int i, int j, int k,
                                             double qc, Stencil<R> &st)
{
    const long long sx = 1, sy = g.px, sz = (long long)g.px * g.py;
    const long long c = pidx(g, i, j, k);
    const long long sd[3] = {sx, sy, sz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.f[d][0] = R(Qv[c - sd[d]] - qc);
        st.f[d][1] = R(Qv[c + sd[d]] - qc);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const long long a = sd[p], b = sd[(p + 1) % 3];
#pragma unroll
        for (int sa = 0; sa < 2; ++sa)
#pragma unroll
            for (int sb = 0; sb < 2; ++sb) st.e[p][sa][sb] = R(Qv[c + (sa ? a : -a) + (sb ? b : -b)] - qc);
    }
}

// literal positivity check (Sec. 4): rho and p of every P_m, m = 0..24, at
// every one of the cell's 24 Gauss points
template <typename R>
__device__ __noinline__ bool positivity_violated(const double *__restrict__ Q, const Geo &g, int i, int j, int k, R gamma)
{
    R qcv[5];
    Stencil<R> st[5];
    for (int v = 0; v < 5; ++v) {
        const double qc = Q[v * g.pstride + pidx(g, i, j, k)];
        qcv[v] = R(qc);
        load_stencil(Q + v * g.pstride, g, i, j, k, qc, st[v]);
    }
    for (int m = 0; m <= 24; ++m) {
        R cf[5][9];
        for (int v = 0; v < 5; ++v) {
            if (m == 0) {
                big_stencil_P0(st[v], cf[v]);
            } else {
                R b[3];
                sub_stencil_rt(st[v], m - 1, b);
                for (int n = 0; n < 9; ++n) cf[v][n] = n < 3 ? b[n] : R(0);
            }
        }
        for (int gq = 0; gq < 24; ++gq) {
            const int d = gq / 8, side = (gq / 4) & 1, ga = (gq >> 1) & 1, gb = gq & 1;
            R X[3];
            X[d] = side ? R(0.5) : R(-0.5);
            X[(d + 1) % 3] = ga ? R(GAUSS_S) : R(-GAUSS_S);
            X[(d + 2) % 3] = gb ? R(GAUSS_S) : R(-GAUSS_S);
            R W[5];
            for (int v = 0; v < 5; ++v) W[v] = qcv[v] + poly9(cf[v], X);
            const R p = (gamma - R(1)) * (W[4] - R(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0]);
            if (W[0] < R(0) || p < R(0)) return true;
        }
    }
    return false;
}

template <typename R>
__global__ void __launch_bounds__(128) k_recon(const double *__restrict__ Q, R *__restrict__ coef,
                                               unsigned char *__restrict__ flag, Geo g, Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.cstride) return;
    const int i = (int)(t % g.cx) - 1, j = (int)((t / g.cx) % g.cy) - 1, k = (int)(t / ((long long)g.cx * g.cy)) - 1;
    R rad[5], qcv[5];
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + v * g.pstride;
        const double qc = Qv[pidx(g, i, j, k)];
        qcv[v] = R(qc);
        Stencil<R> st;
        load_stencil(Qv, g, i, j, k, qc, st);
        R out[9];
        weno_ao(st, S, out, rad[v]);
#pragma unroll
        coef[coef_slot(v, 0) * g.cstride + t] = R(qc);
#pragma unroll
        for (int n = 0; n < 9; ++n) coef[coef_slot(v, 1 + n) * g.cstride + t] = out[n];
    }
    // positivity fallback: the cheap sufficient test first, the literal
    // check of all 25 polynomials at the 24 Gauss points only when it fails
    bool bad = false;
    if (S.limiter && !positivity_certain(qcv, rad, R(S.gamma))) bad = positivity_violated<R>(Q, g, i, j, k, R(S.gamma));
    if (bad) {
        for (int v = 0; v < 5; ++v)
            for (int n = 1; n < 10; ++n) coef[coef_slot(v, n) * g.cstride + t] = R(0);
        atomicAdd(&ctl->flagged, 1);
    }
    flag[t] = bad ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Face flux: one thread per Gauss point, 4 consecutive lanes per face.  The
// local frame of a face normal to axis D is (e_D, e_{D+1}, e_{D+2}) (the
// printed frame for D = x, and its cyclic images).  The 2x2 Gauss sum with
// weights 1/4 is reduced across the 4 lanes in FP64; the stored value is
// the face-averaged flux per unit area.
// ---------------------------------------------------------------------------
template <typename R, int D>
__device__ __forceinline__ void eval_side(const R *__restrict__ coef, const Geo &g, long long ci, R xd, R xa, R xb,
                                          R W[5], R dW[3][5])
{
    R X[3];
    X[D] = xd;
    X[(D + 1) % 3] = xa;
    X[(D + 2) % 3] = xb;
    const R ih = R(g.inv_h);
    R val[5], grad[5][3];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        R c[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) c[n] = coef[coef_slot(v, 1 + n) * g.cstride + ci];
        R s;
        poly_value_grad(c, X, ih, s, grad[v]);
        val[v] = coef[coef_slot(v, 0) * g.cstride + ci] + s;
    }
    // local frame: local axis l is global axis (D + l) % 3
    W[0] = val[0];
    W[4] = val[4];
#pragma unroll
    for (int l = 0; l < 3; ++l) W[1 + l] = val[1 + (D + l) % 3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const int gd = (D + l) % 3;
        dW[l][0] = grad[0][gd];
        dW[l][4] = grad[4][gd];
#pragma unroll
        for (int m = 0; m < 3; ++m) dW[l][1 + m] = grad[1 + (D + m) % 3][gd];
    }
}

template <typename R, int D>
__global__ void __launch_bounds__(128) k_face_flux(const R *__restrict__ coef, double *__restrict__ Fout, Geo g,
                                                   Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    const double dt = ctl->dt;
    const int ex = g.nx + (D == 0), ey = g.ny + (D == 1), ez = g.nz + (D == 2);
    const long long nface = (long long)ex * ey * ez;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long face = t >> 2;
    const int gp = (int)(t & 3);
    const bool valid = face < nface;
    if (!valid) face = nface - 1;
    // (i, j, k) is the right cell; the left cell is one step back along D
    const int i = (int)(face % ex), j = (int)((face / ex) % ey), k = (int)(face / ((long long)ex * ey));
    const int il = i - (D == 0), jl = j - (D == 1), kl = k - (D == 2);
    const R xa = (gp & 2) ? R(GAUSS_S) : R(-GAUSS_S);
    const R xb = (gp & 1) ? R(GAUSS_S) : R(-GAUSS_S);
    R Wl[5], dWl[3][5], Wr[5], dWr[3][5];
    eval_side<R, D>(coef, g, cidx(g, il, jl, kl), R(0.5), xa, xb, Wl, dWl);
    eval_side<R, D>(coef, g, cidx(g, i, j, k), R(-0.5), xa, xb, Wr, dWr);
    R F[5], dF[5];
    gks_flux<R>(Wl, dWl, Wr, dWr, S, R(dt), F, dF);
    // back to the global frame, Gauss weight 1/4, sum of the 4 lanes in the
    // working precision; the face value is stored in FP64
    R f[10];
    f[0] = R(0.25) * F[0];
    f[4] = R(0.25) * F[4];
    f[5] = R(0.25) * dF[0];
    f[9] = R(0.25) * dF[4];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        f[1 + (D + l) % 3] = R(0.25) * F[1 + l];
        f[6 + (D + l) % 3] = R(0.25) * dF[1 + l];
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        f[q] += __shfl_xor_sync(0xffffffffu, f[q], 1);
        f[q] += __shfl_xor_sync(0xffffffffu, f[q], 2);
    }
    if (valid && gp == 0) {
#pragma unroll
        for (int q = 0; q < 10; ++q) Fout[q * nface + face] = double(f[q]);
    }
}

// ---------------------------------------------------------------------------
// update: L = -(1/h) sum over the 3 axes of (F_upper - F_lower) with the
// face-averaged fluxes, and the two-stage fourth-order combination (Sec. 3)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cell_residual(const double *__restrict__ Fx, const double *__restrict__ Fy,
                                              const double *__restrict__ Fz, const Geo &g, int i, int j, int k,
                                              double L[5], double dL[5])
{
    const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
    const long long nfy = (long long)g.nx * (g.ny + 1) * g.nz;
    const long long nfz = (long long)g.nx * g.ny * (g.nz + 1);
    const long long fx0 = ((long long)k * g.ny + j) * (g.nx + 1) + i;
    const long long fy0 = ((long long)k * (g.ny + 1) + j) * g.nx + i;
    const long long fz0 = ((long long)k * g.ny + j) * g.nx + i;
    const long long fzs = (long long)g.nx * g.ny;
#pragma unroll
    for (int v = 0; v < 10; ++v) {
        const double sx = Fx[v * nfx + fx0 + 1] - Fx[v * nfx + fx0];
        const double sy = Fy[v * nfy + fy0 + g.nx] - Fy[v * nfy + fy0];
        const double sz = Fz[v * nfz + fz0 + fzs] - Fz[v * nfz + fz0];
        const double r = -(sx + sy + sz) * g.inv_h;
        if (v < 5) L[v] = r;
        else dL[v - 5] = r;
    }
}

template <int STAGE>
__global__ void __launch_bounds__(256) k_update(double *__restrict__ Qn, double *__restrict__ Qs,
                                                double *__restrict__ Wacc, const double *__restrict__ Fx,
                                                const double *__restrict__ Fy, const double *__restrict__ Fz, Geo g,
                                                double gamma, Ctl *ctl)
{
    if (!ctl->active) return;
    const double dt = ctl->dt;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (STAGE == 2 && t == 0) {
        ctl->t += dt;
        ctl->steps_done += 1;
    }
    if (t >= g.ncell) return;
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
    double L[5], dL[5];
    cell_residual(Fx, Fy, Fz, g, i, j, k, L, dL);
    const long long pi = pidx(g, i, j, k);
    if (STAGE == 1) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double q = Qn[v * g.pstride + pi];
            Qs[v * g.pstride + pi] = q + 0.5 * dt * L[v] + 0.125 * dt * dt * dL[v];
            Wacc[v * g.ncell + t] = q + dt * L[v] + (dt * dt / 6.0) * dL[v];
        }
    } else {
        double W[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            W[v] = Wacc[v * g.ncell + t] + (dt * dt / 3.0) * dL[v];
            Qn[v * g.pstride + pi] = W[v];
        }
        const double p = (gamma - 1.0) * (W[4] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0]);
        if (!(W[0] > 0.0) || !(p > 0.0)) atomicOr(&ctl->status, 1);
    }
}

__global__ void k_residual(const double *__restrict__ Fx, const double *__restrict__ Fy,
                           const double *__restrict__ Fz, Geo g, double *__restrict__ L, double *__restrict__ dL)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
    double l[5], dl[5];
    cell_residual(Fx, Fy, Fz, g, i, j, k, l, dl);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        L[v * g.ncell + t] = l[v];
        dL[v * g.ncell + t] = dl[v];
    }
}

// ---------------------------------------------------------------------------
// CFL: dt = cfl * min_cells h/(|U| + c), reduced in-block with warp
// shuffles and across blocks with an integer atomicMin on the bit pattern
// (positive doubles order like their bits): order-independent, so exact.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cfl(const double *__restrict__ Q, Geo g, double gamma, Ctl *ctl)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = INFINITY;
    if (t < g.ncell) {
        const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
        const long long pi = pidx(g, i, j, k);
        double W[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) W[q] = Q[q * g.pstride + pi];
        const double rho = W[0];
        const double m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
        const double speed = sqrt(m2) / rho;
        const double p = (gamma - 1.0) * (W[4] - 0.5 * m2 / rho);
        const double c = sqrt(gamma * p / rho);
        v = g.h / (speed + c);
        if (!(v > 0.0)) v = 0.0;  // nonphysical: force dt = 0
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) atomicMin(&ctl->minbits, (unsigned long long)__double_as_longlong(v));
    }
}

// one thread: choose dt for this step and arm the stage kernels
__global__ void k_dt(Ctl *ctl, double cfl, double dt_fixed, double t_end)
{
    double dt;
    if (dt_fixed > 0.0) {
        dt = dt_fixed;
    } else {
        dt = cfl * __longlong_as_double((long long)ctl->minbits);
        if (ctl->t + dt > t_end) dt = t_end - ctl->t;
    }
    ctl->dt = dt;
    ctl->active = (dt > 0.0) ? 1 : 0;
    ctl->minbits = (unsigned long long)__double_as_longlong(INFINITY);
    ctl->flagged = 0;
}

__global__ void k_set_ctl(Ctl *ctl, double t, double dt, int active)
{
    ctl->t = t;
    ctl->dt = dt;
    ctl->active = active;
    ctl->status = 0;
    ctl->flagged = 0;
    ctl->minbits = (unsigned long long)__double_as_longlong(INFINITY);
}

// interior <-> padded copies ([5][nz][ny][nx] <-> padded)
__global__ void k_scatter(const double *__restrict__ src, double *__restrict__ Q, Geo g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
    const long long pi = pidx(g, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) Q[v * g.pstride + pi] = src[v * g.ncell + t];
}
__global__ void k_gather(const double *__restrict__ Q, double *__restrict__ dst, Geo g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
    const long long pi = pidx(g, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) dst[v * g.ncell + t] = Q[v * g.pstride + pi];
}

// coefficients of the interior cells to FP64 [ncell][5][9]
template <typename R>
__global__ void k_export_coef(const R *__restrict__ coef, const unsigned char *__restrict__ flag, Geo g,
                              double *__restrict__ out, int *__restrict__ oflag)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
    const long long ci = cidx(g, i, j, k);
    for (int v = 0; v < 5; ++v)
        for (int n = 0; n < 9; ++n) out[t * 45 + v * 9 + n] = double(coef[coef_slot(v, 1 + n) * g.cstride + ci]);
    if (oflag) oflag[t] = flag[ci];
}

// point-flux test surface: one thread per point, inputs in the local frame
template <typename R>
__global__ void k_point_flux(int n, const double *__restrict__ in, const double *__restrict__ ug, double dt,
                             Scheme S, double *__restrict__ F, double *__restrict__ dF)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double *x = in + (long long)p * 40;
    double Ug[3] = {0, 0, 0};
    if (ug)
        for (int d = 0; d < 3; ++d) Ug[d] = ug[(long long)p * 3 + d];
    const double u2 = Ug[0] * Ug[0] + Ug[1] * Ug[1] + Ug[2] * Ug[2];
    R W[2][5], dW[2][3][5];
    for (int s = 0; s < 2; ++s) {
        // shift to the frame moving with the grid: rho U_rel = rho U - rho U_g,
        // E_rel = E - U_g . rho U + |U_g|^2 rho/2 (and the same for slopes)
        const double *b = x + 20 * s;
        W[s][0] = R(b[0]);
        W[s][4] = R(b[4] - (Ug[0] * b[1] + Ug[1] * b[2] + Ug[2] * b[3]) + 0.5 * u2 * b[0]);
        for (int d = 0; d < 3; ++d) W[s][1 + d] = R(b[1 + d] - Ug[d] * b[0]);
        for (int e = 0; e < 3; ++e) {
            const double *db = b + 5 + 5 * e;
            dW[s][e][0] = R(db[0]);
            dW[s][e][4] = R(db[4] - (Ug[0] * db[1] + Ug[1] * db[2] + Ug[2] * db[3]) + 0.5 * u2 * db[0]);
            for (int d = 0; d < 3; ++d) dW[s][e][1 + d] = R(db[1 + d] - Ug[d] * db[0]);
        }
    }
    R f[5], df[5];
    gks_flux<R>(W[0], dW[0], W[1], dW[1], S, R(dt), f, df);
    double Fr[5], dFr[5];
    for (int q = 0; q < 5; ++q) {
        Fr[q] = double(f[q]);
        dFr[q] = double(df[q]);
    }
    // back from the grid frame: u = u_rel + U_g
    double *Fo = F + (long long)p * 5, *dFo = dF + (long long)p * 5;
    Fo[0] = Fr[0];
    dFo[0] = dFr[0];
    for (int d = 0; d < 3; ++d) {
        Fo[1 + d] = Fr[1 + d] + Ug[d] * Fr[0];
        dFo[1 + d] = dFr[1 + d] + Ug[d] * dFr[0];
    }
    Fo[4] = Fr[4] + Ug[0] * Fr[1] + Ug[1] * Fr[2] + Ug[2] * Fr[3] + 0.5 * u2 * Fr[0];
    dFo[4] = dFr[4] + Ug[0] * dFr[1] + Ug[1] * dFr[2] + Ug[2] * dFr[3] + 0.5 * u2 * dFr[0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_halo(double *Q, const Geo &g, cudaStream_t s)
{
    k_halo<<<blocks_for(g.pstride, 256), 256, 0, s>>>(Q, g);
}

template <typename R>
void launch_recon(const double *Q, R *coef, unsigned char *flag, const Geo &g, const Scheme &S, Ctl *ctl,
                  cudaStream_t s)
{
    k_recon<R><<<blocks_for(g.cstride, 128), 128, 0, s>>>(Q, coef, flag, g, S, ctl);
}

template <typename R>
void launch_flux(int axis, const R *coef, double *F, const Geo &g, const Scheme &S, Ctl *ctl, cudaStream_t s)
{
    const long long nface = (long long)(g.nx + (axis == 0)) * (g.ny + (axis == 1)) * (g.nz + (axis == 2));
    const unsigned nb = blocks_for(4 * nface, 128);
    if (axis == 0) k_face_flux<R, 0><<<nb, 128, 0, s>>>(coef, F, g, S, ctl);
    else if (axis == 1) k_face_flux<R, 1><<<nb, 128, 0, s>>>(coef, F, g, S, ctl);
    else k_face_flux<R, 2><<<nb, 128, 0, s>>>(coef, F, g, S, ctl);
}

void launch_update(int stage, double *Qn, double *Qs, double *Wacc, const double *Fx, const double *Fy,
                   const double *Fz, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s)
{
    if (stage == 1) k_update<1><<<blocks_for(g.ncell, 256), 256, 0, s>>>(Qn, Qs, Wacc, Fx, Fy, Fz, g, gamma, ctl);
    else k_update<2><<<blocks_for(g.ncell, 256), 256, 0, s>>>(Qn, Qs, Wacc, Fx, Fy, Fz, g, gamma, ctl);
}

void launch_residual(const double *Fx, const double *Fy, const double *Fz, const Geo &g, double *L, double *dL,
                     cudaStream_t s)
{
    k_residual<<<blocks_for(g.ncell, 256), 256, 0, s>>>(Fx, Fy, Fz, g, L, dL);
}

void launch_cfl(const double *Q, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s)
{
    k_cfl<<<blocks_for(g.ncell, 256), 256, 0, s>>>(Q, g, gamma, ctl);
}

void launch_dt(Ctl *ctl, double cfl, double dt_fixed, double t_end, cudaStream_t s)
{
    k_dt<<<1, 1, 0, s>>>(ctl, cfl, dt_fixed, t_end);
}

void launch_set_ctl(Ctl *ctl, double t, double dt, int active, cudaStream_t s)
{
    k_set_ctl<<<1, 1, 0, s>>>(ctl, t, dt, active);
}

void launch_scatter(const double *src, double *Q, const Geo &g, cudaStream_t s)
{
    k_scatter<<<blocks_for(g.ncell, 256), 256, 0, s>>>(src, Q, g);
}

void launch_gather(const double *Q, double *dst, const Geo &g, cudaStream_t s)
{
    k_gather<<<blocks_for(g.ncell, 256), 256, 0, s>>>(Q, dst, g);
}

template <typename R>
void launch_export_coef(const R *coef, const unsigned char *flag, const Geo &g, double *out, int *oflag,
                        cudaStream_t s)
{
    k_export_coef<R><<<blocks_for(g.ncell, 128), 128, 0, s>>>(coef, flag, g, out, oflag);
}

template <typename R>
void launch_point_flux(int n, const double *in, const double *ug, double dt, const Scheme &S, double *F, double *dF,
                       cudaStream_t s)
{
    k_point_flux<R><<<blocks_for(n, 64), 64, 0, s>>>(n, in, ug, dt, S, F, dF);
}

template void launch_recon<double>(const double *, double *, unsigned char *, const Geo &, const Scheme &, Ctl *,
                                   cudaStream_t);
template void launch_recon<float>(const double *, float *, unsigned char *, const Geo &, const Scheme &, Ctl *,
                                  cudaStream_t);
template void launch_flux<double>(int, const double *, double *, const Geo &, const Scheme &, Ctl *, cudaStream_t);
template void launch_flux<float>(int, const float *, double *, const Geo &, const Scheme &, Ctl *, cudaStream_t);
template void launch_export_coef<double>(const double *, const unsigned char *, const Geo &, double *, int *,
                                         cudaStream_t);
template void launch_export_coef<float>(const float *, const unsigned char *, const Geo &, double *, int *,
                                        cudaStream_t);
template void launch_point_flux<double>(int, const double *, const double *, double, const Scheme &, double *,
                                        double *, cudaStream_t);
template void launch_point_flux<float>(int, const double *, const double *, double, const Scheme &, double *,
                                       double *, cudaStream_t);

}  // namespace hk
