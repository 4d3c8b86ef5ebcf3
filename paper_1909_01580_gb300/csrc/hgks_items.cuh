// Per-item bodies of the stage sweep (one cell, one padded cell or one
// Gauss point per call), shared by the single-instance kernels
// (hgks_kernels.cu) and the batched persistent kernels (hgks_batch.cu) so
// that an instance computes the same arithmetic alone and in a batch.
#pragma once
#include <limits.h>

#include "hgks_device.cuh"

namespace hk {

// the 2-point Gauss-Legendre node on [-1/2, 1/2]
#define GAUSS_S 0.28867513459481288225

// ---------------------------------------------------------------------------
// ghost cells: periodic wrap, reflective mirror (normal momentum negated) or
// non-reflecting outflow (the boundary cell repeated), GHOST layers including
// edge and corner ghosts; every ghost reads its interior source directly, so
// one pass fills all of them.  t: padded linear index.
// ---------------------------------------------------------------------------
// the cell at padded coordinates (ip, jp, kp): nothing for an interior cell
__device__ __forceinline__ void halo_cell(double *__restrict__ Q, const Geo &g, int ip, int jp, int kp)
{
    const long long t = ((long long)kp * g.py + jp) * g.px + ip;
    const int idx[3] = {ip - GHOST, jp - GHOST, kp - GHOST};
    const int n[3] = {g.nx, g.ny, g.nz};
    int src[3];
    int flip[3] = {0, 0, 0};
    bool ghost = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int s = idx[d];
        // periodic wraps modulo n (the ghost layers may be deeper than the
        // grid); reflective needs n >= GHOST (checked at creation)
        if (s < 0) {
            ghost = true;
            if (g.bc[2 * d] == 0) s = ((s % n[d]) + n[d]) % n[d];
            else if (g.bc[2 * d] == 2) s = 0;
            else { s = -1 - s; flip[d] = 1; }
        } else if (s >= n[d]) {
            ghost = true;
            if (g.bc[2 * d + 1] == 0) s = s % n[d];
            else if (g.bc[2 * d + 1] == 2) s = n[d] - 1;
            else { s = 2 * n[d] - 1 - s; flip[d] = 1; }
        }
        src[d] = s;
    }
    if (!ghost) return;
    const long long from = pidx(g, src[0], src[1], src[2]);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        double val = Q[v * g.pstride + from];
        if (v >= 1 && v <= 3 && flip[v - 1]) val = -val;
        Q[v * g.pstride + t] = val;
    }
}

// t: padded linear index
__device__ __forceinline__ void halo_item(double *__restrict__ Q, const Geo &g, long long t)
{
    if (t >= g.pstride) return;
    int ip, jp, kp;
    split3(t, g.px, g.py, ip, jp, kp);
    halo_cell(Q, g, ip, jp, kp);
}

// ghost cells of the padded box, numbered u = 0 .. ghost_count - 1: the
// z-slabs (the GHOST whole padded planes below and above the interior),
// then the y-slabs of the interior planes (GHOST whole padded rows below and
// above the interior rows), then the x-slabs of the interior rows (GHOST
// cells at each end); (ip, jp, kp) padded coordinates
__device__ __forceinline__ long long ghost_count(const Geo &g)
{
    return g.pstride - (long long)g.nx * g.ny * g.nz;
}
__device__ __forceinline__ void ghost_cell(const Geo &g, long long u, int &ip, int &jp, int &kp)
{
    const unsigned G2 = 2u * GHOST, px = (unsigned)g.px, py = (unsigned)g.py;
    const long long zs = (long long)G2 * py * px, ys = (long long)G2 * px * g.nz;
    if (u < zs) {
        const unsigned uu = (unsigned)u, plane = px * py;
        const unsigned kk = uu / plane, r = uu - kk * plane, j = r / px;
        ip = (int)(r - j * px);
        jp = (int)j;
        kp = kk < GHOST ? (int)kk : g.nz + (int)kk;
    } else if (u < zs + ys) {
        const unsigned uu = (unsigned)(u - zs), rows = G2 * px;
        const unsigned k = uu / rows, r = uu - k * rows, jj = r / px;
        ip = (int)(r - jj * px);
        jp = jj < GHOST ? (int)jj : g.ny + (int)jj;
        kp = (int)k + GHOST;
    } else {
        const unsigned uu = (unsigned)(u - zs - ys), jk = uu / G2, ii = uu - jk * G2;
        const unsigned k = jk / (unsigned)g.ny, j = jk - k * (unsigned)g.ny;
        ip = ii < GHOST ? (int)ii : g.nx + (int)ii;
        jp = (int)j + GHOST;
        kp = (int)k + GHOST;
    }
}

// dQ of the 18 big-stencil neighbours of cell (i,j,k), formed in FP64
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

// The mixed path's split state: Q = Q_hi + Q_lo with Q_hi = fl32(Q) and
// Q_lo = fl32(Q - Q_hi) (about 48 significant bits together).  A difference
// of neighbours formed as (hi_nb - hi_c) + (lo_nb - lo_c) in FP32 is the FP64
// difference to about one FP32 rounding: the hi part is exact for values
// within a factor 2 of each other (and otherwise rounds at the size of the
// result), the lo part is 2^-24 smaller.  The reconstruction then needs no
// FP64 arithmetic; the split is formed once per stage by k_split, from the
// bit fields of Q on the integer pipe (split_f64).
// SPLIT_PER: values per thread; a block of bs threads splits the
// SPLIT_PER bs consecutive values from b, value b + threadIdx.x + j bs in
// its j-th pass (coalesced, the SPLIT_PER loads of a thread independent, so
// that enough bytes are in flight to stream Q)
constexpr int SPLIT_PER = 4;
__device__ __forceinline__ void split_item(const double *__restrict__ Q, float *__restrict__ hi,
                                           float *__restrict__ lo, long long n, long long b)
{
    double q[SPLIT_PER];
#pragma unroll
    for (int j = 0; j < SPLIT_PER; ++j) {
        const long long t = b + threadIdx.x + (long long)j * blockDim.x;
        q[j] = t < n ? Q[t] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < SPLIT_PER; ++j) {
        const long long t = b + threadIdx.x + (long long)j * blockDim.x;
        if (t < n) {
            float h, l;
            split_f64(q[j], h, l);
            hi[t] = h;
            lo[t] = l;
        }
    }
}

// the stencil differences of one variable from the split state
__device__ __forceinline__ void load_stencil_split(const float *__restrict__ hv, const float *__restrict__ lv,
                                                   const Geo &g, int i, int j, int k, Stencil<float> &st)
{
    const long long sd[3] = {1, g.px, (long long)g.px * g.py};
    const long long c = pidx(g, i, j, k);
    const float hc = hv[c], lc = lv[c];
    auto diff = [&](long long at) { return (hv[at] - hc) + (lv[at] - lc); };
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.f[d][0] = diff(c - sd[d]);
        st.f[d][1] = diff(c + sd[d]);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const long long a = sd[p], b = sd[(p + 1) % 3];
#pragma unroll
        for (int sa = 0; sa < 2; ++sa)
#pragma unroll
            for (int sb = 0; sb < 2; ++sb) st.e[p][sa][sb] = diff(c + (sa ? a : -a) + (sb ? b : -b));
    }
}

__device__ __forceinline__ void load_stencil_split_far(const float *__restrict__ hv, const float *__restrict__ lv,
                                                       const Geo &g, int i, int j, int k, Stencil<float> &st)
{
    const long long sd[3] = {1, g.px, (long long)g.px * g.py};
    const long long c = pidx(g, i, j, k);
    const float hc = hv[c], lc = lv[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.f2[d][0] = (hv[c - 2 * sd[d]] - hc) + (lv[c - 2 * sd[d]] - lc);
        st.f2[d][1] = (hv[c + 2 * sd[d]] - hc) + (lv[c + 2 * sd[d]] - lc);
    }
}

// the six axis cells two steps away, for S' (formed in FP64 like the rest)
template <typename R>
__device__ __forceinline__ void load_stencil_far(const double *__restrict__ Qv, const Geo &g, int i, int j, int k,
                                                 double qc, Stencil<R> &st)
{
    const long long sd[3] = {1, g.px, (long long)g.px * g.py};
    const long long c = pidx(g, i, j, k);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.f2[d][0] = R(Qv[c - 2 * sd[d]] - qc);
        st.f2[d][1] = R(Qv[c + 2 * sd[d]] - qc);
    }
}

// literal positivity check (Sec. 4): rho and p of every P_m, m = 0..24, at
// every one of the cell's 24 Gauss points
template <typename R>
__device__ __noinline__ bool positivity_violated(const double *__restrict__ Q, const Geo &g, int i, int j, int k,
                                                 R gamma)
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
            for (int v = 0; v < 5; ++v)
                W[v] = qcv[v] + (m == 0 ? poly9(cf[v], X) : cf[v][0] * X[0] + cf[v][1] * X[1] + cf[v][2] * X[2]);
            if (W[0] < R(0) || pressure_negative(W)) return true;
        }
    }
    return false;
}

// the same literal check with S' and its 8 sub-stencils
template <typename R>
__device__ __noinline__ bool positivity_violated_sp(const double *__restrict__ Q, const Geo &g, int i, int j, int k,
                                                    R gamma)
{
    R qcv[5];
    Stencil<R> st[5];
    for (int v = 0; v < 5; ++v) {
        const double qc = Q[v * g.pstride + pidx(g, i, j, k)];
        qcv[v] = R(qc);
        load_stencil(Q + v * g.pstride, g, i, j, k, qc, st[v]);
        load_stencil_far(Q + v * g.pstride, g, i, j, k, qc, st[v]);
    }
    for (int m = 0; m <= 8; ++m) {
        R cf[5][9];
        for (int v = 0; v < 5; ++v) {
            if (m == 0) {
                big_stencil_P0_sp(st[v], cf[v]);
            } else {
                R b[3];
                sub_stencil_sp_rt(st[v], m - 1, b);
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
            for (int v = 0; v < 5; ++v)
                W[v] = qcv[v] + (m == 0 ? poly9(cf[v], X) : cf[v][0] * X[0] + cf[v][1] * X[1] + cf[v][2] * X[2]);
            if (W[0] < R(0) || pressure_negative(W)) return true;
        }
    }
    return false;
}

// WENO-AO reconstruction (Sec. 2) of one cell of the (n+2)^3 box, t its
// linear index there; writes Q_c and the 9 coefficients of P~ - Q_c per
// variable, and the positivity flag
// SPLIT: leave the literal positivity check to positivity_item (a kernel of
// its own, whose register demand then does not weigh on this one) and mark
// the cells whose bound is inconclusive with flag 2
// QS (mixed path): the differences come from the split state Qsplit,
// [hi: 5][pstride] then [lo: 5][pstride]
// rec: where cell t's record (Rec<R> layout) goes, a shared-memory stage
// that store_records copies out
template <typename R, bool SPLIT = false, bool QS = false>
__device__ __forceinline__ void recon_item(const double *__restrict__ Q, R *__restrict__ rec,
                                           unsigned char *__restrict__ flag, const Geo &g, const Scheme &S, Ctl *ctl,
                                           long long t, const float *__restrict__ Qsplit = nullptr,
                                           int *__restrict__ list = nullptr)
{
    if (t >= g.cstride) return;
    int i, j, k;
    split3(t, g.cx, g.cy, i, j, k);
    i -= 1;
    j -= 1;
    k -= 1;
    R rad[5], qcv[5];
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + v * g.pstride;
        Stencil<R> st;
        double qc;
        if constexpr (sizeof(R) == 4 && QS) {
            const float *hv = Qsplit + v * g.pstride, *lv = Qsplit + (5 + v) * g.pstride;
            qc = double(hv[pidx(g, i, j, k)]);  // fl32(Q_c), the value stored below
            load_stencil_split(hv, lv, g, i, j, k, st);
            if (S.sprime) load_stencil_split_far(hv, lv, g, i, j, k, st);
        } else {
            qc = Qv[pidx(g, i, j, k)];
            load_stencil(Qv, g, i, j, k, qc, st);
            if (S.sprime) load_stencil_far(Qv, g, i, j, k, qc, st);
        }
        qcv[v] = R(qc);
        R out[9];
        if (S.sprime) weno_ao_sp(st, S, out, rad[v]);
        else weno_ao(st, S, out, rad[v]);
        rec[v * Rec<R>::VS] = R(qc);
#pragma unroll
        for (int n = 0; n < 9; ++n) rec[v * Rec<R>::VS + 1 + n] = out[n];
    }
    // positivity fallback: the cheap sufficient test first, the literal
    // check of all 25 polynomials at the 24 Gauss points only when it fails
    if (SPLIT) {
        // mark the cells the bound cannot certify and append them to the list
        // of the literal check (one atomic per group of converged lanes)
        const bool marked = S.limiter && !positivity_certain(qcv, rad, fluxk<R>(S).gamma);
        flag[t] = marked ? 2 : 0;
        const unsigned act = __activemask();
        const unsigned m = __ballot_sync(act, marked);
        if (m) {
            const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&ctl->nmarked, (unsigned)__popc(m));
            base = __shfl_sync(act, base, leader);
            if (marked) list[base + __popc(m & ((1u << lane) - 1u))] = (int)t;
        }
        return;
    }
    bool bad = false;
    if (S.limiter && !positivity_certain(qcv, rad, fluxk<R>(S).gamma))
        bad = S.sprime ? positivity_violated_sp<R>(Q, g, i, j, k, fluxk<R>(S).gamma)
                       : positivity_violated<R>(Q, g, i, j, k, fluxk<R>(S).gamma);
    if (bad) {
        for (int v = 0; v < 5; ++v)
            for (int n = 1; n < 10; ++n) rec[v * Rec<R>::VS + n] = R(0);
        atomicAdd(&ctl->flagged, 1);
    }
    flag[t] = bad ? 1 : 0;
}

// The records of a block's consecutive cells [b, b + n), staged in shared
// memory (one record per thread, the global layout), copied out with 16-byte
// stores: coalesced, where each thread storing its own record would touch a
// sector per value.  Every thread of the block calls this after the stage
// is written (it synchronises the block).
template <typename R>
__device__ __forceinline__ void store_records(R *__restrict__ coef, const R *stage, long long b, int n)
{
    __syncthreads();
    constexpr int PER = 16 / sizeof(R);
    const int total = n * (Rec<R>::N / PER);
    const int4 *src = reinterpret_cast<const int4 *>(stage);
    int4 *dst = reinterpret_cast<int4 *>(coef + b * Rec<R>::N);
    for (int e = threadIdx.x; e < total; e += blockDim.x) dst[e] = src[e];
    __syncthreads();
}

// The literal positivity check (Sec. 4) of the cells marked 2 by
// recon_item<R, true>: rho and p of every candidate polynomial (P0 and the
// linear P_m: 24 for S, 8 for S') at every one of the cell's 24 face Gauss
// points.  The marked cells are listed by the reconstruction (list[0 ..
// ctl->nmarked)); one warp takes one listed cell at a time, the warps
// striding over the list.  Per cell the warp stages the stencil
// differences in shared memory once; lane m < nsub builds the linear P_m
// and the warp checks them face by face, stopping at the first violation
// anywhere in the warp (most marked cells at a discontinuity violate);
// only a cell that passes them has P0 built (one lane per variable, into
// shared memory) and checked, one Gauss point per lane.  A violation sets
// P~ to the cell average.  Every polynomial's arithmetic is that of
// sub_stencil / big_stencil_P0 on the same differences, and the same
// (polynomial, point) pairs decide.
template <typename R> struct PosStage {
    R d[5][24];  // dQ per variable: f[dim][-/+] at 2 dim + s, e[plane][sa][sb] at 6 + 4 plane + 2 sa + sb,
                 // the far axis cells of S' at 18 + 2 dim + s
    R qc[5];
    R a0[5][9];  // P0 of each variable
};

// value of X at a Gauss point: face-normal axis d at xd, then (d+1)%3 at xa, (d+2)%3 at xb
template <typename R> __device__ __forceinline__ void gauss_point_frame(int d, R xd, R xa, R xb, R X[3])
{
    X[0] = d == 0 ? xd : (d == 1 ? xb : xa);
    X[1] = d == 0 ? xa : (d == 1 ? xd : xb);
    X[2] = d == 0 ? xb : (d == 1 ? xa : xd);
}

template <typename R>
__device__ __forceinline__ void positivity_list(const double *__restrict__ Q, R *__restrict__ coef,
                                                unsigned char *__restrict__ flag, const Geo &g, const Scheme &S,
                                                Ctl *ctl, const int *__restrict__ list, PosStage<R> &sm,
                                                long long warp, long long nwarps)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nsub = S.sprime ? 8 : 24;
    const int nslot = S.sprime ? 24 : 18;
    const long long sx = 1, sy = g.px, sz = (long long)g.px * g.py;
    const long long nmarked = ctl->nmarked;
    for (long long e = warp; e < nmarked; e += nwarps) {
        const long long t = list[e];
        int i, j, k;
        split3(t, g.cx, g.cy, i, j, k);
        const long long c = pidx(g, i - 1, j - 1, k - 1);
        // stage: lane L < nslot forms dQ of stencil slot L for the 5 variables
        if (lane < nslot) {
            long long off;
            if (lane < 6) {
                const int dd = lane >> 1;
                const long long st = dd == 0 ? sx : (dd == 1 ? sy : sz);
                off = (lane & 1) ? st : -st;
            } else if (lane < 18) {
                const int q = lane - 6, pl = q >> 2;
                const long long sa = pl == 0 ? sx : (pl == 1 ? sy : sz);
                const long long sb = pl == 0 ? sy : (pl == 1 ? sz : sx);
                off = ((q & 2) ? sa : -sa) + ((q & 1) ? sb : -sb);
            } else {
                const int dd = (lane - 18) >> 1;
                const long long st = dd == 0 ? sx : (dd == 1 ? sy : sz);
                off = (lane & 1) ? 2 * st : -2 * st;
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const double *Qv = Q + v * g.pstride;
                sm.d[v][lane] = R(Qv[c + off] - Qv[c]);
            }
        } else if (lane >= 24 && lane < 29) {
            sm.qc[lane - 24] = R(Q[(lane - 24) * g.pstride + c]);
        }
        __syncwarp();
        R qcv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qcv[v] = sm.qc[v];
        // the linear P_m, m = lane
        R b[5][3];
        if (lane < nsub) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                if (S.sprime) {
                    const int sxp = (lane & 1) ? 0 : 1, syp = (lane & 2) ? 0 : 1, szp = (lane & 4) ? 0 : 1;
                    b[v][0] = sxp ? sm.d[v][1] : -sm.d[v][0];
                    b[v][1] = syp ? sm.d[v][3] : -sm.d[v][2];
                    b[v][2] = szp ? sm.d[v][5] : -sm.d[v][4];
                } else {
                    const int pl = lane >> 3, sg = lane & 7;
                    const int sa = (sg & 1) ? 0 : 1, sb = (sg & 2) ? 0 : 1, sc = (sg & 4) ? 0 : 1;
                    const int a = pl, bb = (pl + 1) % 3, cc = (pl + 2) % 3;
                    const R qa = sm.d[v][2 * a + sa], qb = sm.d[v][2 * bb + sb];
                    const R qab = sm.d[v][6 + 4 * pl + 2 * sa + sb], qcc = sm.d[v][2 * cc + sc];
                    const R ba = (R(2) * qa - qb + qab) * R(1.0 / 3.0);
                    const R bbv = (R(2) * qb - qa + qab) * R(1.0 / 3.0);
                    const R va = sa ? ba : -ba, vb = sb ? bbv : -bbv, vc = sc ? qcc : -qcc;
                    b[v][0] = a == 0 ? va : (bb == 0 ? vb : vc);
                    b[v][1] = a == 1 ? va : (bb == 1 ? vb : vc);
                    b[v][2] = a == 2 ? va : (bb == 2 ? vb : vc);
                }
            }
        }
        bool bad = false;
#pragma unroll 1
        for (int fc = 0; fc < 6; ++fc) {
            if (lane < nsub) {
#pragma unroll
                for (int gp = 0; gp < 4; ++gp) {
                    R X[3];
                    gauss_point_frame<R>(fc >> 1, (fc & 1) ? R(0.5) : R(-0.5), (gp & 2) ? R(GAUSS_S) : R(-GAUSS_S),
                                         (gp & 1) ? R(GAUSS_S) : R(-GAUSS_S), X);
                    R W[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v)
                        W[v] = qcv[v] + (b[v][0] * X[0] + b[v][1] * X[1] + b[v][2] * X[2]);
                    if (W[0] < R(0) || pressure_negative(W)) bad = true;
                }
            }
            if (__any_sync(FULL, bad)) {
                bad = true;
                break;
            }
        }
        if (!bad) {
            // P0: lane v < 5 builds variable v, then lane gq < 24 checks Gauss point gq
            if (lane < 5) {
                Stencil<R> st;
#pragma unroll
                for (int dd = 0; dd < 3; ++dd) {
                    st.f[dd][0] = sm.d[lane][2 * dd];
                    st.f[dd][1] = sm.d[lane][2 * dd + 1];
                    st.f2[dd][0] = S.sprime ? sm.d[lane][18 + 2 * dd] : R(0);
                    st.f2[dd][1] = S.sprime ? sm.d[lane][19 + 2 * dd] : R(0);
                }
#pragma unroll
                for (int pl = 0; pl < 3; ++pl)
#pragma unroll
                    for (int q = 0; q < 4; ++q) st.e[pl][q >> 1][q & 1] = sm.d[lane][6 + 4 * pl + q];
                R a[9];
                if (S.sprime) big_stencil_P0_sp(st, a);
                else big_stencil_P0(st, a);
#pragma unroll
                for (int n = 0; n < 9; ++n) sm.a0[lane][n] = a[n];
            }
            __syncwarp();
            if (lane < 24) {
                const int gq = lane;
                R X[3];
                gauss_point_frame<R>(gq / 8, ((gq / 4) & 1) ? R(0.5) : R(-0.5),
                                     ((gq >> 1) & 1) ? R(GAUSS_S) : R(-GAUSS_S), (gq & 1) ? R(GAUSS_S) : R(-GAUSS_S),
                                     X);
                R W[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    R a[9];
#pragma unroll
                    for (int n = 0; n < 9; ++n) a[n] = sm.a0[v][n];
                    W[v] = qcv[v] + poly9(a, X);
                }
                if (W[0] < R(0) || pressure_negative(W)) bad = true;
            }
            bad = __any_sync(FULL, bad);
        }
        if (lane == 0) {
            if (bad) {
                for (int v = 0; v < 5; ++v)
                    for (int n = 1; n < 10; ++n) coef[rec_idx<R>(t, v, n)] = R(0);
                atomicAdd(&ctl->flagged, 1);
            }
            flag[t] = bad ? 1 : 0;
        }
        __syncwarp();  // the stage is rewritten for the next cell
    }
}

// ---------------------------------------------------------------------------
// Face flux: one Gauss point per call, 4 consecutive lanes per face (all 4
// must call together: the Gauss sum uses warp shuffles).  The local frame of
// a face normal to axis D is (e_D, e_{D+1}, e_{D+2}) (the printed frame for
// D = x, and its cyclic images).  The stored value is the face-averaged flux
// per unit area, F and dF/dt, in FP64.  t: 4 * face + Gauss point; t beyond
// the faces computes a clamped face and writes nothing.
// ---------------------------------------------------------------------------
// the 10 values of variable v of a uniform-mesh record (Rec<R>) by vector loads
__device__ __forceinline__ void load_rec_var(const float *__restrict__ rec, int v, float &q0, float c[9])
{
    const float4 *p = reinterpret_cast<const float4 *>(rec + v * Rec<float>::VS);
    const float4 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2);
    q0 = a.x;
    c[0] = a.y; c[1] = a.z; c[2] = a.w;
    c[3] = b.x; c[4] = b.y; c[5] = b.z; c[6] = b.w;
    c[7] = d.x; c[8] = d.y;
}
__device__ __forceinline__ void load_rec_var(const double *__restrict__ rec, int v, double &q0, double c[9])
{
    const double2 *p = reinterpret_cast<const double2 *>(rec + v * Rec<double>::VS);
    const double2 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2), e = __ldg(p + 3), f = __ldg(p + 4);
    q0 = a.x;
    c[0] = a.y; c[1] = b.x; c[2] = b.y; c[3] = d.x; c[4] = d.y;
    c[5] = e.x; c[6] = e.y; c[7] = f.x; c[8] = f.y;
}

// REC: coef is the cell's record (Rec<R>); otherwise one array per slot
// with term stride `stride` and the cell at ci
template <typename R, int D, bool REC = false>
__device__ __forceinline__ void eval_side(const R *__restrict__ coef, long long stride, long long ci, R xd, R xa,
                                          R xb, R W[5], R dW[3][5])
{
    // at a face Gauss point the face-normal coordinate is xd = +-1/2 and the
    // tangential ones are +-1/(2 sqrt 3), so the zero-mean tangential squares
    // X_A^2 - 1/12 and X_B^2 - 1/12 vanish and X_D^2 - 1/12 = 1/6
    constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
    constexpr int DA = D + A == 1 ? 6 : (D + A == 2 ? 7 : 8);
    constexpr int DB = D + B == 1 ? 6 : (D + B == 2 ? 7 : 8);
    constexpr int AB = A + B == 1 ? 6 : (A + B == 2 ? 7 : 8);
    // point factors shared by the five variables; the sums below are chains
    // of multiply-adds.  The gradients stay in the scaled frame (derivatives
    // per cell edge): the flux takes the factor 1/h with its slope data.
    const R xab = xa * xb, xd2 = R(2) * xd, xa2 = R(2) * xa, xb2 = R(2) * xb;
    R val[5], grad[5][3];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        R c[9], e;
        if constexpr (REC) {
            load_rec_var(coef, v, e, c);
        } else {
#pragma unroll
            for (int n = 0; n < 9; ++n) c[n] = coef[coef_slot(v, 1 + n) * stride + ci];
            e = coef[coef_slot(v, 0) * stride + ci];
        }
        e += c[D] * xd;
        e += c[3 + D] * R(1.0 / 6.0);
        e += xa * (c[A] + c[DA] * xd);
        e += xb * (c[B] + c[DB] * xd);
        e += c[AB] * xab;
        val[v] = e;
        e = c[D];
        e += c[3 + D] * xd2;
        e += c[DA] * xa;
        e += c[DB] * xb;
        grad[v][D] = e;
        e = c[A];
        e += c[3 + A] * xa2;
        e += c[DA] * xd;
        e += c[AB] * xb;
        grad[v][A] = e;
        e = c[B];
        e += c[3 + B] * xb2;
        e += c[DB] * xd;
        e += c[AB] * xa;
        grad[v][B] = e;
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

// resident blocks of 128 threads per SM asked of the compiler for the
// single-instance face flux kernel.  FP64: no hint (238 registers, 2
// blocks; 3 blocks with 168 registers and spills measured slower).  FP32: 5
// blocks (96 registers, 56 bytes spilled), measured on the TGV 128^3 step
// at 3.02 ms of flux against 3.20 ms at 4 blocks (128 registers), 3.23 ms
// at 6 and 3.60 ms at 3.  (The batched flux kernel, with its tile loop,
// spills more at 96 registers and runs faster without the hint.)
template <typename R> struct FluxOcc { static constexpr int blocks = 1; };
template <> struct FluxOcc<float> { static constexpr int blocks = 5; };

template <int D> __device__ __forceinline__ long long face_count(const Geo &g)
{
    return (long long)(g.nx + (D == 0)) * (g.ny + (D == 1)) * (g.nz + (D == 2));
}

// CH: the polynomials are per (face, side) in the layout of hgks_char.cuh
// ([side][slot][face], coef pointing at the axis's array) instead of per cell
template <typename R, int D, bool CH = false>
__device__ __forceinline__ void flux_item(const R *__restrict__ coef, double *__restrict__ Fout, const Geo &g,
                                          const Scheme &S, double dt, long long t, long long tlimit = LLONG_MAX)
{
    const int ex = g.nx + (D == 0), ey = g.ny + (D == 1);
    const long long nface = face_count<D>(g);
    long long face = t >> 2;
    const int gp = (int)(t & 3);
    const bool valid = face < nface && t < tlimit;
    if (!valid) face = nface - 1;
    // (i, j, k) is the right cell; the left cell is one step back along D;
    // the face index decoded with the precomputed divisors of ex and ey
    int i, j, k;
    {
        const unsigned u = (unsigned)face;
        const unsigned r = div32(u, g.dv[D == 0 ? 1 : 0]);
        i = (int)(u - r * (unsigned)ex);
        k = (int)div32(r, g.dv[D == 1 ? 3 : 2]);
        j = (int)(r - (unsigned)k * (unsigned)ey);
    }
    const int il = i - (D == 0), jl = j - (D == 1), kl = k - (D == 2);
    const R xa = (gp & 2) ? R(GAUSS_S) : R(-GAUSS_S);
    const R xb = (gp & 1) ? R(GAUSS_S) : R(-GAUSS_S);
    R Wl[5], dWl[3][5], Wr[5], dWr[3][5];
    if (CH) {
        eval_side<R, D>(coef, nface, face, R(0.5), xa, xb, Wl, dWl);
        eval_side<R, D>(coef + 50 * nface, nface, face, R(-0.5), xa, xb, Wr, dWr);
    } else {
        eval_side<R, D, true>(coef + cidx(g, il, jl, kl) * Rec<R>::N, 0, 0, R(0.5), xa, xb, Wl, dWl);
        eval_side<R, D, true>(coef + cidx(g, i, j, k) * Rec<R>::N, 0, 0, R(-0.5), xa, xb, Wr, dWr);
    }
    R F[5], dF[5];
    gks_flux<R>(Wl, dWl, Wr, dWr, S, R(dt), F, dF, R(g.inv_h));
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
    // every lane of the face holds the sums; lane gp stores q = gp, gp + 4,
    // gp + 8, so the FP64 conversions are spread over the 4 lanes
    if (valid) {
        const bool b0 = gp & 1, b1 = gp & 2;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const R v = b1 ? (b0 ? f[4 * r + 3] : f[4 * r + 2]) : (b0 ? f[4 * r + 1] : f[4 * r]);
            Fout[(gp + 4 * r) * nface + face] = double(v);
        }
        if (!b1) Fout[(gp + 8) * nface + face] = double(b0 ? f[9] : f[8]);
    }
}

// ---------------------------------------------------------------------------
// update: L = -(1/h) sum over the 3 axes of (F_upper - F_lower) with the
// face-averaged fluxes, and the two-stage fourth-order combination (Sec. 3)
// ---------------------------------------------------------------------------
// S = sum over the 3 axes of (F_upper - F_lower) (and of dF/dt), so that
// L = -S/h; NV = 5 gives the dF/dt sums only
template <int NV = 10>
__device__ __forceinline__ void cell_face_sums(const double *__restrict__ Fx, const double *__restrict__ Fy,
                                               const double *__restrict__ Fz, const Geo &g, int i, int j, int k,
                                               double Sm[5], double dSm[5])
{
    const long long nfx = (long long)(g.nx + 1) * g.ny * g.nz;
    const long long nfy = (long long)g.nx * (g.ny + 1) * g.nz;
    const long long nfz = (long long)g.nx * g.ny * (g.nz + 1);
    const long long fx0 = ((long long)k * g.ny + j) * (g.nx + 1) + i;
    const long long fy0 = ((long long)k * (g.ny + 1) + j) * g.nx + i;
    const long long fz0 = ((long long)k * g.ny + j) * g.nx + i;
    const long long fzs = (long long)g.nx * g.ny;
#pragma unroll
    for (int v = 10 - NV; v < 10; ++v) {
        const double sx = Fx[v * nfx + fx0 + 1] - Fx[v * nfx + fx0];
        const double sy = Fy[v * nfy + fy0 + g.nx] - Fy[v * nfy + fy0];
        const double sz = Fz[v * nfz + fz0 + fzs] - Fz[v * nfz + fz0];
        if (v < 5) Sm[v] = sx + sy + sz;
        else dSm[v - 5] = sx + sy + sz;
    }
}

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

// one interior cell (t < ncell) of the stage update; the call for t = 0 of
// stage 2 also advances the instance's time and step count
template <int STAGE>
__device__ __forceinline__ void update_item(double *__restrict__ Qn, double *__restrict__ Qs,
                                            double *__restrict__ Wacc, const double *__restrict__ Fx,
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
    // L = -S/h and dL/dt = -dS/h with the 1/h folded into the stage
    // constants (the update is FP64-pipe bound on GB300)
    double Sm[5], dSm[5];
    const double a = -dt * g.inv_h, b = a * dt;
    const long long pi = pidx(g, i, j, k);
    if (STAGE == 1) {
        cell_face_sums<10>(Fx, Fy, Fz, g, i, j, k, Sm, dSm);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double q = Qn[v * g.pstride + pi];
            Qs[v * g.pstride + pi] = q + (0.5 * a) * Sm[v] + (0.125 * b) * dSm[v];
            Wacc[v * g.ncell + t] = q + a * Sm[v] + (b * (1.0 / 6.0)) * dSm[v];
        }
    } else {
        cell_face_sums<5>(Fx, Fy, Fz, g, i, j, k, Sm, dSm);
        double W[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            W[v] = Wacc[v * g.ncell + t] + (b * (1.0 / 3.0)) * dSm[v];
            Qn[v * g.pstride + pi] = W[v];
        }
        // p > 0 with rho > 0 is 2 rho E > |rho U|^2 (no division)
        const double m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
        if (!(W[0] > 0.0) || !(2.0 * W[4] * W[0] > m2)) atomicOr(&ctl->status, 1);
        (void)gamma;
    }
}

// ---------------------------------------------------------------------------
// CFL: dt = cfl * min_cells h/(|U| + c).  cfl_value gives one cell's
// h/(|U| + c) (+inf beyond the cells, 0 for a nonphysical cell);
// block_min_to reduces over the block with warp shuffles and folds into the
// accumulator with an integer atomicMin on the bit pattern (positive
// doubles order like their bits): order-independent, so exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cfl_value(const double *__restrict__ Q, const Geo &g, double gamma, long long t)
{
    if (t >= g.ncell) return INFINITY;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    const long long pi = pidx(g, i, j, k);
    double W[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) W[q] = Q[q * g.pstride + pi];
    const double rho = W[0];
    const double m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
    const double speed = sqrt(m2) / rho;
    const double p = (gamma - 1.0) * (W[4] - 0.5 * m2 / rho);
    const double c = sqrt(gamma * p / rho);
    double v = g.h / (speed + c);
    if (!(v > 0.0)) v = 0.0;  // nonphysical: force dt = 0
    return v;
}

// the same candidate with the arithmetic in FP32 (the mixed path: FP32
// candidates, FP64 minimum); a cell whose FP32 pressure is not clearly
// positive is recomputed in FP64, so that round-off never reads as a
// nonphysical state
__device__ __forceinline__ double cfl_value_mixed(const double *__restrict__ Q, const Geo &g, double gamma,
                                                  long long t)
{
    if (t >= g.ncell) return INFINITY;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    const long long pi = pidx(g, i, j, k);
    float W[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) W[q] = float(Q[q * g.pstride + pi]);
    const float ir = 1.0f / W[0];
    const float m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
    const float p = float(gamma - 1.0) * (W[4] - 0.5f * m2 * ir);
    if (!(W[0] > 0.0f) || !(p > 1e-4f * W[4])) return cfl_value(Q, g, gamma, t);
    const float s = sqrtf(m2) * ir + sqrtf(float(gamma) * p * ir);
    return double(float(g.h) / s);
}

// all threads of the block call it (blockDim a multiple of 32, <= 1024)
__device__ __forceinline__ void block_min_to(double v, unsigned long long *acc)
{
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) atomicMin(acc, (unsigned long long)__double_as_longlong(v));
    }
}

// choose dt for this step and arm (or disarm) the stage kernels
__device__ __forceinline__ void dt_choose(Ctl *ctl, double cfl, double dt_fixed, double t_end)
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

}  // namespace hk
