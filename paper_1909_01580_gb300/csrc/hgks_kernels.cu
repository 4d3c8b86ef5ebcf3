// Kernels of the HGKS stage sweep on sm_103a (uniform mesh of cubes):
// ghost fill, WENO-AO reconstruction (Sec. 2), Gauss-point gas-kinetic
// face flux (Sec. 3), two-stage update and CFL reduction.
#include <algorithm>

#include "hgks_kernels.cuh"
#include "hgks_items.cuh"

namespace hk {

// one thread per ghost cell
__global__ void k_halo(double *__restrict__ Q, Geo g)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= ghost_count(g)) return;
    int ip, jp, kp;
    ghost_cell(g, u, ip, jp, kp);
    halo_cell(Q, g, ip, jp, kp);
}

// one thread per cell of the reconstruction box; the block's records are
// staged in dynamic shared memory (blockDim x Rec<R>::N values) and stored
// coalesced
template <typename R, bool QS>
__global__ void __launch_bounds__(128) k_recon(const double *__restrict__ Q, R *__restrict__ coef,
                                               unsigned char *__restrict__ flag, Geo g, Scheme S, Ctl *ctl,
                                               const float *__restrict__ Qsplit, int *__restrict__ list)
{
    if (!ctl->active) return;
    extern __shared__ int4 recon_stage_raw[];
    R *stage = reinterpret_cast<R *>(recon_stage_raw);
    const long long b = (long long)blockIdx.x * blockDim.x;
    recon_item<R, true, QS>(Q, stage + threadIdx.x * Rec<R>::N, flag, g, S, ctl, b + threadIdx.x, Qsplit, list);
    store_records<R>(coef, stage, b, (int)std::min<long long>(blockDim.x, g.cstride - b));
}

__global__ void k_split(const double *__restrict__ Q, float *__restrict__ hi, float *__restrict__ lo, long long n)
{
    split_item(Q, hi, lo, n, (long long)blockIdx.x * blockDim.x * SPLIT_PER);
}

// the literal positivity check of the listed cells: persistent warps that
// stride over the list, one cell per warp at a time
template <typename R>
__global__ void __launch_bounds__(128) k_positivity(const double *__restrict__ Q, R *__restrict__ coef,
                                                    unsigned char *__restrict__ flag, Geo g, Scheme S, Ctl *ctl,
                                                    const int *__restrict__ list)
{
    if (!ctl->active) return;
    __shared__ PosStage<R> stage[4];
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    positivity_list<R>(Q, coef, flag, g, S, ctl, list, stage[threadIdx.x >> 5], warp, nwarps);
}

template <typename R, int D>
__global__ void __launch_bounds__(128, FluxOcc<R>::blocks) k_face_flux(const R *__restrict__ coef, double *__restrict__ Fout, Geo g,
                                                   Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    flux_item<R, D>(coef, Fout, g, S, ctl->dt, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int STAGE>
__global__ void __launch_bounds__(256) k_update(double *__restrict__ Qn, double *__restrict__ Qs,
                                                double *__restrict__ Wacc, const double *__restrict__ Fx,
                                                const double *__restrict__ Fy, const double *__restrict__ Fz, Geo g,
                                                double gamma, Ctl *ctl)
{
    if (!ctl->active) return;
    update_item<STAGE>(Qn, Qs, Wacc, Fx, Fy, Fz, g, gamma, ctl, ctl->dt,
                       (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_residual(const double *__restrict__ Fx, const double *__restrict__ Fy,
                           const double *__restrict__ Fz, Geo g, double *__restrict__ L, double *__restrict__ dL)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    double l[5], dl[5];
    cell_residual(Fx, Fy, Fz, g, i, j, k, l, dl);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        L[v * g.ncell + t] = l[v];
        dL[v * g.ncell + t] = dl[v];
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(256) k_cfl(const double *__restrict__ Q, Geo g, double gamma, Ctl *ctl)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    block_min_to(MIXED ? cfl_value_mixed(Q, g, gamma, t) : cfl_value(Q, g, gamma, t), &ctl->minbits);
}

// one thread: choose dt for this step and arm the stage kernels
__global__ void k_dt(Ctl *ctl, double cfl, double dt_fixed, double t_end) { dt_choose(ctl, cfl, dt_fixed, t_end); }

// a fresh control block at time t (step count and status cleared)
__global__ void k_init_ctl(Ctl *ctl, double t)
{
    ctl->t = t;
    ctl->dt = 0.0;
    ctl->active = 0;
    ctl->status = 0;
    ctl->flagged = 0;
    ctl->steps_done = 0;
    ctl->minbits = (unsigned long long)__double_as_longlong(INFINITY);
}

// re-arm the stage kernels with dt (time and step count kept)
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
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    const long long pi = pidx(g, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) Q[v * g.pstride + pi] = src[v * g.ncell + t];
}
__global__ void k_gather(const double *__restrict__ Q, double *__restrict__ dst, Geo g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    const long long pi = pidx(g, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) dst[v * g.ncell + t] = Q[v * g.pstride + pi];
}

// coefficients of the interior cells to FP64 [ncell][5][9]
// (rec: the uniform mesh's per-cell records; otherwise one array per slot)
template <typename R>
__global__ void k_export_coef(const R *__restrict__ coef, const unsigned char *__restrict__ flag, Geo g,
                              double *__restrict__ out, int *__restrict__ oflag, bool rec)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    const long long ci = cidx(g, i, j, k);
    for (int v = 0; v < 5; ++v)
        for (int n = 0; n < 9; ++n)
            out[t * 45 + v * 9 + n] = double(rec ? coef[rec_idx<R>(ci, v, 1 + n)] : coef[mrec_idx<R>(ci, v, 1 + n)]);
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

// multiprocessors of the current device (cached per device)
static int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cache[dev] = n;
    }
    return cache[dev];
}

void launch_halo(double *Q, const Geo &g, cudaStream_t s)
{
    k_halo<<<blocks_for(g.pstride - (long long)g.nx * g.ny * g.nz, 256), 256, 0, s>>>(Q, g);
}

template <typename R>
void launch_recon(const double *Q, R *coef, unsigned char *flag, const Geo &g, const Scheme &S, Ctl *ctl,
                  cudaStream_t s, int *list, float *split)
{
    cudaMemsetAsync(&ctl->nmarked, 0, sizeof(unsigned), s);
    if (split) {
        const long long n = 5 * g.pstride;
        k_split<<<blocks_for(n, 256 * SPLIT_PER), 256, 0, s>>>(Q, split, split + n, n);
    }
    const int smem = 128 * Rec<R>::N * (int)sizeof(R);  // 30 KB FP32, 50 KB FP64 (opted in at first use)
    // the attribute is per device: set once per device and kernel
    static bool opted[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !opted[dev][split ? 1 : 0]) {
        if (split) cudaFuncSetAttribute(k_recon<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        else cudaFuncSetAttribute(k_recon<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (dev >= 0 && dev < 64) opted[dev][split ? 1 : 0] = true;
    }
    if (split) k_recon<R, true><<<blocks_for(g.cstride, 128), 128, smem, s>>>(Q, coef, flag, g, S, ctl, split, list);
    else k_recon<R, false><<<blocks_for(g.cstride, 128), 128, smem, s>>>(Q, coef, flag, g, S, ctl, nullptr, list);
    // persistent: 8 blocks of 4 warps per SM stride over the list of marked cells
    k_positivity<R><<<8u * (unsigned)sm_count(), 128, 0, s>>>(Q, coef, flag, g, S, ctl, list);
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

void launch_cfl(const double *Q, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s, bool mixed)
{
    if (mixed) k_cfl<true><<<blocks_for(g.ncell, 256), 256, 0, s>>>(Q, g, gamma, ctl);
    else k_cfl<false><<<blocks_for(g.ncell, 256), 256, 0, s>>>(Q, g, gamma, ctl);
}

void launch_dt(Ctl *ctl, double cfl, double dt_fixed, double t_end, cudaStream_t s)
{
    k_dt<<<1, 1, 0, s>>>(ctl, cfl, dt_fixed, t_end);
}

void launch_init_ctl(Ctl *ctl, double t, cudaStream_t s) { k_init_ctl<<<1, 1, 0, s>>>(ctl, t); }

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
                        cudaStream_t s, bool rec)
{
    k_export_coef<R><<<blocks_for(g.ncell, 128), 128, 0, s>>>(coef, flag, g, out, oflag, rec);
}

template <typename R>
void launch_point_flux(int n, const double *in, const double *ug, double dt, const Scheme &S, double *F, double *dF,
                       cudaStream_t s)
{
    k_point_flux<R><<<blocks_for(n, 64), 64, 0, s>>>(n, in, ug, dt, S, F, dF);
}

template void launch_recon<double>(const double *, double *, unsigned char *, const Geo &, const Scheme &, Ctl *,
                                   cudaStream_t, int *, float *);
template void launch_recon<float>(const double *, float *, unsigned char *, const Geo &, const Scheme &, Ctl *,
                                  cudaStream_t, int *, float *);
template void launch_flux<double>(int, const double *, double *, const Geo &, const Scheme &, Ctl *, cudaStream_t);
template void launch_flux<float>(int, const float *, double *, const Geo &, const Scheme &, Ctl *, cudaStream_t);
template void launch_export_coef<double>(const double *, const unsigned char *, const Geo &, double *, int *,
                                         cudaStream_t, bool);
template void launch_export_coef<float>(const float *, const unsigned char *, const Geo &, double *, int *,
                                        cudaStream_t, bool);
template void launch_point_flux<double>(int, const double *, const double *, double, const Scheme &, double *,
                                        double *, cudaStream_t);
template void launch_point_flux<float>(int, const double *, const double *, double, const Scheme &, double *,
                                       double *, cudaStream_t);

}  // namespace hk
