// Kernels of the stage sweep on mapped and moving meshes (item bodies in
// hgks_mapped.cuh).  The stage time is t_n (half = 0) or t_n + dt/2
// (half = 1), read from the control block.
#include "hgks_mapped.cuh"
#include "hgks_mapped_launch.cuh"

namespace hk {

__device__ __forceinline__ double stage_time(const Ctl *ctl, int half) { return ctl->t + (half ? 0.5 * ctl->dt : 0.0); }

// geometry of every cell of the padded box at the stage time (or at t_fixed
// when ctl is null); MIXED: the small quantities in FP32 (cell_geometry_mixed)
template <bool MIXED>
__global__ void __launch_bounds__(128) k_geom(double *__restrict__ geo, Geo g, MapGeo m, Ctl *ctl, int half,
                                              double t_fixed)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.pstride) return;
    int i, j, k;
    split3(t, g.px, g.py, i, j, k);
    i -= GHOST;
    j -= GHOST;
    k -= GHOST;
    const double ts = ctl ? stage_time(ctl, half) : t_fixed;
    const double Sf = map_factor(m, ts);
    if (ctl && t == 0) {
        // the map's time factors of this stage, for the reconstruction and
        // flux kernels that follow
        ctl->mapS = Sf;
        ctl->mapC = m.moving ? cos(m.omega * ts) : 0.0;
        ctl->mapAS = float(m.amp * Sf);
        ctl->mapAUC = float(m.amp * m.omega * ctl->mapC);
    }
    double rec[NGEO];
    if constexpr (MIXED) {
        float fm[GEOF];
        cell_geometry_mixed(m, i, j, k, float(m.amp * Sf), rec, fm);
#pragma unroll
        for (int e = 0; e < GEOF; ++e) m.geof[e * g.pstride + t] = fm[e];
    } else {
        cell_geometry(m, i, j, k, Sf, rec);
        if (m.geof) {
            const int idx[3] = {i, j, k};
#pragma unroll
            for (int e = 0; e < 6; ++e) m.geof[e * g.pstride + t] = float(rec[4 + e]);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                m.geof[(6 + d) * g.pstride + t] = float(rec[1 + d] - (m.lo[d] + ((double)idx[d] + 0.5) * m.h[d]));
        }
    }
#pragma unroll
    for (int e = 0; e < NGEO; ++e) geo[e * g.pstride + t] = rec[e];
}

__global__ void k_vol_from_geo(const double *__restrict__ geo, double *__restrict__ vol, Geo g)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    vol[t] = geo[pidx(g, i, j, k)];
}

// resident blocks per SM asked of the compiler for the mapped
// reconstruction: the FP32 kernel fits 6 (its shared-memory limit) in 168
// registers without spilling; the FP64 kernel (198 registers) runs 5
template <typename R> struct MapReconOcc { static constexpr int blocks = 1; };
template <> struct MapReconOcc<float> { static constexpr int blocks = 6; };

template <typename R>
__global__ void __launch_bounds__(RM_BS, MapReconOcc<R>::blocks) k_recon_mapped(const double *__restrict__ Q, const double *__restrict__ geo,
                                                        R *__restrict__ coef, unsigned char *__restrict__ flag, Geo g,
                                                        MapGeo m, Scheme S, Ctl *ctl, int half)
{
    __shared__ __align__(16) R stage[RmStage<R>::n * RM_BS];
    if (!ctl->active) return;
    const long long b = (long long)blockIdx.x * RM_BS;
    recon_mapped_item<R>(Q, geo, coef, flag, g, m, ctl->mapS, S, ctl, stage + threadIdx.x, b + threadIdx.x);
    if constexpr (RmStage<R>::dq) {
        // FP32: the block's records, staged by the item, copied out with
        // 16-byte coalesced stores
        static_assert(RM_BS * MRec<R>::N <= RmStage<R>::n * RM_BS, "the records fit the stage");
        __syncthreads();
        const int nrec = (int)(g.cstride - b < RM_BS ? g.cstride - b : RM_BS);
        const int4 *src = reinterpret_cast<const int4 *>(stage);
        int4 *dst = reinterpret_cast<int4 *>(coef + b * MRec<R>::N);
        for (int e = threadIdx.x; e < nrec * (MRec<R>::N * (int)sizeof(R) / 16); e += RM_BS) dst[e] = src[e];
    }
}

// split state Q = Q_hi + Q_lo of the stage's Q for the mixed reconstruction
__global__ void k_split_mapped(const double *__restrict__ Q, float *__restrict__ hi, float *__restrict__ lo,
                               long long n)
{
    split_item(Q, hi, lo, n, (long long)blockIdx.x * blockDim.x * SPLIT_PER);
}

template <typename R>
__global__ void __launch_bounds__(128) k_positivity_mapped(const double *__restrict__ Q, const double *__restrict__ geo,
                                                           R *__restrict__ coef, unsigned char *__restrict__ flag,
                                                           Geo g, MapGeo m, Scheme S, Ctl *ctl, int half)
{
    if (!ctl->active) return;
    positivity_mapped_item<R>(Q, geo, coef, flag, g, m, ctl->mapS, S, ctl,
                              (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// resident blocks of 128 threads per SM asked of the compiler for the mapped
// face flux: the FP32 kernel fits 4 in 128 registers without spilling
// (about 200 registers otherwise)
template <typename R> struct MapFluxOcc { static constexpr int blocks = 1; };
template <> struct MapFluxOcc<float> { static constexpr int blocks = 4; };

template <typename R, int D>
__global__ void __launch_bounds__(128, MapFluxOcc<R>::blocks) k_flux_mapped(const R *__restrict__ coef, double *__restrict__ Fout, Geo g,
                                                     MapGeo m, Scheme S, Ctl *ctl, int half)
{
    if (!ctl->active) return;
    flux_mapped_item<R, D>(coef, Fout, g, m, ctl->mapS, ctl->mapC, ctl->mapAS, ctl->mapAUC, S, ctl->dt,
                           (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int STAGE>
__global__ void __launch_bounds__(256) k_update_mapped(double *__restrict__ Qn, double *__restrict__ Qs,
                                                       double *__restrict__ Wacc, double *__restrict__ vol,
                                                       double *__restrict__ vnext, const double *__restrict__ Fx,
                                                       const double *__restrict__ Fy, const double *__restrict__ Fz,
                                                       Geo g, double gamma, Ctl *ctl)
{
    if (!ctl->active) return;
    update_mapped_item<STAGE>(Qn, Qs, Wacc, vol, vnext, Fx, Fy, Fz, g, gamma, ctl, ctl->dt,
                              (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// L = R/|Omega| and dL/dt with the geometric volumes of the stage geometry
__global__ void k_residual_mapped(const double *__restrict__ Fx, const double *__restrict__ Fy,
                                  const double *__restrict__ Fz, const double *__restrict__ geo, Geo g,
                                  double *__restrict__ L, double *__restrict__ dL)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i, j, k;
    split3(t, g.nx, g.ny, i, j, k);
    double Rr[5], dR[5], V;
    cell_residual_mapped(Fx, Fy, Fz, g, i, j, k, Rr, dR, V);
    const double vol = geo[pidx(g, i, j, k)];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        L[v * g.ncell + t] = Rr[v] / vol;
        dL[v * g.ncell + t] = dR[v] / vol;
    }
}

// CFL with h = |Omega|^(1/3) of the geometry at t_n; MIXED: FP32
// candidates (FP64 minimum), a cell whose FP32 pressure is not clearly
// positive recomputed in FP64
template <bool MIXED>
__global__ void __launch_bounds__(256) k_cfl_mapped(const double *__restrict__ Q, const double *__restrict__ geo,
                                                    Geo g, double gamma, Ctl *ctl)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = INFINITY;
    bool done = false;
    if (MIXED && t < g.ncell) {
        int i, j, k;
        split3(t, g.nx, g.ny, i, j, k);
        const long long pi = pidx(g, i, j, k);
        float W[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) W[q] = float(Q[q * g.pstride + pi]);
        const float ir = 1.0f / W[0];
        const float m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
        const float p = float(gamma - 1.0) * (W[4] - 0.5f * m2 * ir);
        if (W[0] > 0.0f && p > 1e-4f * W[4]) {
            const float s = sqrtf(m2) * ir + sqrtf(float(gamma) * p * ir);
            v = double(cbrtf(float(geo[pi])) / s);
            done = true;
        }
    }
    if (!done && t < g.ncell) {
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
        v = cbrt(geo[pi]) / (speed + c);
        if (!(v > 0.0)) v = 0.0;
    }
    block_min_to(v, &ctl->minbits);
}

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_geom(double *geo, const Geo &g, const MapGeo &m, Ctl *ctl, int half, double t_fixed,
                 cudaStream_t s)
{
    // a mixed handle's stage geometry in FP32 arithmetic; the FP64 geometry
    // for FP64 handles and for the initial volumes (ctl null)
    if (m.geof && ctl) k_geom<true><<<nblk(g.pstride, 128), 128, 0, s>>>(geo, g, m, ctl, half, t_fixed);
    else k_geom<false><<<nblk(g.pstride, 128), 128, 0, s>>>(geo, g, m, ctl, half, t_fixed);
}

void launch_vol_from_geo(const double *geo, double *vol, const Geo &g, cudaStream_t s)
{
    k_vol_from_geo<<<nblk(g.ncell, 256), 256, 0, s>>>(geo, vol, g);
}

template <typename R>
void launch_recon_mapped(const double *Q, const double *geo, R *coef, unsigned char *flag, const Geo &g,
                         const MapGeo &m, const Scheme &S, Ctl *ctl, int half, cudaStream_t s)
{
    if (sizeof(R) == 4 && m.qsplit) {
        const long long n = 5 * g.pstride;
        k_split_mapped<<<nblk(n, 256 * SPLIT_PER), 256, 0, s>>>(Q, (float *)m.qsplit, (float *)m.qsplit + n, n);
    }
    k_recon_mapped<R><<<nblk(g.cstride, RM_BS), RM_BS, 0, s>>>(Q, geo, coef, flag, g, m, S, ctl, half);
    k_positivity_mapped<R><<<nblk(g.cstride, 128), 128, 0, s>>>(Q, geo, coef, flag, g, m, S, ctl, half);
}

template <typename R>
void launch_flux_mapped(int axis, const R *coef, double *F, const Geo &g, const MapGeo &m, const Scheme &S, Ctl *ctl,
                        int half, cudaStream_t s)
{
    const long long nface = (long long)(g.nx + (axis == 0)) * (g.ny + (axis == 1)) * (g.nz + (axis == 2));
    const unsigned nb = nblk(4 * nface, 128);
    if (axis == 0) k_flux_mapped<R, 0><<<nb, 128, 0, s>>>(coef, F, g, m, S, ctl, half);
    else if (axis == 1) k_flux_mapped<R, 1><<<nb, 128, 0, s>>>(coef, F, g, m, S, ctl, half);
    else k_flux_mapped<R, 2><<<nb, 128, 0, s>>>(coef, F, g, m, S, ctl, half);
}

void launch_update_mapped(int stage, double *Qn, double *Qs, double *Wacc, double *vol, double *vnext,
                          const double *Fx, const double *Fy, const double *Fz, const Geo &g, double gamma, Ctl *ctl,
                          cudaStream_t s)
{
    if (stage == 1)
        k_update_mapped<1><<<nblk(g.ncell, 256), 256, 0, s>>>(Qn, Qs, Wacc, vol, vnext, Fx, Fy, Fz, g, gamma, ctl);
    else
        k_update_mapped<2><<<nblk(g.ncell, 256), 256, 0, s>>>(Qn, Qs, Wacc, vol, vnext, Fx, Fy, Fz, g, gamma, ctl);
}

void launch_residual_mapped(const double *Fx, const double *Fy, const double *Fz, const double *geo, const Geo &g,
                            double *L, double *dL, cudaStream_t s)
{
    k_residual_mapped<<<nblk(g.ncell, 256), 256, 0, s>>>(Fx, Fy, Fz, geo, g, L, dL);
}

void launch_cfl_mapped(const double *Q, const double *geo, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s,
                       bool mixed)
{
    if (mixed) k_cfl_mapped<true><<<nblk(g.ncell, 256), 256, 0, s>>>(Q, geo, g, gamma, ctl);
    else k_cfl_mapped<false><<<nblk(g.ncell, 256), 256, 0, s>>>(Q, geo, g, gamma, ctl);
}

template void launch_recon_mapped<double>(const double *, const double *, double *, unsigned char *, const Geo &,
                                          const MapGeo &, const Scheme &, Ctl *, int, cudaStream_t);
template void launch_recon_mapped<float>(const double *, const double *, float *, unsigned char *, const Geo &,
                                         const MapGeo &, const Scheme &, Ctl *, int, cudaStream_t);
template void launch_flux_mapped<double>(int, const double *, double *, const Geo &, const MapGeo &, const Scheme &,
                                         Ctl *, int, cudaStream_t);
template void launch_flux_mapped<float>(int, const float *, double *, const Geo &, const MapGeo &, const Scheme &,
                                        Ctl *, int, cudaStream_t);

}  // namespace hk
