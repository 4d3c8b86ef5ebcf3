// Launchers of the HGKS kernels (definitions in hgks_kernels.cu).
#pragma once
#include "hgks_device.cuh"

namespace hk {

void launch_halo(double *Q, const Geo &g, cudaStream_t s);
// split (mixed path, or null): a [2][5][pstride] FP32 buffer; when given, the
// split state of Q is formed first (one more launch) and the FP32
// reconstruction takes its differences from it
template <typename R>
// list: room for one int per cell of the (n+2)^3 box, free until the
// reconstruction's positivity pass ends (the callers lend the z-face flux
// buffer, which the z sweep of the same stage overwrites afterwards)
void launch_recon(const double *Q, R *coef, unsigned char *flag, const Geo &g, const Scheme &S, Ctl *ctl,
                  cudaStream_t s, int *list, float *split = nullptr);
template <typename R>
void launch_flux(int axis, const R *coef, double *F, const Geo &g, const Scheme &S, Ctl *ctl, cudaStream_t s);
void launch_update(int stage, double *Qn, double *Qs, double *Wacc, const double *Fx, const double *Fy,
                   const double *Fz, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s);
void launch_residual(const double *Fx, const double *Fy, const double *Fz, const Geo &g, double *L, double *dL,
                     cudaStream_t s);
// mixed: FP32 candidates (FP64 minimum) for the mixed path
void launch_cfl(const double *Q, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s, bool mixed = false);
void launch_dt(Ctl *ctl, double cfl, double dt_fixed, double t_end, cudaStream_t s);
void launch_init_ctl(Ctl *ctl, double t, cudaStream_t s);
void launch_set_ctl(Ctl *ctl, double t, double dt, int active, cudaStream_t s);
void launch_scatter(const double *src, double *Q, const Geo &g, cudaStream_t s);
void launch_gather(const double *Q, double *dst, const Geo &g, cudaStream_t s);
template <typename R>
void launch_export_coef(const R *coef, const unsigned char *flag, const Geo &g, double *out, int *oflag,
                        cudaStream_t s, bool rec);
template <typename R>
void launch_point_flux(int n, const double *in, const double *ug, double dt, const Scheme &S, double *F, double *dF,
                       cudaStream_t s);

}  // namespace hk
