// Launchers of the mapped- and moving-mesh kernels (hgks_mapped.cu).
#pragma once
#include "hgks_device.cuh"

namespace hk {

struct MapGeo;

void launch_geom(double *geo, const Geo &g, const MapGeo &m, Ctl *ctl, int half, double t_fixed,
                 cudaStream_t s);
void launch_vol_from_geo(const double *geo, double *vol, const Geo &g, cudaStream_t s);
template <typename R>
void launch_recon_mapped(const double *Q, const double *geo, R *coef, unsigned char *flag, const Geo &g,
                         const MapGeo &m, const Scheme &S, Ctl *ctl, int half, cudaStream_t s);
template <typename R>
void launch_flux_mapped(int axis, const R *coef, double *F, const Geo &g, const MapGeo &m, const Scheme &S, Ctl *ctl,
                        int half, cudaStream_t s);
void launch_update_mapped(int stage, double *Qn, double *Qs, double *Wacc, double *vol, double *vnext,
                          const double *Fx, const double *Fy, const double *Fz, const Geo &g, double gamma, Ctl *ctl,
                          cudaStream_t s);
void launch_residual_mapped(const double *Fx, const double *Fy, const double *Fz, const double *geo, const Geo &g,
                            double *L, double *dL, cudaStream_t s);
void launch_cfl_mapped(const double *Q, const double *geo, const Geo &g, double gamma, Ctl *ctl, cudaStream_t s,
                       bool mixed = false);

}  // namespace hk
