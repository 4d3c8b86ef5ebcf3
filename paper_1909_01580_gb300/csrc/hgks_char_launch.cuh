// Launchers of the characteristic-variable reconstruction and its face flux
// (hgks_char.cu).  coefc of axis a holds 2 x 50 x nface(a) values in the
// working precision, flagc 2 x nface(a) bytes.
#pragma once
#include "hgks_device.cuh"

namespace hk {

constexpr int CHAR_SLOTS_API = 50;  // values per (face, side): Q_c and 9 coefficients of 5 variables

// reconstruction of both sides of every face normal to `axis`, then the
// literal positivity check of the items whose bound was inconclusive
template <typename R>
void launch_recon_char(int axis, const double *Q, R *coefc, unsigned char *flagc, const Geo &g, const Scheme &S,
                       Ctl *ctl, cudaStream_t s);
template <typename R>
void launch_flux_char(int axis, const R *coefc, double *F, const Geo &g, const Scheme &S, Ctl *ctl, cudaStream_t s);

}  // namespace hk
