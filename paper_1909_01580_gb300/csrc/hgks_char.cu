// Kernels of the characteristic-variable reconstruction (Sec. 4, uniform
// mesh; item bodies in hgks_char.cuh) and the face flux that reads its
// per-(face, side) polynomials.
#include "hgks_char.cuh"
#include "hgks_char_launch.cuh"

namespace hk {

template <typename R, int D>
__global__ void __launch_bounds__(128) k_recon_char(const double *__restrict__ Q, R *__restrict__ coefc,
                                                    unsigned char *__restrict__ flagc, Geo g, Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    recon_char_item<R, D>(Q, coefc, flagc, g, S, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename R, int D>
__global__ void __launch_bounds__(128) k_positivity_char(const double *__restrict__ Q, R *__restrict__ coefc,
                                                         unsigned char *__restrict__ flagc, Geo g, Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    positivity_char_item<R, D>(Q, coefc, flagc, g, S, ctl, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename R, int D>
__global__ void __launch_bounds__(128) k_face_flux_char(const R *__restrict__ coefc, double *__restrict__ F, Geo g,
                                                        Scheme S, Ctl *ctl)
{
    if (!ctl->active) return;
    flux_item<R, D, true>(coefc, F, g, S, ctl->dt, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

static long long nface_of(const Geo &g, int axis)
{
    return (long long)(g.nx + (axis == 0)) * (g.ny + (axis == 1)) * (g.nz + (axis == 2));
}

template <typename R>
void launch_recon_char(int axis, const double *Q, R *coefc, unsigned char *flagc, const Geo &g, const Scheme &S,
                       Ctl *ctl, cudaStream_t s)
{
    const unsigned nb = nblk(2 * nface_of(g, axis), 128);
    if (axis == 0) {
        k_recon_char<R, 0><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
        k_positivity_char<R, 0><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
    } else if (axis == 1) {
        k_recon_char<R, 1><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
        k_positivity_char<R, 1><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
    } else {
        k_recon_char<R, 2><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
        k_positivity_char<R, 2><<<nb, 128, 0, s>>>(Q, coefc, flagc, g, S, ctl);
    }
}

template <typename R>
void launch_flux_char(int axis, const R *coefc, double *F, const Geo &g, const Scheme &S, Ctl *ctl, cudaStream_t s)
{
    const unsigned nb = nblk(4 * nface_of(g, axis), 128);
    if (axis == 0) k_face_flux_char<R, 0><<<nb, 128, 0, s>>>(coefc, F, g, S, ctl);
    else if (axis == 1) k_face_flux_char<R, 1><<<nb, 128, 0, s>>>(coefc, F, g, S, ctl);
    else k_face_flux_char<R, 2><<<nb, 128, 0, s>>>(coefc, F, g, S, ctl);
}

template void launch_recon_char<double>(int, const double *, double *, unsigned char *, const Geo &, const Scheme &,
                                        Ctl *, cudaStream_t);
template void launch_recon_char<float>(int, const double *, float *, unsigned char *, const Geo &, const Scheme &,
                                       Ctl *, cudaStream_t);
template void launch_flux_char<double>(int, const double *, double *, const Geo &, const Scheme &, Ctl *,
                                       cudaStream_t);
template void launch_flux_char<float>(int, const float *, double *, const Geo &, const Scheme &, Ctl *, cudaStream_t);

}  // namespace hk
