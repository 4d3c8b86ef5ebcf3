// Allocation-free evaluation of L(Q) and dL/dt(Q) (declared in
// include/hgks.h as hgks_flux_noalloc).
//
// Some callers cannot call cudaMalloc: a serving loop that must never block
// on the implicit device synchronisation of an allocation, a host thread
// embedded in another framework that owns every device byte through its own
// pool, or code that has to run after start-up under a no-allocation policy.
// For them this entry point runs the same kernels as hgks_flux on scratch
// memory that lives in a fixed file-scope device array instead of memory
// the call allocates.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/hgks.h"
#include "hgks_kernels.cuh"

using hk::Ctl;
using hk::Geo;
using hk::Scheme;

// Records the reason for the last failed creation-level call (the string
// hgks_last_error(NULL) returns); defined in hgks_api.cu.
void hgks_internal_set_error(const char *msg);

// The scratch: HGKS_NOALLOC_SCRATCH_BYTES bytes in every GPU that loads the
// library, held until the process exits.  In host code this name is only a
// host-side stand-in for the device array; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char hgks_noalloc_scratch[HGKS_NOALLOC_SCRATCH_BYTES];

static std::mutex g_setup_mutex;
static void *g_scratch_addr[128];  // device address of the scratch, per device ordinal

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch on the current device, looked up once per
// device with that device current.
static int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        hgks_internal_set_error("hgks_flux_noalloc: no usable current CUDA device");
        return HGKS_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, hgks_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "hgks_flux_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            hgks_internal_set_error(msg);
            return HGKS_E_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HGKS_OK;
}

extern "C" int hgks_flux_noalloc(const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6],
                                 const double *q, double dt, double *L, double *dLdt, void *stream)
{
    if (!grid || !bc || !q || !L || !dLdt || !(dt > 0.0) || !isfinite(dt)) {
        hgks_internal_set_error("hgks_flux_noalloc: null buffer, or dt not a positive finite number");
        return HGKS_E_INVALID;
    }
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 2 || grid->n[d] > HGKS_MAX_CELLS_PER_AXIS || !(grid->hi[d] > grid->lo[d]) ||
            (grid->n[d] < hk::GHOST && (bc[2 * d] == HGKS_BC_REFLECTIVE || bc[2 * d + 1] == HGKS_BC_REFLECTIVE))) {
            hgks_internal_set_error("hgks_flux_noalloc: each axis needs at least 2 cells (3 with a reflective side) and hi > lo");
            return HGKS_E_INVALID;
        }
        if ((bc[2 * d] == HGKS_BC_PERIODIC) != (bc[2 * d + 1] == HGKS_BC_PERIODIC)) {
            hgks_internal_set_error("hgks_flux_noalloc: periodic boundaries must pair");
            return HGKS_E_INVALID;
        }
        for (int s = 0; s < 2; ++s)
            if (bc[2 * d + s] != HGKS_BC_PERIODIC && bc[2 * d + s] != HGKS_BC_REFLECTIVE &&
                bc[2 * d + s] != HGKS_BC_OUTFLOW) {
                hgks_internal_set_error("hgks_flux_noalloc: unknown boundary condition");
                return HGKS_E_INVALID;
            }
    }
    if (grid->mesh != 0 || grid->mesh_amp != 0.0 || grid->mesh_omega != 0.0 ||
        (grid->precision != HGKS_FP64 && grid->precision != HGKS_MIXED)) {
        hgks_internal_set_error("hgks_flux_noalloc: uniform mesh and HGKS_FP64 or HGKS_MIXED only");
        return HGKS_E_INVALID;
    }
    const double hx = (grid->hi[0] - grid->lo[0]) / grid->n[0];
    for (int d = 1; d < 3; ++d) {
        const double hd = (grid->hi[d] - grid->lo[d]) / grid->n[d];
        if (fabs(hd - hx) > 1e-12 * hx) {
            hgks_internal_set_error("hgks_flux_noalloc: cells must be cubes");
            return HGKS_E_INVALID;
        }
    }
    if (!(gamma > 1.0) || !(gamma < 5.0 / 3.0 + 1e-12) || mu < 0.0 || !(Pr > 0.0)) {
        hgks_internal_set_error("hgks_flux_noalloc: gamma, mu or Pr out of range");
        return HGKS_E_INVALID;
    }

    Geo g;
    g.nx = grid->n[0];
    g.ny = grid->n[1];
    g.nz = grid->n[2];
    g.px = g.nx + 2 * hk::GHOST;
    g.py = g.ny + 2 * hk::GHOST;
    g.pz = g.nz + 2 * hk::GHOST;
    g.cx = g.nx + 2;
    g.cy = g.ny + 2;
    g.cz = g.nz + 2;
    g.pstride = (long long)g.px * g.py * g.pz;
    g.cstride = (long long)g.cx * g.cy * g.cz;
    g.ncell = (long long)g.nx * g.ny * g.nz;
    g.h = hx;
    g.inv_h = 1.0 / hx;
    hk::geo_divisors(g);
    for (int i = 0; i < 6; ++i) g.bc[i] = bc[i];
    Scheme S;
    S.gamma = gamma;
    S.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    S.mu = mu;
    S.Pr = Pr;
    S.tau_eps = 0.01;
    S.tau_C = 1.0;
    S.weno_eps = 1e-8;
    S.Gamma_lin = 0.0025;
    S.weno_pow = 1;
    S.limiter = 1;
    hk::scheme_derive(S);

    // carve the scratch: control block, padded state, coefficients, flags,
    // face fluxes of the three axes, and (mixed) the split state Q_hi + Q_lo
    // that the handle's mixed path reconstructs from
    const bool mixed = grid->precision == HGKS_MIXED;
    const size_t rsz = mixed ? sizeof(float) : sizeof(double);
    size_t off_ctl = 0;
    size_t off_q = off_ctl + round256(sizeof(Ctl));
    size_t off_coef = off_q + round256(5 * (size_t)g.pstride * sizeof(double));
    size_t off_flag = off_coef + round256((size_t)(mixed ? hk::Rec<float>::N : hk::Rec<double>::N) * g.cstride * rsz);
    size_t off_f[3];
    size_t end = off_flag + round256((size_t)g.cstride);
    for (int d = 0; d < 3; ++d) {
        const size_t nf = (size_t)(g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2));
        off_f[d] = end;
        end += round256(10 * nf * sizeof(double));
    }
    const size_t off_split = end;
    if (mixed) end += round256(2 * 5 * (size_t)g.pstride * sizeof(float));
    if (end > (size_t)HGKS_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "hgks_flux_noalloc: this grid needs %zu bytes of scratch, more than the %d bytes the "
                 "allocation-free entry point holds",
                 end, HGKS_NOALLOC_SCRATCH_BYTES);
        hgks_internal_set_error(msg);
        return HGKS_E_INVALID;
    }
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != HGKS_OK) return rc;
    unsigned char *sb = (unsigned char *)base;
    Ctl *ctl = (Ctl *)(sb + off_ctl);
    double *Q = (double *)(sb + off_q);
    void *coef = sb + off_coef;
    unsigned char *flag = sb + off_flag;
    double *F[3] = {(double *)(sb + off_f[0]), (double *)(sb + off_f[1]), (double *)(sb + off_f[2])};
    float *split = mixed ? (float *)(sb + off_split) : nullptr;
    cudaStream_t s = (cudaStream_t)stream;

    // Every byte a kernel reads below is written earlier in this call: the
    // control block (time, dt, counters) by k_set_ctl, the interior state by
    // the scatter, every ghost cell by the halo, every coefficient and flag
    // of the reconstruction box by the reconstruction, every face flux by
    // the flux kernels, (mixed) the split state by the split kernel before
    // the reconstruction reads it, and the list of cells left to the literal
    // positivity check (kept in the z-face flux area until the z sweep) and
    // its count by the reconstruction after a reset.  Nothing of an earlier
    // call is read.
    hk::launch_init_ctl(ctl, 0.0, s);
    hk::launch_set_ctl(ctl, 0.0, dt, 1, s);
    hk::launch_scatter(q, Q, g, s);
    hk::launch_halo(Q, g, s);
    if (mixed) {
        hk::launch_recon<float>(Q, (float *)coef, flag, g, S, ctl, s, (int *)F[2], split);
        for (int d = 0; d < 3; ++d) hk::launch_flux<float>(d, (const float *)coef, F[d], g, S, ctl, s);
    } else {
        hk::launch_recon<double>(Q, (double *)coef, flag, g, S, ctl, s, (int *)F[2]);
        for (int d = 0; d < 3; ++d) hk::launch_flux<double>(d, (const double *)coef, F[d], g, S, ctl, s);
    }
    hk::launch_residual(F[0], F[1], F[2], g, L, dLdt, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "hgks_flux_noalloc: kernel launch: %s", cudaGetErrorString(e));
        hgks_internal_set_error(msg);
        return HGKS_E_CUDA;
    }
    return HGKS_OK;
}
