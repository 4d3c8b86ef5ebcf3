// C ABI of the HGKS solver (declarations and contracts in include/hgks.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/hgks.h"
#include "hgks_kernels.cuh"
#include "hgks_mapped.cuh"
#include "hgks_mapped_launch.cuh"
#include "hgks_char_launch.cuh"

using hk::Ctl;
using hk::Geo;
using hk::Scheme;

struct hgks {
    Geo g;
    Scheme S;
    int precision;
    cudaStream_t stream;
    bool own_stream;
    int device;
    double *Qn, *Qs, *Wacc;      // padded Q^n, padded Q*, accumulator / staging [5][ncell]
    void *coef;                  // [cstride] records: Rec<R> (uniform mesh), MRec<R> (mapped)
    unsigned char *flag;         // [cstride]
    double *F[3];                // face fluxes [10][nface_d]
    Ctl *ctl;                    // device control block
    Ctl *ctl_host;               // pinned mirror for read-back
    // mapped and moving meshes (mesh 1, 2)
    int mesh;
    hk::MapGeo map;
    double *geo;                 // [NGEO][pstride] cell geometry at the stage time
    double *vol, *vnext;         // [ncell] volumes of the discrete conservation law
    double *sintab;              // sine factors of the map at the vertex indices
    // mixed path: the split state Q_hi + Q_lo in FP32 ([2][5][pstride]) that
    // the reconstruction takes its differences from
    float *Qsplit;
    // mixed path on a mapped mesh: FP32 copy of the cells' central second
    // moments ([6][pstride]), written with the geometry
    float *geof;
    // reconstruction in characteristic variables (option "characteristic")
    int charvar;
    void *coefc[3];              // per axis [2][50][nface_d] in the working precision
    unsigned char *flagc[3];     // per axis [2][nface_d]
    bool have_state;
    // optional per-phase timing with CUDA events on the handle's stream
    bool timing;
    struct Mark { int phase; int nlaunch; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
    double phase_ms[HGKS_NPHASE];
    unsigned long long phase_launches[HGKS_NPHASE];
    unsigned long long launches;
    unsigned long long bytes;
    char err[256];
};

static char g_create_err[256] = "";

// lets the allocation-free entry point (hgks_noalloc.cu) report through
// hgks_last_error(NULL)
void hgks_internal_set_error(const char *msg) { snprintf(g_create_err, sizeof g_create_err, "%s", msg); }

static int fail(hgks_t *h, int code, const char *fmt, const char *detail = nullptr)
{
    char *dst = h ? h->err : g_create_err;
    snprintf(dst, 256, fmt, detail ? detail : "");
    return code;
}

#define CUDA_OK(h, call)                                                         \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return fail((h), HGKS_E_CUDA, "CUDA: %s", cudaGetErrorString(e_)); \
    } while (0)

static int check_launch(hgks_t *h, int nlaunch)
{
    h->launches += nlaunch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, HGKS_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return HGKS_OK;
}

static cudaEvent_t take_event(hgks_t *h)
{
    if (!h->spare.empty()) {
        cudaEvent_t e = h->spare.back();
        h->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// bracket a group of launches of one phase with events (when timing is on)
struct PhaseTimer {
    hgks_t *h;
    int phase, n;
    cudaEvent_t a = nullptr;
    PhaseTimer(hgks_t *hh, int ph, int nl) : h(hh), phase(ph), n(nl)
    {
        if (h->timing) {
            a = take_event(h);
            cudaEventRecord(a, h->stream);
        }
    }
    ~PhaseTimer()
    {
        if (h->timing && a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, h->stream);
            h->marks.push_back({phase, n, a, b});
        }
    }
};

static void collect_timing(hgks_t *h)
{
    for (auto &m : h->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) h->phase_ms[m.phase] += ms;
        h->phase_launches[m.phase] += m.nlaunch;
        h->spare.push_back(m.a);
        h->spare.push_back(m.b);
    }
    h->marks.clear();
    cudaGetLastError();
}

static long long nface(const Geo &g, int d)
{
    return (long long)(g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2));
}

static void free_all(hgks_t *h)
{
    for (auto &m : h->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : h->spare) cudaEventDestroy(e);
    h->marks.clear();
    h->spare.clear();
    cudaFree(h->Qn);
    cudaFree(h->Qs);
    cudaFree(h->Wacc);
    cudaFree(h->coef);
    cudaFree(h->flag);
    for (int d = 0; d < 3; ++d) cudaFree(h->F[d]);
    cudaFree(h->ctl);
    cudaFreeHost(h->ctl_host);
    cudaFree(h->geo);
    cudaFree(h->vol);
    cudaFree(h->vnext);
    cudaFree(h->sintab);
    for (int d = 0; d < 3; ++d) {
        cudaFree(h->coefc[d]);
        cudaFree(h->flagc[d]);
    }
    cudaFree(h->Qsplit);
    cudaFree(h->geof);
}

extern "C" int hgks_create(const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6], void *stream,
                           hgks_t **out)
{
    if (!grid || !bc || !out) return fail(nullptr, HGKS_E_INVALID, "null argument%s");
    *out = nullptr;
    for (int d = 0; d < 3; ++d) {
        // periodic ghosts wrap modulo n (2 cells suffice); the GHOST = 3
        // reflective ghost layers mirror three interior cells
        if (grid->n[d] < 2 || grid->n[d] > HGKS_MAX_CELLS_PER_AXIS || !(grid->hi[d] > grid->lo[d]) ||
            (grid->n[d] < hk::GHOST && (bc[2 * d] == HGKS_BC_REFLECTIVE || bc[2 * d + 1] == HGKS_BC_REFLECTIVE)))
            return fail(nullptr, HGKS_E_INVALID,
                        "each axis needs at least 2 cells (3 with a reflective side) and hi > lo%s");
    }
    if (grid->mesh < 0 || grid->mesh > 2)
        return fail(nullptr, HGKS_E_INVALID, "mesh must be 0 (uniform), 1 (static mapped) or 2 (moving)%s");
    if (grid->mesh == 0 && (grid->mesh_amp != 0.0 || grid->mesh_omega != 0.0))
        return fail(nullptr, HGKS_E_INVALID, "a uniform mesh takes mesh_amp = mesh_omega = 0%s");
    if (grid->mesh != 0)
        for (int i = 0; i < 6; ++i)
            if (bc[i] != HGKS_BC_PERIODIC) return fail(nullptr, HGKS_E_INVALID, "mapped meshes are periodic%s");
    if (grid->precision != HGKS_FP64 && grid->precision != HGKS_MIXED)
        return fail(nullptr, HGKS_E_INVALID, "precision must be HGKS_FP64 or HGKS_MIXED%s");
    double hx = (grid->hi[0] - grid->lo[0]) / grid->n[0];
    for (int d = 1; d < 3 && grid->mesh == 0; ++d) {
        double hd = (grid->hi[d] - grid->lo[d]) / grid->n[d];
        if (fabs(hd - hx) > 1e-12 * hx) return fail(nullptr, HGKS_E_INVALID, "cells must be cubes%s");
    }
    if (!(gamma > 1.0) || !(gamma < 5.0 / 3.0 + 1e-12)) return fail(nullptr, HGKS_E_INVALID, "gamma out of range%s");
    if (mu < 0.0 || !(Pr > 0.0)) return fail(nullptr, HGKS_E_INVALID, "mu < 0 or Pr <= 0%s");
    for (int d = 0; d < 3; ++d) {
        if ((bc[2 * d] == HGKS_BC_PERIODIC) != (bc[2 * d + 1] == HGKS_BC_PERIODIC))
            return fail(nullptr, HGKS_E_INVALID, "periodic boundaries must pair%s");
        for (int s = 0; s < 2; ++s)
            if (bc[2 * d + s] != HGKS_BC_PERIODIC && bc[2 * d + s] != HGKS_BC_REFLECTIVE &&
                bc[2 * d + s] != HGKS_BC_OUTFLOW)
                return fail(nullptr, HGKS_E_INVALID, "unknown boundary condition%s");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, HGKS_E_CUDA, "no CUDA device%s");
    }

    hgks_t *h = new (std::nothrow) hgks_t();
    if (!h) return fail(nullptr, HGKS_E_NOMEM, "host allocation failed%s");
    cudaGetDevice(&h->device);
    Geo &g = h->g;
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
    Scheme &S = h->S;
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
    h->precision = grid->precision;

    if (stream) {
        h->stream = (cudaStream_t)stream;
        h->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, HGKS_E_CUDA, "stream creation failed%s");
        }
        h->own_stream = true;
    }
    const size_t rsz = grid->precision == HGKS_MIXED ? sizeof(float) : sizeof(double);
    h->mesh = grid->mesh;
    const bool mapped = h->mesh != 0;
    const bool f32 = grid->precision == HGKS_MIXED;
    const int ncoef = mapped ? (f32 ? hk::MRec<float>::N : hk::MRec<double>::N)
                             : (f32 ? hk::Rec<float>::N : hk::Rec<double>::N);
    const int nfv = mapped ? hk::NFACE_M : 10;
    size_t sizes[] = {5 * g.pstride * sizeof(double), 5 * g.pstride * sizeof(double), 5 * g.ncell * sizeof(double),
                      ncoef * g.cstride * rsz, (size_t)g.cstride};
    void **ptrs[] = {(void **)&h->Qn, (void **)&h->Qs, (void **)&h->Wacc, &h->coef, (void **)&h->flag};
    bool ok = true;
    for (int i = 0; i < 5 && ok; ++i) {
        ok = cudaMalloc(ptrs[i], sizes[i]) == cudaSuccess;
        h->bytes += sizes[i];
    }
    if (ok && grid->precision == HGKS_MIXED) {
        const size_t b = 2 * 5 * g.pstride * sizeof(float);
        ok = cudaMalloc((void **)&h->Qsplit, b) == cudaSuccess;
        h->bytes += b;
    }
    for (int d = 0; d < 3 && ok; ++d) {
        size_t b = nfv * nface(g, d) * sizeof(double);
        ok = cudaMalloc((void **)&h->F[d], b) == cudaSuccess;
        h->bytes += b;
    }
    if (mapped && ok) {
        // the map x = xi + amp S(t) prod sin(2 pi (xi - lo)/L): sine factors
        // at vertex indices -GHOST..n+GHOST of each axis
        const int nv[3] = {g.nx + 2 * hk::GHOST + 1, g.ny + 2 * hk::GHOST + 1, g.nz + 2 * hk::GHOST + 1};
        std::vector<double> tab(nv[0] + nv[1] + nv[2]);
        size_t o = 0;
        for (int d = 0; d < 3; ++d)
            for (int iv = -hk::GHOST; iv <= grid->n[d] + hk::GHOST; ++iv, ++o) {
                const double xi = grid->lo[d] + (grid->hi[d] - grid->lo[d]) * (double)iv / (double)grid->n[d];
                tab[o] = sin(2.0 * M_PI * (xi - grid->lo[d]) / (grid->hi[d] - grid->lo[d]));
            }
        // the same factors in FP32 after the FP64 ones, in one allocation
        std::vector<float> tabf(tab.begin(), tab.end());
        const size_t tbytes = tab.size() * sizeof(double) + tabf.size() * sizeof(float);
        ok = cudaMalloc((void **)&h->sintab, tbytes) == cudaSuccess &&
             cudaMemcpy(h->sintab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(h->sintab + tab.size(), tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice) ==
                 cudaSuccess;
        ok = ok && cudaMalloc((void **)&h->geo, hk::NGEO * g.pstride * sizeof(double)) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&h->vol, g.ncell * sizeof(double)) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&h->vnext, g.ncell * sizeof(double)) == cudaSuccess;
        h->bytes += tbytes + (hk::NGEO * g.pstride + 2 * g.ncell) * sizeof(double);
        if (ok && grid->precision == HGKS_MIXED) {
            ok = cudaMalloc((void **)&h->geof, hk::GEOF * g.pstride * sizeof(float)) == cudaSuccess;
            h->bytes += hk::GEOF * g.pstride * sizeof(float);
            h->map.geof = h->geof;
            h->map.qsplit = h->Qsplit;
        }
        for (int d = 0; d < 3; ++d) {
            h->map.lo[d] = grid->lo[d];
            h->map.hi[d] = grid->hi[d];
            h->map.n[d] = grid->n[d];
            h->map.h[d] = (grid->hi[d] - grid->lo[d]) / (double)grid->n[d];
            h->map.ih[d] = 1.0 / h->map.h[d];
        }
        h->map.amp = grid->mesh_amp;
        h->map.omega = grid->mesh_omega;
        h->map.moving = grid->mesh == 2;
        h->map.sx = h->sintab;
        h->map.sy = h->sintab + nv[0];
        h->map.sz = h->sintab + nv[0] + nv[1];
        const float *tf = (const float *)(h->sintab + tab.size());
        h->map.sxf = tf;
        h->map.syf = tf + nv[0];
        h->map.szf = tf + nv[0] + nv[1];
        for (int d = 0; d < 3; ++d) {
            h->map.lof[d] = float(grid->lo[d]);
            h->map.hf[d] = float((grid->hi[d] - grid->lo[d]) / grid->n[d]);
            h->map.ihf[d] = float(grid->n[d] / (grid->hi[d] - grid->lo[d]));
        }
    }
    ok = ok && cudaMalloc((void **)&h->ctl, sizeof(Ctl)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&h->ctl_host, sizeof(Ctl)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return fail(nullptr, HGKS_E_NOMEM, "device allocation failed%s");
    }
    // zero everything once so that no kernel ever reads uninitialised memory
    cudaMemsetAsync(h->Qn, 0, sizes[0], h->stream);
    cudaMemsetAsync(h->Qs, 0, sizes[1], h->stream);
    cudaMemsetAsync(h->Wacc, 0, sizes[2], h->stream);
    cudaMemsetAsync(h->coef, 0, sizes[3], h->stream);
    cudaMemsetAsync(h->flag, 0, sizes[4], h->stream);
    hk::launch_init_ctl(h->ctl, 0.0, h->stream);
    if (check_launch(h, 1) != HGKS_OK || cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return fail(nullptr, HGKS_E_CUDA, "initialisation failed%s");
    }
    *out = h;
    return HGKS_OK;
}

extern "C" int hgks_set_option(hgks_t *h, const char *key, double value)
{
    if (!h || !key) return HGKS_E_INVALID;
    if (!strcmp(key, "Gamma")) {
        if (!(value > 0.0) || !(value < 1.0 / 24.0)) return fail(h, HGKS_E_INVALID, "Gamma must be in (0, 1/24)%s");
        h->S.Gamma_lin = value;
    } else if (!strcmp(key, "weno_eps")) {
        if (!(value > 0.0)) return fail(h, HGKS_E_INVALID, "weno_eps must be > 0%s");
        h->S.weno_eps = value;
    } else if (!strcmp(key, "weno_pow")) {
        if (value != 1.0 && value != 2.0) return fail(h, HGKS_E_INVALID, "weno_pow must be 1 or 2%s");
        h->S.weno_pow = (int)value;
    } else if (!strcmp(key, "tau_eps")) {
        if (!(value >= 0.0)) return fail(h, HGKS_E_INVALID, "tau_eps must be >= 0%s");
        h->S.tau_eps = value;
    } else if (!strcmp(key, "tau_C")) {
        if (!(value >= 0.0)) return fail(h, HGKS_E_INVALID, "tau_C must be >= 0%s");
        h->S.tau_C = value;
    } else if (!strcmp(key, "limiter")) {
        h->S.limiter = value != 0.0;
    } else if (!strcmp(key, "mu_power")) {
        if (!(value >= 0.0) || !(value <= 4.0)) return fail(h, HGKS_E_INVALID, "mu_power must be in [0, 4]%s");
        h->S.mu_pow = value;
    } else if (!strcmp(key, "mu_T_ref")) {
        if (!(value > 0.0)) return fail(h, HGKS_E_INVALID, "mu_T_ref must be > 0%s");
        h->S.T_ref = value;
    } else if (!strcmp(key, "stencil")) {
        // 0: the big stencil S with 24 sub-stencils; 1: S' with 8 (Remark of Sec. 2)
        if (value != 0.0 && value != 1.0) return fail(h, HGKS_E_INVALID, "stencil must be 0 (S) or 1 (S')%s");
        if (value == 1.0 && (h->mesh != 0 || h->charvar))
            return fail(h, HGKS_E_INVALID, "the stencil S' needs the uniform mesh and conservative variables%s");
        h->S.sprime = value == 1.0;
    } else if (!strcmp(key, "characteristic")) {
        if (value != 0.0 && value != 1.0) return fail(h, HGKS_E_INVALID, "characteristic must be 0 or 1%s");
        if (value == 1.0 && h->mesh != 0)
            return fail(h, HGKS_E_INVALID, "characteristic variables need the uniform mesh%s");
        if (value == 1.0 && h->S.sprime)
            return fail(h, HGKS_E_INVALID, "characteristic variables use the stencil S%s");
        if (value == 1.0 && !h->coefc[0]) {
            const Geo &g = h->g;
            const size_t elem = h->precision == HGKS_MIXED ? sizeof(float) : sizeof(double);
            for (int d = 0; d < 3; ++d) {
                const size_t nface = (size_t)(g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2));
                const size_t bc = 2 * hk::CHAR_SLOTS_API * nface * elem, bf = 2 * nface;
                if (cudaMalloc(&h->coefc[d], bc) != cudaSuccess || cudaMalloc((void **)&h->flagc[d], bf) != cudaSuccess) {
                    cudaGetLastError();
                    for (int e = 0; e <= d; ++e) {
                        cudaFree(h->coefc[e]);
                        cudaFree(h->flagc[e]);
                        h->coefc[e] = nullptr;
                        h->flagc[e] = nullptr;
                    }
                    return fail(h, HGKS_E_NOMEM, "characteristic buffers: device allocation failed%s");
                }
                CUDA_OK(h, cudaMemsetAsync(h->coefc[d], 0, bc, h->stream));
                CUDA_OK(h, cudaMemsetAsync(h->flagc[d], 0, bf, h->stream));
                h->bytes += bc + bf;
            }
        }
        h->charvar = value == 1.0;
    } else {
        return fail(h, HGKS_E_INVALID, "unknown option %s", key);
    }
    hk::scheme_derive(h->S);
    return HGKS_OK;
}

// the device address of a host buffer that the GPU can address directly
// (pinned or registered host memory), or null (pageable memory)
static void *addressable_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" int hgks_set_state(hgks_t *h, const double *q, int on_device, double t)
{
    if (!h || !q) return HGKS_E_INVALID;
    const Geo &g = h->g;
    const double *src = q;
    if (!on_device) {
        // addressable host memory: the scatter kernel reads it over the host
        // link; otherwise a copy to the device buffer first
        src = static_cast<const double *>(addressable_host(q));
        if (!src) {
            CUDA_OK(h, cudaMemcpyAsync(h->Wacc, q, 5 * g.ncell * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            src = h->Wacc;
        }
    }
    hk::launch_scatter(src, h->Qn, g, h->stream);
    hk::launch_init_ctl(h->ctl, t, h->stream);
    int rc = check_launch(h, 2);
    if (rc) return rc;
    if (h->mesh != 0) {
        // the volumes of the discrete conservation law start from the
        // geometric volumes of the mesh at t
        hk::launch_geom(h->geo, g, h->map, nullptr, 0, t, h->stream);
        hk::launch_vol_from_geo(h->geo, h->vol, g, h->stream);
        if ((rc = check_launch(h, 2))) return rc;
    }
    if (!on_device) CUDA_OK(h, cudaStreamSynchronize(h->stream));
    h->have_state = true;
    return HGKS_OK;
}

extern "C" int hgks_get_state(hgks_t *h, double *q, int on_device, double *t)
{
    if (!h || !q) return HGKS_E_INVALID;
    if (!h->have_state) return fail(h, HGKS_E_STATE, "no state loaded%s");
    const Geo &g = h->g;
    // addressable host memory: the gather kernel writes it over the host
    // link; otherwise through the device buffer
    double *mapped = on_device ? nullptr : static_cast<double *>(addressable_host(q));
    double *dst = on_device ? q : (mapped ? mapped : h->Wacc);
    hk::launch_gather(h->Qn, dst, g, h->stream);
    int rc = check_launch(h, 1);
    if (rc) return rc;
    if (!on_device && !mapped)
        CUDA_OK(h, cudaMemcpyAsync(q, h->Wacc, 5 * g.ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (t) {
        CUDA_OK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
        CUDA_OK(h, cudaStreamSynchronize(h->stream));
        *t = h->ctl_host->t;
    } else if (!on_device) {
        CUDA_OK(h, cudaStreamSynchronize(h->stream));
    }
    return HGKS_OK;
}

// one evaluation of the fluxes of the state in Q (its ghosts are filled here)
// face fluxes of a stage on a mapped or moving mesh; the cell geometry of
// the stage time is computed first (half: 0 for t_n, 1 for t_n + dt/2)
// unless geom_ready says the CFL reduction of this step already did it
static int stage_fluxes_mapped(hgks_t *h, double *Q, int half, bool geom_ready)
{
    const Geo &g = h->g;
    cudaStream_t s = h->stream;
    {
        PhaseTimer t(h, HGKS_PHASE_HALO, geom_ready ? 1 : 2);
        if (!geom_ready) hk::launch_geom(h->geo, g, h->map, h->ctl, half, 0.0, s);
        hk::launch_halo(Q, g, s);
    }
    if (h->precision == HGKS_MIXED) {
        float *c = (float *)h->coef;
        {
            // split of Q (map.qsplit), reconstruction, positivity pass
            PhaseTimer t(h, HGKS_PHASE_RECON, 3);
            hk::launch_recon_mapped<float>(Q, h->geo, c, h->flag, g, h->map, h->S, h->ctl, half, s);
        }
        PhaseTimer t(h, HGKS_PHASE_FLUX, 3);
        for (int d = 0; d < 3; ++d) hk::launch_flux_mapped<float>(d, c, h->F[d], g, h->map, h->S, h->ctl, half, s);
    } else {
        double *c = (double *)h->coef;
        {
            PhaseTimer t(h, HGKS_PHASE_RECON, 2);
            hk::launch_recon_mapped<double>(Q, h->geo, c, h->flag, g, h->map, h->S, h->ctl, half, s);
        }
        PhaseTimer t(h, HGKS_PHASE_FLUX, 3);
        for (int d = 0; d < 3; ++d) hk::launch_flux_mapped<double>(d, c, h->F[d], g, h->map, h->S, h->ctl, half, s);
    }
    // geometry, halo, (mixed: split of Q,) reconstruction and its positivity
    // pass, three face sweeps
    return check_launch(h, (geom_ready ? 6 : 7) + (h->Qsplit ? 1 : 0));
}

static int stage_fluxes(hgks_t *h, double *Q, int half = 0, bool geom_ready = false)
{
    if (h->mesh != 0) return stage_fluxes_mapped(h, Q, half, geom_ready);
    const Geo &g = h->g;
    cudaStream_t s = h->stream;
    {
        PhaseTimer t(h, HGKS_PHASE_HALO, 1);
        hk::launch_halo(Q, g, s);
    }
    if (h->charvar) {
        // characteristic variables: both sides of every face reconstructed
        // in the face's eigenbasis (and the literal positivity pass), then
        // the face fluxes from those polynomials
        {
            PhaseTimer t(h, HGKS_PHASE_RECON, 6);
            for (int d = 0; d < 3; ++d) {
                if (h->precision == HGKS_MIXED)
                    hk::launch_recon_char<float>(d, Q, (float *)h->coefc[d], h->flagc[d], g, h->S, h->ctl, s);
                else
                    hk::launch_recon_char<double>(d, Q, (double *)h->coefc[d], h->flagc[d], g, h->S, h->ctl, s);
            }
        }
        PhaseTimer t(h, HGKS_PHASE_FLUX, 3);
        for (int d = 0; d < 3; ++d) {
            if (h->precision == HGKS_MIXED)
                hk::launch_flux_char<float>(d, (const float *)h->coefc[d], h->F[d], g, h->S, h->ctl, s);
            else
                hk::launch_flux_char<double>(d, (const double *)h->coefc[d], h->F[d], g, h->S, h->ctl, s);
        }
        return check_launch(h, 10);
    }
    if (h->precision == HGKS_MIXED) {
        float *c = (float *)h->coef;
        {
            PhaseTimer t(h, HGKS_PHASE_RECON, 3);
            hk::launch_recon<float>(Q, c, h->flag, g, h->S, h->ctl, s, (int *)h->F[2], h->Qsplit);
        }
        PhaseTimer t(h, HGKS_PHASE_FLUX, 3);
        for (int d = 0; d < 3; ++d) hk::launch_flux<float>(d, c, h->F[d], g, h->S, h->ctl, s);
    } else {
        double *c = (double *)h->coef;
        {
            PhaseTimer t(h, HGKS_PHASE_RECON, 2);
            hk::launch_recon<double>(Q, c, h->flag, g, h->S, h->ctl, s, (int *)h->F[2]);
        }
        PhaseTimer t(h, HGKS_PHASE_FLUX, 3);
        for (int d = 0; d < 3; ++d) hk::launch_flux<double>(d, c, h->F[d], g, h->S, h->ctl, s);
    }
    // halo, (split state,) reconstruction and its positivity pass, three face
    // sweeps
    return check_launch(h, 6 + (h->Qsplit ? 1 : 0));
}

extern "C" int hgks_step(hgks_t *h, int nsteps, double cfl, double dt_fixed, double t_end, double *t_out,
                         int *steps_done)
{
    if (!h || nsteps < 0) return HGKS_E_INVALID;
    if (!h->have_state) return fail(h, HGKS_E_STATE, "no state loaded%s");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(h, HGKS_E_INVALID, "need cfl > 0 or dt_fixed > 0%s");
    const Geo &g = h->g;
    cudaStream_t s = h->stream;
    int rc;
    for (int n = 0; n < nsteps; ++n) {
        int nl = 1;
        {
            PhaseTimer t(h, HGKS_PHASE_CFL, (dt_fixed > 0.0 ? 1 : 2) + (h->mesh != 0 ? 1 : 0));
            if (!(dt_fixed > 0.0)) {
                if (h->mesh != 0) {
                    // h = |Omega|^(1/3) of the mesh at t_n
                    hk::launch_geom(h->geo, g, h->map, h->ctl, 0, 0.0, s);
                    hk::launch_cfl_mapped(h->Qn, h->geo, g, h->S.gamma, h->ctl, s, h->precision == HGKS_MIXED);
                    ++nl;
                } else {
                    hk::launch_cfl(h->Qn, g, h->S.gamma, h->ctl, s, h->precision == HGKS_MIXED);
                }
                ++nl;
            }
            hk::launch_dt(h->ctl, cfl, dt_fixed, t_end, s);
        }
        if ((rc = check_launch(h, nl))) return rc;
        // on a mapped mesh the CFL reduction computed the geometry of t_n
        if ((rc = stage_fluxes(h, h->Qn, 0, h->mesh != 0 && !(dt_fixed > 0.0)))) return rc;
        {
            PhaseTimer t(h, HGKS_PHASE_UPDATE, 1);
            if (h->mesh != 0)
                hk::launch_update_mapped(1, h->Qn, h->Qs, h->Wacc, h->vol, h->vnext, h->F[0], h->F[1], h->F[2], g,
                                         h->S.gamma, h->ctl, s);
            else
                hk::launch_update(1, h->Qn, h->Qs, h->Wacc, h->F[0], h->F[1], h->F[2], g, h->S.gamma, h->ctl, s);
        }
        if ((rc = check_launch(h, 1))) return rc;
        if ((rc = stage_fluxes(h, h->Qs, 1))) return rc;
        {
            PhaseTimer t(h, HGKS_PHASE_UPDATE, 1);
            if (h->mesh != 0)
                hk::launch_update_mapped(2, h->Qn, h->Qs, h->Wacc, h->vol, h->vnext, h->F[0], h->F[1], h->F[2], g,
                                         h->S.gamma, h->ctl, s);
            else
                hk::launch_update(2, h->Qn, h->Qs, h->Wacc, h->F[0], h->F[1], h->F[2], g, h->S.gamma, h->ctl, s);
        }
        if ((rc = check_launch(h, 1))) return rc;
        // with a finite end time, look every 16 steps whether it is reached
        // and stop issuing steps that would do nothing
        if (!(dt_fixed > 0.0) && isfinite(t_end) && (n + 1) % 16 == 0 && n + 1 < nsteps) {
            CUDA_OK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CUDA_OK(h, cudaStreamSynchronize(s));
            if (h->ctl_host->t >= t_end) break;
        }
    }
    if (t_out || steps_done) {
        CUDA_OK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CUDA_OK(h, cudaStreamSynchronize(s));
        if (t_out) *t_out = h->ctl_host->t;
        if (steps_done) *steps_done = h->ctl_host->steps_done;
        if (h->ctl_host->status & 1) return fail(h, HGKS_E_NONPHYSICAL, "nonphysical state (NaN or rho, p <= 0)%s");
    }
    return HGKS_OK;
}

extern "C" int hgks_flux(hgks_t *h, double dt, double *L, double *dLdt, int on_device)
{
    if (!h || !L || !dLdt || !(dt > 0.0) || !isfinite(dt)) return HGKS_E_INVALID;
    if (!h->have_state) return fail(h, HGKS_E_STATE, "no state loaded%s");
    const Geo &g = h->g;
    cudaStream_t s = h->stream;
    // arm the stage kernels with this dt, keeping the time
    CUDA_OK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CUDA_OK(h, cudaStreamSynchronize(s));
    hk::launch_set_ctl(h->ctl, h->ctl_host->t, dt, 1, s);
    int rc = check_launch(h, 1);
    if (rc) return rc;
    if ((rc = stage_fluxes(h, h->Qn))) return rc;
    double *dL = nullptr, *dD = nullptr;
    if (on_device) {
        dL = L;
        dD = dLdt;
    } else {
        CUDA_OK(h, cudaMalloc((void **)&dL, 10 * g.ncell * sizeof(double)));
        dD = dL + 5 * g.ncell;
    }
    if (h->mesh != 0) hk::launch_residual_mapped(h->F[0], h->F[1], h->F[2], h->geo, g, dL, dD, s);
    else hk::launch_residual(h->F[0], h->F[1], h->F[2], g, dL, dD, s);
    rc = check_launch(h, 1);
    hk::launch_set_ctl(h->ctl, h->ctl_host->t, 0.0, 0, s);
    if (!rc) rc = check_launch(h, 1);
    if (!on_device) {
        if (!rc) {
            cudaMemcpyAsync(L, dL, 5 * g.ncell * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(dLdt, dD, 5 * g.ncell * sizeof(double), cudaMemcpyDeviceToHost, s);
        }
        cudaStreamSynchronize(s);
        cudaFree(dL);
        CUDA_OK(h, cudaGetLastError());
    }
    return rc;
}

extern "C" int hgks_reconstruct(hgks_t *h, double *coef, int *flag)
{
    if (!h || !coef) return HGKS_E_INVALID;
    if (!h->have_state) return fail(h, HGKS_E_STATE, "no state loaded%s");
    if (h->charvar)
        return fail(h, HGKS_E_STATE, "per-cell polynomials do not exist with characteristic variables (they are "
                                     "per face and side)%s");
    const Geo &g = h->g;
    cudaStream_t s = h->stream;
    CUDA_OK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CUDA_OK(h, cudaStreamSynchronize(s));
    hk::launch_set_ctl(h->ctl, h->ctl_host->t, 1.0, 1, s);
    hk::launch_halo(h->Qn, g, s);
    int rc = check_launch(h, 2);
    if (rc) return rc;
    double *dc = nullptr;
    CUDA_OK(h, cudaMalloc((void **)&dc, 45 * g.ncell * sizeof(double) + g.ncell * sizeof(int)));
    int *df = (int *)(dc + 45 * g.ncell);
    if (h->mesh != 0) hk::launch_geom(h->geo, g, h->map, h->ctl, 0, 0.0, s);
    if (h->precision == HGKS_MIXED) {
        if (h->mesh != 0) hk::launch_recon_mapped<float>(h->Qn, h->geo, (float *)h->coef, h->flag, g, h->map, h->S, h->ctl, 0, s);
        else hk::launch_recon<float>(h->Qn, (float *)h->coef, h->flag, g, h->S, h->ctl, s, (int *)h->F[2], h->Qsplit);
        hk::launch_export_coef<float>((float *)h->coef, h->flag, g, dc, df, s, h->mesh == 0);
    } else {
        if (h->mesh != 0) hk::launch_recon_mapped<double>(h->Qn, h->geo, (double *)h->coef, h->flag, g, h->map, h->S, h->ctl, 0, s);
        else hk::launch_recon<double>(h->Qn, (double *)h->coef, h->flag, g, h->S, h->ctl, s, (int *)h->F[2]);
        hk::launch_export_coef<double>((double *)h->coef, h->flag, g, dc, df, s, h->mesh == 0);
    }
    hk::launch_set_ctl(h->ctl, h->ctl_host->t, 0.0, 0, s);
    // reconstruction, export and control reset; on a mapped mesh also the
    // geometry and the positivity pass
    rc = check_launch(h, 4 + (h->mesh != 0 ? 1 : 0) + (h->Qsplit ? 1 : 0));
    if (!rc) {
        cudaMemcpyAsync(coef, dc, 45 * g.ncell * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (flag) cudaMemcpyAsync(flag, df, g.ncell * sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    cudaStreamSynchronize(s);
    cudaFree(dc);
    CUDA_OK(h, cudaGetLastError());
    return rc;
}

extern "C" int hgks_point_flux(int n, const double *in, const double *ug, double dt, const double params[5],
                               int precision, double *F, double *dF)
{
    if (n < 0 || (n > 0 && (!in || !F || !dF || !params)) || !(dt > 0.0) || !isfinite(dt)) return HGKS_E_INVALID;
    if (precision != HGKS_FP64 && precision != HGKS_MIXED) return HGKS_E_INVALID;
    if (n == 0) return HGKS_OK;
    Scheme S;
    S.gamma = params[0];
    S.K = (5.0 - 3.0 * params[0]) / (params[0] - 1.0);
    S.mu = params[1];
    S.Pr = params[2];
    S.tau_eps = params[3];
    S.tau_C = params[4];
    S.weno_eps = 1e-8;
    S.Gamma_lin = 0.0025;
    S.weno_pow = 1;
    S.limiter = 1;
    hk::scheme_derive(S);
    double *buf = nullptr;
    size_t nin = (size_t)n * 40, nug = ug ? (size_t)n * 3 : 0, nout = (size_t)n * 10;
    if (cudaMalloc((void **)&buf, (nin + nug + nout) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, HGKS_E_NOMEM, "device allocation failed%s");
    }
    double *din = buf, *dug = ug ? buf + nin : nullptr, *dout = buf + nin + nug;
    int rc = HGKS_OK;
    if (cudaMemcpy(din, in, nin * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) rc = HGKS_E_CUDA;
    if (!rc && ug && cudaMemcpy(dug, ug, nug * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) rc = HGKS_E_CUDA;
    if (!rc) {
        if (precision == HGKS_MIXED) hk::launch_point_flux<float>(n, din, dug, dt, S, dout, dout + 5 * (size_t)n, 0);
        else hk::launch_point_flux<double>(n, din, dug, dt, S, dout, dout + 5 * (size_t)n, 0);
        if (cudaGetLastError() != cudaSuccess) rc = HGKS_E_CUDA;
    }
    if (!rc && cudaMemcpy(F, dout, 5 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HGKS_E_CUDA;
    if (!rc && cudaMemcpy(dF, dout + 5 * (size_t)n, 5 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = HGKS_E_CUDA;
    cudaFree(buf);
    if (rc) {
        cudaGetLastError();
        return fail(nullptr, rc, "point flux failed%s");
    }
    return HGKS_OK;
}

extern "C" int hgks_set_timing(hgks_t *h, int enable)
{
    if (!h) return HGKS_E_INVALID;
    CUDA_OK(h, cudaStreamSynchronize(h->stream));
    collect_timing(h);
    for (int i = 0; i < HGKS_NPHASE; ++i) {
        h->phase_ms[i] = 0.0;
        h->phase_launches[i] = 0;
    }
    h->timing = enable != 0;
    return HGKS_OK;
}

extern "C" int hgks_get_timing(hgks_t *h, double ms[HGKS_NPHASE], unsigned long long launches[HGKS_NPHASE])
{
    if (!h || !ms || !launches) return HGKS_E_INVALID;
    CUDA_OK(h, cudaStreamSynchronize(h->stream));
    collect_timing(h);
    for (int i = 0; i < HGKS_NPHASE; ++i) {
        ms[i] = h->phase_ms[i];
        launches[i] = h->phase_launches[i];
    }
    return HGKS_OK;
}

extern "C" unsigned long long hgks_launch_count(const hgks_t *h) { return h ? h->launches : 0ULL; }

extern "C" unsigned long long hgks_device_bytes(const hgks_t *h) { return h ? h->bytes : 0ULL; }

extern "C" const char *hgks_last_error(const hgks_t *h) { return h ? h->err : g_create_err; }

extern "C" void hgks_destroy(hgks_t *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}
