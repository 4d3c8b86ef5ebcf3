// Batched execution of many solver instances of different sizes (declared
// in include/hgks.h as hgks_batch_*): one persistent launch per phase of a
// stage covers every resident instance through a per-instance tile table,
// the whole step is captured once as a CUDA graph, and an autotuner picks
// the tile sizes, persistent grid sizes and the tile schedule.  Instances
// live in one device arena allocated at creation, so admission and
// retirement allocate nothing; a change of composition only rewrites the
// device-side instance and tile tables that the captured kernels read.
#include <cuda_runtime.h>

#include <cmath>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "../../include/hgks.h"
#include "hgks_items.cuh"
#include "hgks_kernels.cuh"

using hk::Ctl;
using hk::Geo;
using hk::Scheme;

namespace {

// one resident instance, as the batched kernels see it
struct BInst {
    Geo g;
    Scheme S;
    double *Qn, *Qs, *Wacc;
    void *coef;
    unsigned char *flag;
    double *F[3];
    Ctl *ctl;
    double cfl, t_end;
    int mixed;  // FP32 CFL candidates, as on a single handle of the mixed path
};

// a tile: items [first, last) of one instance in one phase
struct BTile {
    int inst;
    int pad;
    long long first, last;
};

// phases with their own tile table
enum { PH_CFL = 0, PH_HALO, PH_RECON, PH_FX, PH_FY, PH_FZ, PH_UPD, NPH };
// tuning groups: CFL, HALO, RECON, FLUX (the three axes), UPDATE
enum { TG_CFL = 0, TG_HALO, TG_RECON, TG_FLUX, TG_UPD, NTG };
static int group_of(int ph) { return ph == PH_CFL ? TG_CFL : ph == PH_HALO ? TG_HALO : ph == PH_RECON ? TG_RECON : ph == PH_UPD ? TG_UPD : TG_FLUX; }
static const int BLOCK[NTG] = {256, 256, 128, 128, 256};

long long items_of(const Geo &g, int ph)
{
    switch (ph) {
    case PH_CFL:
    case PH_UPD: return g.ncell;
    case PH_HALO: return g.pstride;
    case PH_RECON: return g.cstride;
    case PH_FX: return 4LL * (g.nx + 1) * g.ny * g.nz;
    case PH_FY: return 4LL * g.nx * (g.ny + 1) * g.nz;
    default: return 4LL * g.nx * g.ny * (g.nz + 1);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// batched persistent kernels: blocks stride over the tiles of their phase;
// a tile belongs to one instance, so per-instance branches are uniform
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kb_cfl(const BInst *__restrict__ I, const BTile *__restrict__ tiles,
                                              const int *__restrict__ ntiles)
{
    const int nt = ntiles[PH_CFL];
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const BTile T = tiles[tile];
        const BInst &in = I[T.inst];
        double v = INFINITY;
        for (long long b = T.first; b < T.last; b += blockDim.x) {
            const long long t = b + threadIdx.x;
            if (t < T.last)
                v = fmin(v, in.mixed ? hk::cfl_value_mixed(in.Qn, in.g, in.S.gamma, t)
                                     : hk::cfl_value(in.Qn, in.g, in.S.gamma, t));
        }
        hk::block_min_to(v, &in.ctl->minbits);
    }
}

__global__ void kb_dt(const BInst *__restrict__ I, const int *__restrict__ inuse, int nslot)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nslot && inuse[s]) hk::dt_choose(I[s].ctl, I[s].cfl, 0.0, I[s].t_end);
}

template <int STAGE>
__global__ void __launch_bounds__(256) kb_halo(const BInst *__restrict__ I, const BTile *__restrict__ tiles,
                                               const int *__restrict__ ntiles)
{
    const int nt = ntiles[PH_HALO];
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const BTile T = tiles[tile];
        const BInst &in = I[T.inst];
        if (!in.ctl->active) continue;
        double *Q = STAGE == 1 ? in.Qn : in.Qs;
        for (long long b = T.first; b < T.last; b += blockDim.x) {
            const long long t = b + threadIdx.x;
            if (t < T.last) hk::halo_item(Q, in.g, t);
        }
    }
}

template <typename R, int STAGE>
__global__ void __launch_bounds__(128) kb_recon(const BInst *__restrict__ I, const BTile *__restrict__ tiles,
                                                const int *__restrict__ ntiles)
{
    const int nt = ntiles[PH_RECON];
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const BTile T = tiles[tile];
        const BInst &in = I[T.inst];
        if (!in.ctl->active) continue;
        const double *Q = STAGE == 1 ? in.Qn : in.Qs;
        // records staged in shared memory and stored coalesced, as in k_recon
        extern __shared__ int4 kb_recon_stage_raw[];
        R *stage = reinterpret_cast<R *>(kb_recon_stage_raw);
        for (long long b = T.first; b < T.last; b += blockDim.x) {
            const long long t = b + threadIdx.x;
            if (t < T.last) hk::recon_item<R>(Q, stage + threadIdx.x * hk::Rec<R>::N, in.flag, in.g, in.S, in.ctl, t);
            hk::store_records<R>((R *)in.coef, stage, b, (int)std::min<long long>(blockDim.x, T.last - b));
        }
    }
}

// dynamic shared memory of kb_recon: one record per thread of the block
template <typename R> static int recon_smem() { return BLOCK[TG_RECON] * hk::Rec<R>::N * (int)sizeof(R); }
template <typename R> static void recon_smem_optin()
{
    cudaFuncSetAttribute(kb_recon<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, recon_smem<R>());
    cudaFuncSetAttribute(kb_recon<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, recon_smem<R>());
}

template <typename R, int D>
__global__ void __launch_bounds__(128) kb_flux(const BInst *__restrict__ I, const BTile *__restrict__ tiles,
                                               const int *__restrict__ ntiles)
{
    const int nt = ntiles[PH_FX + D];
    const BTile *tl = tiles;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const BTile T = tl[tile];
        const BInst &in = I[T.inst];
        if (!in.ctl->active) continue;
        const double dt = in.ctl->dt;
        // all lanes call the item (the Gauss sum shuffles across 4 lanes);
        // lanes past the tile compute a clamped point and write nothing
        for (long long b = T.first; b < T.last; b += blockDim.x)
            hk::flux_item<R, D>((const R *)in.coef, in.F[D], in.g, in.S, dt, b + threadIdx.x, T.last);
    }
}

template <int STAGE>
__global__ void __launch_bounds__(256) kb_update(const BInst *__restrict__ I, const BTile *__restrict__ tiles,
                                                 const int *__restrict__ ntiles)
{
    const int nt = ntiles[PH_UPD];
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const BTile T = tiles[tile];
        const BInst &in = I[T.inst];
        if (!in.ctl->active) continue;
        const double dt = in.ctl->dt;
        for (long long b = T.first; b < T.last; b += blockDim.x) {
            const long long t = b + threadIdx.x;
            if (t < T.last)
                hk::update_item<STAGE>(in.Qn, in.Qs, in.Wacc, in.F[0], in.F[1], in.F[2], in.g, in.S.gamma, in.ctl, dt,
                                       t);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct hgks_batch {
    int precision;
    cudaStream_t stream;
    bool own_stream;
    int sm_count;
    // arena and its first-fit free list (offset -> size)
    unsigned char *arena;
    size_t arena_bytes;
    std::map<size_t, size_t> free_list;
    // slots
    int nslot;
    std::vector<BInst> inst;        // host mirror of the instance table
    std::vector<int> inuse;
    std::vector<size_t> arena_off, arena_len;
    std::vector<double> t_end;
    Ctl *ctl;                       // [nslot] device
    Ctl *ctl_host;                  // [nslot] pinned
    // device tables
    BInst *d_inst;
    int *d_inuse;
    BTile *d_tiles[NPH];
    int tile_cap[NPH];
    int *d_ntiles;                  // [NPH]
    BTile *h_tiles;                 // pinned staging
    int h_tile_cap;
    int *h_small;                   // pinned staging for ntiles and inuse
    BInst *h_inst;                  // pinned staging for the instance table
    // tuning
    int schedule;                   // 0 slot order, 1 largest first, 2 round robin
    int tile_mult[NTG];             // tile = tile_mult * block items
    int bps[NTG];                   // persistent blocks per SM
    // graph
    bool graph_dirty;
    cudaGraphExec_t exec;
    cudaGraph_t graph;
    unsigned long long launches;
    char err[256];
};

static char g_batch_err[256] = "";

static int bfail(hgks_batch_t *b, int code, const char *msg)
{
    snprintf(b ? b->err : g_batch_err, 256, "%s", msg);
    return code;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int validate_grid(const hgks_grid_t *grid, double gamma, double mu, double Pr, const int bc[6], double *hx_out)
{
    if (!grid || !bc) return HGKS_E_INVALID;
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 2 || grid->n[d] > HGKS_MAX_CELLS_PER_AXIS || !(grid->hi[d] > grid->lo[d]))
            return HGKS_E_INVALID;
        if (grid->n[d] < hk::GHOST && (bc[2 * d] == HGKS_BC_REFLECTIVE || bc[2 * d + 1] == HGKS_BC_REFLECTIVE))
            return HGKS_E_INVALID;
    }
    if (grid->mesh != 0 || grid->mesh_amp != 0.0 || grid->mesh_omega != 0.0) return HGKS_E_INVALID;
    const double hx = (grid->hi[0] - grid->lo[0]) / grid->n[0];
    for (int d = 1; d < 3; ++d) {
        const double hd = (grid->hi[d] - grid->lo[d]) / grid->n[d];
        if (fabs(hd - hx) > 1e-12 * hx) return HGKS_E_INVALID;
    }
    if (!(gamma > 1.0) || !(gamma < 5.0 / 3.0 + 1e-12) || mu < 0.0 || !(Pr > 0.0)) return HGKS_E_INVALID;
    for (int d = 0; d < 3; ++d) {
        if ((bc[2 * d] == HGKS_BC_PERIODIC) != (bc[2 * d + 1] == HGKS_BC_PERIODIC)) return HGKS_E_INVALID;
        for (int s = 0; s < 2; ++s)
            if (bc[2 * d + s] != HGKS_BC_PERIODIC && bc[2 * d + s] != HGKS_BC_REFLECTIVE &&
                bc[2 * d + s] != HGKS_BC_OUTFLOW) return HGKS_E_INVALID;
    }
    *hx_out = hx;
    return HGKS_OK;
}

static Geo make_geo(const hgks_grid_t *grid, double hx, const int bc[6])
{
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
    return g;
}

// sizes of one instance's buffers in the arena, in carve order
static void inst_sizes(const Geo &g, int precision, size_t sz[8])
{
    const size_t rsz = precision == HGKS_MIXED ? sizeof(float) : sizeof(double);
    sz[0] = align256(5 * (size_t)g.pstride * sizeof(double));
    sz[1] = sz[0];
    sz[2] = align256(5 * (size_t)g.ncell * sizeof(double));
    sz[3] = align256((size_t)(rsz == sizeof(float) ? hk::Rec<float>::N : hk::Rec<double>::N) * g.cstride * rsz);
    sz[4] = align256((size_t)g.cstride);
    for (int d = 0; d < 3; ++d)
        sz[5 + d] = align256(10 * (size_t)(g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2)) * sizeof(double));
}

extern "C" unsigned long long hgks_batch_footprint(const hgks_grid_t *grid)
{
    if (!grid) return 0ULL;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    double hx;
    if (validate_grid(grid, 1.4, 0.0, 1.0, bc, &hx) != HGKS_OK) return 0ULL;
    size_t sz[8], tot = 0;
    inst_sizes(make_geo(grid, hx, bc), grid->precision, sz);
    for (int i = 0; i < 8; ++i) tot += sz[i];
    return tot;
}

static bool arena_take(hgks_batch_t *b, size_t len, size_t *off)
{
    for (auto it = b->free_list.begin(); it != b->free_list.end(); ++it) {
        if (it->second >= len) {
            *off = it->first;
            const size_t rest = it->second - len, roff = it->first + len;
            b->free_list.erase(it);
            if (rest) b->free_list[roff] = rest;
            return true;
        }
    }
    return false;
}

static void arena_give(hgks_batch_t *b, size_t off, size_t len)
{
    auto it = b->free_list.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != b->free_list.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        b->free_list.erase(nx);
    }
    if (it != b->free_list.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            b->free_list.erase(it);
        }
    }
}

// rebuild and upload the instance and tile tables (synchronises the stream)
static int upload_tables(hgks_batch_t *b)
{
    cudaStream_t s = b->stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, HGKS_E_CUDA, "stream error before table upload");
    std::vector<int> order;
    for (int i = 0; i < b->nslot; ++i)
        if (b->inuse[i]) order.push_back(i);
    if (b->schedule == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b->inst[x].g.ncell > b->inst[y].g.ncell; });
    int nt_all[NPH];
    std::vector<BTile> tiles[NPH];
    for (int ph = 0; ph < NPH; ++ph) {
        const long long tsz = (long long)BLOCK[group_of(ph)] * b->tile_mult[group_of(ph)];
        if (b->schedule == 2) {
            // round robin: tile k of every instance before tile k + 1 of any
            std::vector<long long> next(order.size(), 0);
            bool more = true;
            while (more) {
                more = false;
                for (size_t o = 0; o < order.size(); ++o) {
                    const long long n = items_of(b->inst[order[o]].g, ph);
                    if (next[o] < n) {
                        tiles[ph].push_back({order[o], 0, next[o], std::min(n, next[o] + tsz)});
                        next[o] += tsz;
                        more = more || next[o] < n;
                    }
                }
            }
        } else {
            for (int sl : order) {
                const long long n = items_of(b->inst[sl].g, ph);
                for (long long f = 0; f < n; f += tsz) tiles[ph].push_back({sl, 0, f, std::min(n, f + tsz)});
            }
        }
        nt_all[ph] = (int)tiles[ph].size();
        if (nt_all[ph] > b->tile_cap[ph]) {
            // grow (rare; the captured graph holds the old pointer)
            cudaFree(b->d_tiles[ph]);
            const int cap = std::max(nt_all[ph] * 2, 1024);
            if (cudaMalloc((void **)&b->d_tiles[ph], cap * sizeof(BTile)) != cudaSuccess) {
                b->d_tiles[ph] = nullptr;
                b->tile_cap[ph] = 0;
                cudaGetLastError();
                return bfail(b, HGKS_E_NOMEM, "tile table allocation failed");
            }
            b->tile_cap[ph] = cap;
            b->graph_dirty = true;
        }
    }
    size_t need = 0;
    for (int ph = 0; ph < NPH; ++ph) need = std::max(need, (size_t)nt_all[ph]);
    if ((int)need > b->h_tile_cap) {
        cudaFreeHost(b->h_tiles);
        const int cap = std::max((int)need * 2, 1024);
        if (cudaMallocHost((void **)&b->h_tiles, cap * sizeof(BTile)) != cudaSuccess) {
            b->h_tiles = nullptr;
            b->h_tile_cap = 0;
            cudaGetLastError();
            return bfail(b, HGKS_E_NOMEM, "host staging allocation failed");
        }
        b->h_tile_cap = cap;
    }
    for (int ph = 0; ph < NPH; ++ph) {
        if (nt_all[ph]) {
            memcpy(b->h_tiles, tiles[ph].data(), nt_all[ph] * sizeof(BTile));
            if (cudaMemcpyAsync(b->d_tiles[ph], b->h_tiles, nt_all[ph] * sizeof(BTile), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return bfail(b, HGKS_E_CUDA, "tile table upload failed");
        }
    }
    memcpy(b->h_inst, b->inst.data(), b->nslot * sizeof(BInst));
    for (int ph = 0; ph < NPH; ++ph) b->h_small[ph] = nt_all[ph];
    for (int i = 0; i < b->nslot; ++i) b->h_small[NPH + i] = b->inuse[i];
    if (cudaMemcpyAsync(b->d_inst, b->h_inst, b->nslot * sizeof(BInst), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->d_ntiles, b->h_small, NPH * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->d_inuse, b->h_small + NPH, b->nslot * sizeof(int), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bfail(b, HGKS_E_CUDA, "instance table upload failed");
    return HGKS_OK;
}

template <typename R> static void launch_step_kernels(hgks_batch_t *b)
{
    cudaStream_t s = b->stream;
    const int n = b->sm_count;
    const BInst *I = b->d_inst;
    const int *nt = b->d_ntiles;
    kb_cfl<<<b->bps[TG_CFL] * n, BLOCK[TG_CFL], 0, s>>>(I, b->d_tiles[PH_CFL], nt);
    kb_dt<<<(b->nslot + 127) / 128, 128, 0, s>>>(I, b->d_inuse, b->nslot);
    kb_halo<1><<<b->bps[TG_HALO] * n, BLOCK[TG_HALO], 0, s>>>(I, b->d_tiles[PH_HALO], nt);
    kb_recon<R, 1><<<b->bps[TG_RECON] * n, BLOCK[TG_RECON], recon_smem<R>(), s>>>(I, b->d_tiles[PH_RECON], nt);
    kb_flux<R, 0><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FX], nt);
    kb_flux<R, 1><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FY], nt);
    kb_flux<R, 2><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FZ], nt);
    kb_update<1><<<b->bps[TG_UPD] * n, BLOCK[TG_UPD], 0, s>>>(I, b->d_tiles[PH_UPD], nt);
    kb_halo<2><<<b->bps[TG_HALO] * n, BLOCK[TG_HALO], 0, s>>>(I, b->d_tiles[PH_HALO], nt);
    kb_recon<R, 2><<<b->bps[TG_RECON] * n, BLOCK[TG_RECON], recon_smem<R>(), s>>>(I, b->d_tiles[PH_RECON], nt);
    kb_flux<R, 0><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FX], nt);
    kb_flux<R, 1><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FY], nt);
    kb_flux<R, 2><<<b->bps[TG_FLUX] * n, BLOCK[TG_FLUX], 0, s>>>(I, b->d_tiles[PH_FZ], nt);
    kb_update<2><<<b->bps[TG_UPD] * n, BLOCK[TG_UPD], 0, s>>>(I, b->d_tiles[PH_UPD], nt);
}
static const int LAUNCHES_PER_STEP = 14;

// (re)capture the step graph
static int capture(hgks_batch_t *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaStream_t s = b->stream;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, HGKS_E_CUDA, "stream capture could not begin");
    if (b->precision == HGKS_MIXED) launch_step_kernels<float>(b);
    else launch_step_kernels<double>(b);
    cudaError_t e = cudaStreamEndCapture(s, &b->graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, HGKS_E_CUDA, "stream capture failed");
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, HGKS_E_CUDA, "graph instantiation failed");
    }
    b->graph_dirty = false;
    return HGKS_OK;
}

extern "C" int hgks_batch_create(int precision, unsigned long long arena_bytes, int max_instances, void *stream,
                                 hgks_batch_t **out)
{
    if (!out || max_instances < 1 || max_instances > 4096 || arena_bytes < 4096 ||
        (precision != HGKS_FP64 && precision != HGKS_MIXED))
        return bfail(nullptr, HGKS_E_INVALID, "bad batch arguments");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return bfail(nullptr, HGKS_E_CUDA, "no CUDA device");
    }
    hgks_batch_t *b = new (std::nothrow) hgks_batch_t();
    if (!b) return bfail(nullptr, HGKS_E_NOMEM, "host allocation failed");
    b->precision = precision;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    // the reconstruction's record stage exceeds the default 48 KB in FP64
    if (precision == HGKS_MIXED) recon_smem_optin<float>();
    else recon_smem_optin<double>();
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = true;
    }
    b->nslot = max_instances;
    b->inst.assign(b->nslot, BInst());
    b->inuse.assign(b->nslot, 0);
    b->arena_off.assign(b->nslot, 0);
    b->arena_len.assign(b->nslot, 0);
    b->t_end.assign(b->nslot, 0.0);
    b->arena_bytes = (size_t)arena_bytes & ~(size_t)255;
    bool ok = cudaMalloc((void **)&b->arena, b->arena_bytes) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->ctl, b->nslot * sizeof(Ctl)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&b->ctl_host, b->nslot * sizeof(Ctl)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->d_inst, b->nslot * sizeof(BInst)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->d_inuse, b->nslot * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->d_ntiles, NPH * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&b->h_small, (NPH + b->nslot) * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&b->h_inst, b->nslot * sizeof(BInst)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        hgks_batch_destroy(b);
        return bfail(nullptr, HGKS_E_NOMEM, "device allocation of the batch arena failed");
    }
    b->free_list[0] = b->arena_bytes;
    cudaMemsetAsync(b->arena, 0, b->arena_bytes, b->stream);
    cudaMemsetAsync(b->ctl, 0, b->nslot * sizeof(Ctl), b->stream);
    b->schedule = 1;
    for (int gidx = 0; gidx < NTG; ++gidx) {
        b->tile_mult[gidx] = 4;
        b->bps[gidx] = 2;
    }
    b->bps[TG_HALO] = b->bps[TG_UPD] = b->bps[TG_CFL] = 4;
    b->graph_dirty = true;
    int rc = upload_tables(b);
    if (rc != HGKS_OK) {
        hgks_batch_destroy(b);
        return bfail(nullptr, rc, "batch table initialisation failed");
    }
    *out = b;
    return HGKS_OK;
}

// Admission check of a request's initial state (host FP64 [5][ncell]):
// every value finite, density and pressure positive in every cell, so that
// a bad request is refused before it takes a slot and never reaches the
// graph that advances the others.
static bool host_state_physical(const double *q, long long ncell, double gamma)
{
    for (long long c = 0; c < ncell; ++c) {
        const double r = q[c], mx = q[ncell + c], my = q[2 * ncell + c], mz = q[3 * ncell + c], e = q[4 * ncell + c];
        if (!std::isfinite(r) || !std::isfinite(mx) || !std::isfinite(my) || !std::isfinite(mz) || !std::isfinite(e))
            return false;
        const double p = (gamma - 1.0) * (e - 0.5 * (mx * mx + my * my + mz * mz) / r);
        if (!(r > 0.0) || !(p > 0.0)) return false;
    }
    return true;
}

extern "C" int hgks_batch_add(hgks_batch_t *b, const hgks_grid_t *grid, double gamma, double mu, double Pr,
                              const int bc[6], const double *q, double t0, double t_end, double cfl, int *slot)
{
    if (!b || !grid || !q || !slot || !(cfl > 0.0) || !(t_end >= t0)) return HGKS_E_INVALID;
    if (grid->precision != b->precision) return bfail(b, HGKS_E_INVALID, "instance precision differs from the batch");
    double hx;
    if (validate_grid(grid, gamma, mu, Pr, bc, &hx) != HGKS_OK) return bfail(b, HGKS_E_INVALID, "invalid instance");
    if (!host_state_physical(q, (long long)grid->n[0] * grid->n[1] * grid->n[2], gamma))
        return bfail(b, HGKS_E_NONPHYSICAL, "initial state not finite, or with non-positive density or pressure");
    int sl = -1;
    for (int i = 0; i < b->nslot && sl < 0; ++i)
        if (!b->inuse[i]) sl = i;
    if (sl < 0) return bfail(b, HGKS_E_NOMEM, "no free slot");
    Geo g = make_geo(grid, hx, bc);
    size_t sz[8], tot = 0;
    inst_sizes(g, b->precision, sz);
    for (int i = 0; i < 8; ++i) tot += sz[i];
    size_t off;
    if (!arena_take(b, tot, &off)) return bfail(b, HGKS_E_NOMEM, "not enough free arena memory for this instance");
    BInst &in = b->inst[sl];
    in.g = g;
    in.mixed = b->precision == HGKS_MIXED;
    Scheme &S = in.S;
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
    unsigned char *p = b->arena + off;
    in.Qn = (double *)p;
    p += sz[0];
    in.Qs = (double *)p;
    p += sz[1];
    in.Wacc = (double *)p;
    p += sz[2];
    in.coef = p;
    p += sz[3];
    in.flag = p;
    p += sz[4];
    for (int d = 0; d < 3; ++d) {
        in.F[d] = (double *)p;
        p += sz[5 + d];
    }
    in.ctl = b->ctl + sl;
    in.cfl = cfl;
    in.t_end = t_end;
    b->arena_off[sl] = off;
    b->arena_len[sl] = tot;
    b->t_end[sl] = t_end;
    cudaStream_t s = b->stream;
    if (cudaMemcpyAsync(in.Wacc, q, 5 * (size_t)g.ncell * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        arena_give(b, off, tot);
        return bfail(b, HGKS_E_CUDA, "state upload failed");
    }
    hk::launch_scatter(in.Wacc, in.Qn, g, s);
    hk::launch_init_ctl(in.ctl, t0, s);
    b->launches += 2;
    if (cudaGetLastError() != cudaSuccess) {
        arena_give(b, off, tot);
        return bfail(b, HGKS_E_CUDA, "instance initialisation failed");
    }
    b->inuse[sl] = 1;
    int rc = upload_tables(b);
    if (rc != HGKS_OK) return rc;
    *slot = sl;
    return HGKS_OK;
}

extern "C" int hgks_batch_remove(hgks_batch_t *b, int slot)
{
    if (!b || slot < 0 || slot >= b->nslot || !b->inuse[slot]) return HGKS_E_INVALID;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, HGKS_E_CUDA, "stream error");
    b->inuse[slot] = 0;
    arena_give(b, b->arena_off[slot], b->arena_len[slot]);
    b->inst[slot] = BInst();
    return upload_tables(b);
}

extern "C" int hgks_batch_step(hgks_batch_t *b, int nsteps)
{
    if (!b || nsteps < 0) return HGKS_E_INVALID;
    if (b->graph_dirty) {
        int rc = capture(b);
        if (rc != HGKS_OK) return rc;
    }
    for (int n = 0; n < nsteps; ++n) {
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, HGKS_E_CUDA, "graph launch failed");
        }
        b->launches += LAUNCHES_PER_STEP;
    }
    return HGKS_OK;
}

extern "C" int hgks_batch_poll(hgks_batch_t *b, double *t, int *steps, int *state)
{
    if (!b) return HGKS_E_INVALID;
    if (cudaMemcpyAsync(b->ctl_host, b->ctl, b->nslot * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, HGKS_E_CUDA, "poll failed");
    for (int i = 0; i < b->nslot; ++i) {
        const Ctl &c = b->ctl_host[i];
        if (t) t[i] = b->inuse[i] ? c.t : 0.0;
        if (steps) steps[i] = b->inuse[i] ? c.steps_done : 0;
        if (state) {
            int st = 0;
            if (b->inuse[i]) {
                st = c.t >= b->t_end[i] ? 2 : 1;
                if (c.status & 1) st = 3;
            }
            state[i] = st;
        }
    }
    return HGKS_OK;
}

extern "C" int hgks_batch_get_state(hgks_batch_t *b, int slot, double *q)
{
    if (!b || !q || slot < 0 || slot >= b->nslot || !b->inuse[slot]) return HGKS_E_INVALID;
    const BInst &in = b->inst[slot];
    hk::launch_gather(in.Qn, in.Wacc, in.g, b->stream);
    b->launches += 1;
    if (cudaMemcpyAsync(q, in.Wacc, 5 * (size_t)in.g.ncell * sizeof(double), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, HGKS_E_CUDA, "state download failed");
    return HGKS_OK;
}

// time nsteps of the current configuration with CUDA events
static float time_steps(hgks_batch_t *b, int nsteps)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    hgks_batch_step(b, nsteps);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 1e30f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

static void get_params(const hgks_batch_t *b, int p[HGKS_TUNE_NPARAM])
{
    p[0] = b->schedule;
    for (int gidx = 0; gidx < NTG; ++gidx) {
        p[1 + gidx] = b->tile_mult[gidx];
        p[1 + NTG + gidx] = b->bps[gidx];
    }
}

extern "C" int hgks_batch_set_tuning(hgks_batch_t *b, const int params[HGKS_TUNE_NPARAM])
{
    if (!b || !params) return HGKS_E_INVALID;
    if (params[0] < 0 || params[0] > 2) return bfail(b, HGKS_E_INVALID, "schedule must be 0, 1 or 2");
    for (int gidx = 0; gidx < NTG; ++gidx) {
        const int tm = params[1 + gidx], bp = params[1 + NTG + gidx];
        if (tm < 1 || tm > 64 || bp < 1 || bp > 32) return bfail(b, HGKS_E_INVALID, "tuning parameter out of range");
    }
    b->schedule = params[0];
    for (int gidx = 0; gidx < NTG; ++gidx) {
        b->tile_mult[gidx] = params[1 + gidx];
        b->bps[gidx] = params[1 + NTG + gidx];
    }
    b->graph_dirty = true;
    return upload_tables(b);
}

// resident blocks per SM of each group's kernel (caps the search)
template <typename R> static void occupancy_caps(int cap[NTG])
{
    int v = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_cfl, BLOCK[TG_CFL], 0);
    cap[TG_CFL] = std::max(1, v);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_halo<1>, BLOCK[TG_HALO], 0);
    cap[TG_HALO] = std::max(1, v);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_recon<R, 1>, BLOCK[TG_RECON], recon_smem<R>());
    cap[TG_RECON] = std::max(1, v);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_flux<R, 0>, BLOCK[TG_FLUX], 0);
    cap[TG_FLUX] = std::max(1, v);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kb_update<1>, BLOCK[TG_UPD], 0);
    cap[TG_UPD] = std::max(1, v);
    cudaGetLastError();
}

extern "C" int hgks_batch_tune(hgks_batch_t *b, int steps_per_trial, int params_out[HGKS_TUNE_NPARAM])
{
    if (!b || steps_per_trial < 1) return HGKS_E_INVALID;
    int cap[NTG];
    if (b->precision == HGKS_MIXED) occupancy_caps<float>(cap);
    else occupancy_caps<double>(cap);
    int p[HGKS_TUNE_NPARAM];
    get_params(b, p);
    // coordinate descent: each group's tile multiple and grid size, then the schedule
    if (hgks_batch_set_tuning(b, p) != HGKS_OK) return HGKS_E_CUDA;
    time_steps(b, 1);  // warm the graph
    float best = time_steps(b, steps_per_trial);
    const int tms[] = {1, 4, 16};
    for (int gidx = 0; gidx < NTG; ++gidx) {
        for (int bp = 1; bp <= cap[gidx]; bp *= 2) {
            for (int tm : tms) {
                int q[HGKS_TUNE_NPARAM];
                memcpy(q, p, sizeof q);
                q[1 + gidx] = tm;
                q[1 + NTG + gidx] = bp;
                if (!memcmp(q, p, sizeof q)) continue;
                if (hgks_batch_set_tuning(b, q) != HGKS_OK) return HGKS_E_CUDA;
                time_steps(b, 1);
                const float ms = time_steps(b, steps_per_trial);
                if (ms < best) {
                    best = ms;
                    memcpy(p, q, sizeof p);
                }
            }
        }
    }
    for (int sch = 0; sch < 3; ++sch) {
        int q[HGKS_TUNE_NPARAM];
        memcpy(q, p, sizeof q);
        q[0] = sch;
        if (!memcmp(q, p, sizeof q)) continue;
        if (hgks_batch_set_tuning(b, q) != HGKS_OK) return HGKS_E_CUDA;
        time_steps(b, 1);
        const float ms = time_steps(b, steps_per_trial);
        if (ms < best) {
            best = ms;
            memcpy(p, q, sizeof p);
        }
    }
    int rc = hgks_batch_set_tuning(b, p);
    if (rc == HGKS_OK && params_out) memcpy(params_out, p, sizeof p);
    return rc;
}

extern "C" int hgks_batch_get_tuning(const hgks_batch_t *b, int params[HGKS_TUNE_NPARAM])
{
    if (!b || !params) return HGKS_E_INVALID;
    get_params(b, params);
    return HGKS_OK;
}

extern "C" unsigned long long hgks_batch_launch_count(const hgks_batch_t *b) { return b ? b->launches : 0ULL; }

extern "C" const char *hgks_batch_last_error(const hgks_batch_t *b) { return b ? b->err : g_batch_err; }

extern "C" void hgks_batch_destroy(hgks_batch_t *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int ph = 0; ph < NPH; ++ph) cudaFree(b->d_tiles[ph]);
    cudaFree(b->arena);
    cudaFree(b->ctl);
    cudaFreeHost(b->ctl_host);
    cudaFree(b->d_inst);
    cudaFree(b->d_inuse);
    cudaFree(b->d_ntiles);
    cudaFreeHost(b->h_tiles);
    cudaFreeHost(b->h_small);
    cudaFreeHost(b->h_inst);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}
