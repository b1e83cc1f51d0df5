// The resident batch (opaque to callers), shared with the serving engine.
#pragma once

#include <cstdint>
#include <vector>

#include "afd_ctx.h"
#include "afd_internal.h"

struct afd_batch {
    afd_ctx *ctx = nullptr;
    int count = 0;
    int S = 0;
    float scale = 1.0f;
    double units = 1.0;  // storage units per value unit
    std::vector<int64_t> nx, ny, nz, px, off;  // off: element offset of each cube
    int64_t total = 0;                          // elements per role
    void *arena[3] = {nullptr, nullptr, nullptr};
    std::vector<afd::BatchDesc> h_desc;
    afd::BatchDesc *d_desc = nullptr;
    int2 *d_list = nullptr;
    int64_t ntiles = 0;
    int zc = 0;  // 0 = automatic
    int tiles = 1;  // 0: 64 x 32 tiles (4 x 2 voxels per thread); 1: per-cube wide tiles (8 x 2)
    int grid = 0;
    int bpc = 8;                 // stats blocks per cube
    double *d_part = nullptr;    // stats partials: count * bpc * 4
    float *d_kin = nullptr;      // K requests (device), count
    float *h_kin = nullptr;      // pinned staging of the K requests
    float *d_kout = nullptr;     // K used, count
    cudaStream_t cap = nullptr;  // private capture stream
    cudaGraphExec_t exec = nullptr;
    // parameters the captured graph was built for
    int g_n = -1, g_cond = -1, g_kind = -1;
    float g_dt = 0.0f, g_h[3] = {0, 0, 0};
    int g_zc = -1, g_tiles = -1;
};

// Tiles of cube c per z-chunk under the batch's tile kind.
inline int64_t batch_cube_txy(const afd_batch *b, int c)
{
    const afd::BatchDesc &d = b->h_desc[c];
    return b->tiles ? static_cast<int64_t>(d.wtiles_x) * d.wtiles_y
                    : static_cast<int64_t>(d.tiles_x) * d.tiles_y;
}

// One batched pass under the batch's tile kind.
inline cudaError_t batch_launch(const afd_batch *b, int cond, const afd::BatchDesc *desc,
                                const int2 *list, const int2 *roles, int64_t ntiles, int src,
                                int dst, int grid, unsigned long long *ctr,
                                unsigned long long base, bool pdl, int *err, cudaStream_t st)
{
    if (b->tiles)
        return afd::launch_pm_wide_batch(b->S, cond, desc, list, roles, ntiles, src, dst, grid,
                                         ctr, base, pdl, err, st);
    return afd::launch_pm_batch(b->S, cond, desc, list, roles, ntiles, src, dst, grid, ctr, base,
                                pdl, err, st);
}

// CTAs per SM of the batch's kernel.
inline int batch_bps(const afd_batch *b)
{
    const int v = b->tiles ? b->ctx->wide_bps : b->ctx->stream_bps;
    return v > 0 ? v : 1;
}

