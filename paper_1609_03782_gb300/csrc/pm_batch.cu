// A resident batch of cubes filtered together (the batching line: hundreds
// of galaxy cutouts of uneven size).
//
// The cubes live in a library-owned arena with rows padded to a multiple of
// 16 bytes, so that the streaming kernel's TMA loads work for any nx (the
// TMA needs an aligned row pitch, not an aligned width).  One call
//   1. reduces every cube's FP64 statistics in one launch,
//   2. turns them into each cube's K (K_i = k_i * noise rms, or a given K) and
//      conductance coefficients on the device, with the same double-precision
//      operations as the host does for a single cube,
//   3. runs n_iter launches of the batched streaming kernel, each over the
//      tiles of all cubes (persistent CTAs walking one (cube, tile) list),
// all captured once in a CUDA graph and replayed: one graph launch per call.
// A cube's result is bit-identical to afd_filter_out on that cube alone with
// the same K (the per-voxel arithmetic is the same code).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "afd_batch.h"
#include "afd_trace.h"
#include "afd_ctx.h"
#include "afd_internal.h"
#include "afd_store.cuh"

namespace {

using namespace afd;

constexpr int kBatchStatsThreads = 256;

// Per-cube FP64 statistics over the padded buffer of role 0 (padding is zero
// and changes none of the four sums).  Block b of cube c reads 16-element
// chunks c*16 ... grid-strided over the cube's blocks; float32 pairwise
// sums of 16, promoted to double, fixed combination order.
template <int S>
__global__ void __launch_bounds__(kBatchStatsThreads)
    batch_stats_kernel(const BatchDesc *__restrict__ desc, const int64_t *__restrict__ len,
                       int bpc, double *__restrict__ part)
{
    typedef typename Store<S>::T E;
    const int c = blockIdx.x / bpc;
    const int b = blockIdx.x - c * bpc;
    const E *x = static_cast<const E *>(desc[c].buf[0]);
    const int64_t n = len[c];
    const int64_t nchunk = n / 16;
    double s = 0.0, s2 = 0.0, ns2 = 0.0;
    long long cnt = 0;
    for (int64_t ch = static_cast<int64_t>(b) * blockDim.x + threadIdx.x; ch < nchunk;
         ch += static_cast<int64_t>(bpc) * blockDim.x) {
        float a[16], q[16], d[16];
        if constexpr (S == STORE_F32) {
            const float4 *p = reinterpret_cast<const float4 *>(x + ch * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = p[i];
                a[4 * i] = v.x;
                a[4 * i + 1] = v.y;
                a[4 * i + 2] = v.z;
                a[4 * i + 3] = v.w;
            }
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(x + ch * 16);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const uint4 v = p[i];
                const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a[8 * i + 2 * j] = Store<S>::load(static_cast<E>(w[j] & 0xffffu));
                    a[8 * i + 2 * j + 1] = Store<S>::load(static_cast<E>(w[j] >> 16));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            q[i] = __fmul_rn(a[i], a[i]);
            const bool neg = a[i] < 0.0f;
            d[i] = neg ? q[i] : 0.0f;
            cnt += neg ? 1 : 0;
        }
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
            for (int i = 0; i < w; ++i) {
                a[i] = __fadd_rn(a[i], a[i + w]);
                q[i] = __fadd_rn(q[i], q[i + w]);
                d[i] = __fadd_rn(d[i], d[i + w]);
            }
        s += static_cast<double>(a[0]);
        s2 += static_cast<double>(q[0]);
        ns2 += static_cast<double>(d[0]);
    }
    if (b == 0 && threadIdx.x == 0) {
        for (int64_t i = nchunk * 16; i < n; ++i) {
            const double v = static_cast<double>(Store<S>::load(x[i]));
            s += v;
            s2 += v * v;
            if (v < 0.0) {
                ns2 += v * v;
                cnt += 1;
            }
        }
    }
    double cd = static_cast<double>(cnt);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, off);
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
        ns2 += __shfl_down_sync(0xffffffffu, ns2, off);
        cd += __shfl_down_sync(0xffffffffu, cd, off);
    }
    __shared__ double red[kBatchStatsThreads / 32][4];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[warp][0] = s;
        red[warp][1] = s2;
        red[warp][2] = ns2;
        red[warp][3] = cd;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < kBatchStatsThreads / 32; ++w)
            acc += red[w][threadIdx.x];
        part[static_cast<int64_t>(blockIdx.x) * 4 + threadIdx.x] = acc;
    }
}

// One thread per cube: noise rms from the partials, K, and the coefficients
// (afd::make_coef's operations: double precision, rounded once to float;
// the spacing-only terms B and w come precomputed from the host).
__global__ void batch_coef_kernel(BatchDesc *__restrict__ desc, int count, int bpc,
                                  const double *__restrict__ part, const float *__restrict__ kin,
                                  float *__restrict__ kout, double inv_units, int kind, double dt,
                                  double h0, double h1, double h2, float b0, float b1, float b2)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count)
        return;
    double ns2 = 0.0, nneg = 0.0;
    for (int b = 0; b < bpc; ++b) {
        ns2 += part[(static_cast<int64_t>(c) * bpc + b) * 4 + 2];
        nneg += part[(static_cast<int64_t>(c) * bpc + b) * 4 + 3];
    }
    // statistics are in storage units; sigma in value units
    const double sigma = nneg > 0.0 ? sqrt(ns2 / nneg) * inv_units : 0.0;
    const float kreq = kin[c];
    const float K = kreq < 0.0f ? static_cast<float>(static_cast<double>(-kreq) * sigma) : kreq;
    kout[c] = K;
    // coefficients in storage units: K_s = K * units (exact, units = 2^m)
    const double Kd = static_cast<double>(K) / inv_units;
    Coef k;
    k.ax = static_cast<float>(coef_a_device(Kd, kind, dt, h0));
    k.ay = static_cast<float>(coef_a_device(Kd, kind, dt, h1));
    k.az = static_cast<float>(coef_a_device(Kd, kind, dt, h2));
    k.bx = b0;
    k.by = b1;
    k.bz = b2;
    k.nz = -0.0f;
    k.ai = 0.0f;
    desc[c].coef = k;
    desc[c].K = K;
}

template <int S>
cudaError_t launch_batch_stats(const BatchDesc *desc, const int64_t *len, int count, int bpc,
                               double *part, cudaStream_t st)
{
    batch_stats_kernel<S><<<count * bpc, kBatchStatsThreads, 0, st>>>(desc, len, bpc, part);
    return cudaGetLastError();
}

cudaError_t batch_stats(int S, const BatchDesc *desc, const int64_t *len, int count, int bpc,
                        double *part, cudaStream_t st)
{
    switch (S) {
    case STORE_F32: return launch_batch_stats<STORE_F32>(desc, len, count, bpc, part, st);
    case STORE_F16: return launch_batch_stats<STORE_F16>(desc, len, count, bpc, part, st);
    case STORE_BF16: return launch_batch_stats<STORE_BF16>(desc, len, count, bpc, part, st);
    default: return launch_batch_stats<STORE_I16>(desc, len, count, bpc, part, st);
    }
}

// Tiles of every cube for z-chunk zc (0: 64 planes) under tile kind `kind`
// (0: 64 x 32 tiles, 1: each cube's wide tiles), in cube order, x fastest,
// then stably sorted by chunk length, longest first: the tiles are handed
// out dynamically in this order, so the last ones are the short remainder
// chunks and the CTAs end close together (the tiles of one cube's chunk stay
// together, so neighbouring tiles run at the same time and share their halo
// rows and columns through L2).  Returns the z-chunk used per cube through
// desc.
std::vector<int2> build_tiles(std::vector<BatchDesc> &desc, int zc_req, int kind)
{
    std::vector<int2> list;
    std::vector<int> len;
    for (size_t c = 0; c < desc.size(); ++c) {
        BatchDesc &d = desc[c];
        d.tiles_x = (d.nx + kStreamTX - 1) / kStreamTX;
        d.tiles_y = (d.ny + kStreamTY - 1) / kStreamTY;
        int zc = zc_req > 0 ? zc_req : 64;
        if (zc > d.nz)
            zc = d.nz;
        d.zc = zc;
        const int txy = kind ? d.wtiles_x * d.wtiles_y : d.tiles_x * d.tiles_y;
        const int nt = txy * ((d.nz + zc - 1) / zc);
        for (int t = 0; t < nt; ++t) {
            list.push_back(make_int2(static_cast<int>(c), t));
            const int z0 = (t / txy) * zc;
            len.push_back(std::min(zc, d.nz - z0));
        }
    }
    std::vector<size_t> order(list.size());
    for (size_t i = 0; i < order.size(); ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return len[a] > len[b]; });
    std::vector<int2> sorted(list.size());
    for (size_t i = 0; i < order.size(); ++i)
        sorted[i] = list[order[i]];
    return sorted;
}

void free_batch(afd_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    for (int r = 0; r < 3; ++r)
        if (b->arena[r])
            cudaFree(b->arena[r]);
    if (b->d_desc)
        cudaFree(b->d_desc);
    if (b->d_list)
        cudaFree(b->d_list);
    if (b->d_part)
        cudaFree(b->d_part);
    if (b->h_kin)
        cudaFreeHost(b->h_kin);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    delete b;
}

afd_status upload_tiles(afd_batch *b)
{
    using namespace afd_host;
    std::vector<int2> list = build_tiles(b->h_desc, b->zc, b->tiles);
    if (b->d_list) {
        cudaFree(b->d_list);
        b->d_list = nullptr;
    }
    void *p = nullptr;
    afd_status st = device_alloc(b->ctx, &p, list.size() * sizeof(int2));
    if (st != AFD_OK)
        return st;
    b->d_list = static_cast<int2 *>(p);
    b->ntiles = static_cast<int64_t>(list.size());
    cudaError_t e = cudaMemcpy(b->d_list, list.data(), list.size() * sizeof(int2),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_desc, b->h_desc.data(), b->h_desc.size() * sizeof(BatchDesc),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(b->ctx, e);
    const int64_t gmax = static_cast<int64_t>(b->ctx->sm_count) * batch_bps(b);
    b->grid = static_cast<int>(b->ntiles < gmax ? b->ntiles : gmax);
    if (b->exec) {  // the tile list is baked into the graph
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return AFD_OK;
}

}  // namespace

using namespace afd_host;

extern "C" {

afd_status afd_batch_create(afd_ctx *ctx, afd_batch **out, int count, const int64_t *dims,
                            afd_storage storage, float scale)
{
    if (!ctx || !out || count < 1 || !dims || !storage_ok(storage))
        return AFD_EINVAL;
    if (storage == AFD_F32)
        scale = 1.0f;
    if (!pow2_scale_ok(scale))
        return AFD_EINVAL;
    *out = nullptr;
    for (int c = 0; c < count; ++c)
        if (!dims_ok(dims[3 * c], dims[3 * c + 1], dims[3 * c + 2]))
            return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    if (ctx->stream_bps == 0) {
        cudaError_t e = afd::pm_stream_prepare();
        if (e == cudaSuccess)
            e = afd::pm_stream_occupancy(&ctx->stream_bps);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (ctx->stream_bps < 1)
            ctx->stream_bps = 1;
    }
    if (ctx->wide_bps == 0) {
        cudaError_t e = afd::pm_wide_prepare();
        if (e == cudaSuccess)
            e = afd::pm_wide_occupancy(&ctx->wide_bps);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (ctx->wide_bps < 1)
            ctx->wide_bps = 1;
    }
    afd_batch *b = new (std::nothrow) afd_batch();
    if (!b)
        return AFD_ENOMEM;
    b->ctx = ctx;
    b->count = count;
    b->S = storage;
    b->scale = scale;
    b->units = afd::store_units_per_value(storage, scale);
    const int es = afd::store_bytes(storage);
    const int64_t align = 16 / es;  // elements per 16 bytes
    int64_t total = 0;
    for (int c = 0; c < count; ++c) {
        const int64_t nx = dims[3 * c], ny = dims[3 * c + 1], nz = dims[3 * c + 2];
        const int64_t px = (nx + 7) / 8 * 8;  // 16-byte rows for every storage kind
        b->nx.push_back(nx);
        b->ny.push_back(ny);
        b->nz.push_back(nz);
        b->px.push_back(px);
        b->off.push_back(total);
        total += (px * ny * nz + align - 1) / align * align;
    }
    (void)align;
    b->total = total;
    const size_t bytes = static_cast<size_t>(total) * es;
    for (int r = 0; r < 3; ++r) {
        st = device_alloc(ctx, &b->arena[r], bytes);
        if (st != AFD_OK) {
            free_batch(b);
            return st;
        }
        cudaError_t e = cudaMemset(b->arena[r], 0, bytes);  // padding stays zero
        if (e != cudaSuccess) {
            free_batch(b);
            return cuda_fail(ctx, e);
        }
    }
    b->h_desc.resize(count);
    int box_w = 0, box_h = 0, hx = 0;
    afd::pm_stream_box(storage, &box_w, &box_h, &hx);
    for (int c = 0; c < count; ++c) {
        afd::BatchDesc &d = b->h_desc[c];
        std::memset(static_cast<void *>(&d), 0, sizeof(d));
        d.nx = static_cast<int>(b->nx[c]);
        d.ny = static_cast<int>(b->ny[c]);
        d.nz = static_cast<int>(b->nz[c]);
        d.px = b->px[c];
        afd::pm_wide_shape(storage, d.nx, &d.wtx, &d.wty, &d.wtiles_x);
        d.wtiles_y = (d.ny + d.wty - 1) / d.wty;
        for (int r = 0; r < 3; ++r) {
            d.buf[r] = static_cast<char *>(b->arena[r]) + b->off[c] * es;
            st = encode_pitched_map(ctx, &d.map[r], d.buf[r], storage, box_w, box_h, d.nx, d.ny,
                                    d.nz, d.px);
            if (st == AFD_OK)
                st = encode_pitched_map(ctx, &d.mapw[r], d.buf[r], storage, d.wtx + 2 * (16 / es),
                                        d.wty + 2, d.nx, d.ny, d.nz, d.px);
            if (st != AFD_OK) {
                free_batch(b);
                return st;
            }
        }
    }
    // device tables: descriptors, per-cube lengths (for the stats), partials, K
    void *p = nullptr;
    const size_t small = count * sizeof(afd::BatchDesc) + 64;
    if ((st = device_alloc(ctx, &p, small)) != AFD_OK) {
        free_batch(b);
        return st;
    }
    b->d_desc = static_cast<afd::BatchDesc *>(p);
    const size_t aux = count * (sizeof(int64_t) + b->bpc * 4 * sizeof(double) + 2 * sizeof(float));
    if ((st = device_alloc(ctx, &p, aux + 256)) != AFD_OK) {
        free_batch(b);
        return st;
    }
    b->d_part = static_cast<double *>(p);
    int64_t *d_len = reinterpret_cast<int64_t *>(b->d_part + static_cast<size_t>(count) * b->bpc * 4);
    b->d_kin = reinterpret_cast<float *>(d_len + count);
    b->d_kout = b->d_kin + count;
    std::vector<int64_t> len(count);
    for (int c = 0; c < count; ++c)
        len[c] = b->px[c] * b->ny[c] * b->nz[c];
    cudaError_t e = cudaMemcpy(d_len, len.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMallocHost(reinterpret_cast<void **>(&b->h_kin), count * sizeof(float));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        st = cuda_fail(ctx, e);
        free_batch(b);
        return st;
    }
    if ((st = upload_tiles(b)) != AFD_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return AFD_OK;
}

afd_status afd_batch_destroy(afd_batch *b)
{
    if (!b)
        return AFD_OK;
    set_device(b->ctx);
    cudaStreamSynchronize(b->ctx->stream);
    free_batch(b);
    return AFD_OK;
}

afd_status afd_batch_set_tiles(afd_batch *b, int kind)
{
    if (!b || (kind != AFD_TILES_64X32 && kind != AFD_TILES_WIDE))
        return AFD_EINVAL;
    afd_status st = set_device(b->ctx);
    if (st != AFD_OK)
        return st;
    cudaStreamSynchronize(b->ctx->stream);
    b->tiles = kind;
    return upload_tiles(b);
}

afd_status afd_batch_set_zchunk(afd_batch *b, int zc)
{
    if (!b || zc < 0)
        return AFD_EINVAL;
    afd_status st = set_device(b->ctx);
    if (st != AFD_OK)
        return st;
    cudaStreamSynchronize(b->ctx->stream);
    b->zc = zc;
    return upload_tiles(b);
}

// Copy a dense cube (rows of nx elements) into / out of the padded arena.
static afd_status batch_copy(afd_batch *b, int i, const void *src, void *dst, int role, bool in)
{
    if (!b || i < 0 || i >= b->count || (in ? !src : !dst))
        return AFD_EINVAL;
    afd_status st = set_device(b->ctx);
    if (st != AFD_OK)
        return st;
    const size_t es = static_cast<size_t>(afd::store_bytes(b->S));
    char *cube = static_cast<char *>(b->arena[role]) + b->off[i] * es;
    const size_t width = static_cast<size_t>(b->nx[i]) * es;
    const size_t pitch = static_cast<size_t>(b->px[i]) * es;
    const size_t rows = static_cast<size_t>(b->ny[i] * b->nz[i]);
    cudaError_t e = in ? cudaMemcpy2DAsync(cube, pitch, src, width, width, rows,
                                           cudaMemcpyDefault, b->ctx->stream)
                       : cudaMemcpy2DAsync(dst, width, cube, pitch, width, rows,
                                           cudaMemcpyDefault, b->ctx->stream);
    return e == cudaSuccess ? AFD_OK : cuda_fail(b->ctx, e);
}

afd_status afd_batch_set(afd_batch *b, int i, const void *cube)
{
    return batch_copy(b, i, cube, nullptr, 0, true);
}

afd_status afd_batch_get(afd_batch *b, int i, void *cube)
{
    return batch_copy(b, i, nullptr, cube, 1, false);
}

afd_status afd_batch_filter(afd_batch *b, const float *K, const float *spacing, float dt,
                            int n_iter, afd_conductance cond)
{
    const afd_host::TraceRange trace_("afd_batch_filter");
    if (!b || !K || !params_ok(spacing, 1.0f, dt, n_iter, cond) || n_iter < 1)
        return AFD_EINVAL;
    bool lin = false, fin = false;
    for (int c = 0; c < b->count; ++c) {
        if (std::isnan(K[c]) || K[c] == 0.0f || (std::isinf(K[c]) && K[c] < 0.0f))
            return AFD_EINVAL;
        if (std::isinf(K[c]))
            lin = true;
        else
            fin = true;
    }
    if (lin && fin)
        return AFD_EINVAL;  // one conductance kind per call
    afd_ctx *ctx = b->ctx;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const float h[3] = {spacing ? spacing[0] : 1.0f, spacing ? spacing[1] : 1.0f,
                        spacing ? spacing[2] : 1.0f};
    int kind = 0;
    // the spacing-only coefficients (B) come from the host formulas
    const afd::Coef base = afd::make_coef(h, lin ? INFINITY : 1.0f, dt,
                                          cond == AFD_COND_EXPONENTIAL, &kind);
    const bool same = b->exec && b->g_n == n_iter && b->g_cond == cond && b->g_kind == kind &&
                      b->g_dt == dt && b->g_h[0] == h[0] && b->g_h[1] == h[1] &&
                      b->g_h[2] == h[2] && b->g_zc == b->zc && b->g_tiles == b->tiles;
    cudaError_t e = cudaSuccess;
    if (!same) {
        if (b->exec) {
            cudaStreamSynchronize(ctx->stream);
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            // the passes' tile counter starts from zero at every replay
            cudaError_t le = cudaMemsetAsync(ctx->d_tiles, 0, sizeof(unsigned long long), b->cap);
            if (le == cudaSuccess)
                le = batch_stats(b->S, b->d_desc,
                                         reinterpret_cast<const int64_t *>(
                                             b->d_part + static_cast<size_t>(b->count) * b->bpc * 4),
                                         b->count, b->bpc, b->d_part, b->cap);
            if (le == cudaSuccess) {
                batch_coef_kernel<<<(b->count + 127) / 128, 128, 0, b->cap>>>(
                    b->d_desc, b->count, b->bpc, b->d_part, b->d_kin, b->d_kout, 1.0 / b->units,
                    kind, static_cast<double>(dt), h[0], h[1], h[2], base.bx, base.by, base.bz);
                le = cudaGetLastError();
            }
            for (int i = 0; i < n_iter && le == cudaSuccess; ++i) {
                const int dst = ((n_iter - 1 - i) & 1) ? 2 : 1;
                const int src = i == 0 ? 0 : (((n_iter - i) & 1) ? 2 : 1);
                le = batch_launch(b, kind, b->d_desc, b->d_list, nullptr, b->ntiles, src, dst,
                                  b->grid, ctx->d_tiles,
                                  static_cast<unsigned long long>(i) *
                                      static_cast<unsigned long long>(b->ntiles),
                                  i > 0, ctx->d_err, b->cap);
            }
            e = cudaStreamEndCapture(b->cap, &graph);
            if (e == cudaSuccess)
                e = le;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph)
            cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(ctx, e);
        }
        b->g_n = n_iter;
        b->g_cond = cond;
        b->g_kind = kind;
        b->g_dt = dt;
        b->g_h[0] = h[0];
        b->g_h[1] = h[1];
        b->g_h[2] = h[2];
        b->g_zc = b->zc;
        b->g_tiles = b->tiles;
    }
    // K requests: through pinned staging, stream-ordered before the graph
    e = cudaStreamSynchronize(ctx->stream);  // the staging buffer may still be read
    if (e == cudaSuccess) {
        std::memcpy(b->h_kin, K, b->count * sizeof(float));
        e = cudaMemcpyAsync(b->d_kin, b->h_kin, b->count * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaGraphLaunch(b->exec, ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    ctx->launches += 2 + n_iter;
    return AFD_OK;
}

afd_status afd_batch_k(afd_batch *b, float *K_out)
{
    if (!b || !K_out)
        return AFD_EINVAL;
    afd_status st = set_device(b->ctx);
    if (st != AFD_OK)
        return st;
    cudaError_t e = cudaMemcpyAsync(K_out, b->d_kout, b->count * sizeof(float),
                                    cudaMemcpyDeviceToHost, b->ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->ctx->stream);
    return e == cudaSuccess ? AFD_OK : cuda_fail(b->ctx, e);
}

}  // extern "C"
