// C ABI of the anisotropic-diffusion library (declared in include/afd.h).
//
// Host-side logic only: argument validation, per-call coefficients, scratch
// management, kernel selection, TMA descriptor encoding and the ping-pong
// iteration driver.  Every step of the filter runs in the CUDA kernels of
// this directory.
#include <cmath>
#include <algorithm>
#include <vector>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/afd.h"
#include "afd_ctx.h"
#include "afd_trace.h"
#include "afd_check.cuh"
#include "afd_internal.h"
#include "afd_store.cuh"


namespace afd_host {

// ---- fault injection: AFD_FAULT=alloc:N makes the N-th scratch allocation
// of the process fail as if the device were out of memory (host side only).
std::mutex g_fault_mu;
long g_alloc_calls = 0;

bool injected_alloc_failure()
{
    const char *f = std::getenv("AFD_FAULT");
    if (!f || std::strncmp(f, "alloc:", 6) != 0)
        return false;
    const long n = std::strtol(f + 6, nullptr, 10);
    std::lock_guard<std::mutex> lk(g_fault_mu);
    return ++g_alloc_calls == n;
}

afd_status cuda_fail(afd_ctx *ctx, cudaError_t e)
{
    if (ctx)
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "%s: %s", cudaGetErrorName(e),
                      cudaGetErrorString(e));
    return AFD_ECUDA;
}

afd_status device_alloc(afd_ctx *ctx, void **p, size_t bytes)
{
    if (injected_alloc_failure())
        return AFD_ENOMEM;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return AFD_ENOMEM;
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    return AFD_OK;
}

// Grow a context-owned device buffer to at least `bytes`.
afd_status ensure_buffer(afd_ctx *ctx, float **buf, size_t *cap, size_t bytes)
{
    if (*cap >= bytes)
        return AFD_OK;
    if (*buf) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    void *p = nullptr;
    afd_status st = device_alloc(ctx, &p, bytes);
    if (st != AFD_OK)
        return st;
    *buf = static_cast<float *>(p);
    *cap = bytes;
    return AFD_OK;
}

bool dims_ok(int64_t nx, int64_t ny, int64_t nz)
{
    if (nx < 1 || ny < 1 || nz < 1)
        return false;
    const int64_t imax = std::numeric_limits<int>::max();
    if (nx > imax || ny > imax || nz > imax)
        return false;
    const int64_t lim = std::numeric_limits<int64_t>::max() / 8;
    if (nx > lim / ny || nx * ny > lim / nz)
        return false;
    return true;
}

bool params_ok(const float *spacing, float K, float dt, int n_iter, afd_conductance cond)
{
    if (cond != AFD_COND_EXPONENTIAL && cond != AFD_COND_RATIONAL)
        return false;
    if (spacing)
        for (int a = 0; a < 3; ++a)
            if (!(spacing[a] > 0.0f) || !std::isfinite(spacing[a]))
                return false;
    if (std::isnan(K) || K < 0.0f)
        return false;
    if (!(dt > 0.0f) || !std::isfinite(dt))
        return false;
    return n_iter >= 0;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool resolve_encode()
{
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

afd_status encode_plane_map(afd_ctx *ctx, CUtensorMap *map, const float *ptr, int nx, int ny,
                            int nz)
{
    if (!resolve_encode()) {
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "cuTensorMapEncodeTiled unavailable");
        return AFD_ECUDA;
    }
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                                static_cast<cuuint64_t>(nz)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(nx) * 4,
                                   static_cast<cuuint64_t>(nx) * static_cast<cuuint64_t>(ny) * 4};
    const cuuint32_t box[3] = {afd::kStreamTX + 8, afd::kStreamTY + 2, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "cuTensorMapEncodeTiled failed (%d)",
                      static_cast<int>(r));
        return AFD_ECUDA;
    }
    return AFD_OK;
}

bool stream_kernel_fits(const float *a, const float *b, int64_t nx)
{
    return (nx % 4) == 0 && (reinterpret_cast<uintptr_t>(a) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(b) & 15u) == 0;
}

afd_status set_device(afd_ctx *ctx)
{
    cudaError_t e = cudaSetDevice(ctx->device);
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

// Pass timing: record a begin event now and hand back the end event to be
// recorded after the passes.
cudaError_t timing_begin(afd_ctx *ctx, cudaEvent_t *end)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess)
        e = cudaEventCreate(&b);
    if (e == cudaSuccess)
        e = cudaEventRecord(a, ctx->stream);
    if (e != cudaSuccess) {
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
        return e;
    }
    ctx->tev.push_back(a);
    ctx->tev.push_back(b);
    *end = b;
    return cudaSuccess;
}

// Zero the streaming kernel's tile counter (stream-ordered) before a sequence
// of launches.
cudaError_t tiles_reset(afd_ctx *ctx)
{
    ctx->tiles_base = 0;
    return cudaMemsetAsync(ctx->d_tiles, 0, sizeof(unsigned long long), ctx->stream);
}

// The iteration driver shared by afd_filter, afd_filter_out and
// afd_filter_host.  Pass i reads src_i and writes dst_i, src_0 = in,
// src_i = dst_{i-1}.  Out of place (in != out) the destinations alternate
// between `out` and scratch so that the last pass lands in `out`; in place
// they alternate starting with scratch, and an odd count ends with a copy.
afd_status run_passes(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                      int64_t nz, int kind, const afd::Coef &k, int n_iter,
                      const afd::Coef *kdev = nullptr);

// What a host-staged call filters with: a conductance kind and its
// coefficients, or the identity.
struct DeviceFilter {
    int kind;
    afd::Coef k;
    bool identity;
};

// The per-face filter of afd_filter (K = 0: the identity).
DeviceFilter per_face_filter(const float *spacing, float K, float dt, afd_conductance cond)
{
    DeviceFilter f{};
    f.identity = K == 0.0f;
    if (!f.identity)
        f.k = afd::make_coef(spacing, K, dt, cond == AFD_COND_EXPONENTIAL, &f.kind);
    return f;
}

// The intensity-driven filter of afd_filter_intensity (K = 0 or rms = 0:
// the identity).
DeviceFilter intensity_filter(const float *C, float K, float rms, float tau)
{
    DeviceFilter f{};
    f.identity = K == 0.0f || rms == 0.0f;
    f.kind = afd::COND_INT;
    if (!f.identity)
        f.k = afd::make_coef_intensity(C, K, rms, tau);
    return f;
}

// The intensity form's parameters as afd_filter_intensity accepts them.
bool intensity_args_ok(const float *C, float K, float rms, float tau, int n_iter)
{
    if (!C || n_iter < 0)
        return false;
    for (int a = 0; a < 3; ++a)
        if (!(C[a] >= 0.0f) || !std::isfinite(C[a]))
            return false;
    return !(std::isnan(K) || K < 0.0f || std::isnan(rms) || rms < 0.0f || !(tau > 0.0f) ||
             !std::isfinite(tau));
}

afd_status filter_device(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                         int64_t nz, const DeviceFilter &f, int n_iter)
{
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * sizeof(float);
    if (n_iter == 0 || f.identity) {
        cudaError_t e = cudaSuccess;
        if (in != out)
            e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
    }
    return run_passes(ctx, in, out, nx, ny, nz, f.kind, f.k, n_iter);
}

afd_status filter_device(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                         int64_t nz, const float *spacing, float K, float dt, int n_iter,
                         afd_conductance cond)
{
    return filter_device(ctx, in, out, nx, ny, nz, per_face_filter(spacing, K, dt, cond),
                         n_iter);
}

// n_iter >= 1 passes of conductance kind `kind` with coefficients k, or
// with the coefficients at kdev (device memory; streaming kernel only).
afd_status run_passes(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                      int64_t nz, int kind, const afd::Coef &k, int n_iter,
                      const afd::Coef *kdev)
{
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * sizeof(float);
    cudaError_t e = cudaSuccess;
    afd_status st = ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, bytes);
    if (st != AFD_OK)
        return st;

    const afd::PassSeq q{kind, in, out, ctx->scratch, static_cast<int>(nx), static_cast<int>(ny),
                         static_cast<int>(nz), k, n_iter, ctx->stream, &ctx->launches};

    const bool fits = stream_kernel_fits(in, out, nx) &&
                      (reinterpret_cast<uintptr_t>(ctx->scratch) & 15u) == 0;
    bool use_stream = false;
    if (ctx->kernel == AFD_KERNEL_STREAM) {
        if (!fits)
            return AFD_EINVAL;
        use_stream = true;
    } else if (ctx->kernel == AFD_KERNEL_AUTO || ctx->kernel == AFD_KERNEL_TWO_STAGE) {
        use_stream = fits;
    }
    if (kdev && !use_stream)
        return AFD_EINVAL;  // callers check this first

    if (use_stream) {
        if (ctx->stream_bps == 0) {
            e = afd::pm_stream_prepare();
            if (e == cudaSuccess)
                e = afd::pm_stream_occupancy(&ctx->stream_bps);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e);
            if (ctx->stream_bps < 1)
                ctx->stream_bps = 1;
        }
        // one TMA descriptor per distinct source buffer
        const float *srcs[3] = {in, out, ctx->scratch};
        CUtensorMap maps[3];
        for (int b = 0; b < 3; ++b) {
            st = encode_plane_map(ctx, &maps[b], srcs[b], static_cast<int>(nx),
                                  static_cast<int>(ny), static_cast<int>(nz));
            if (st != AFD_OK)
                return st;
        }
        afd::StreamPlan plan =
            afd::pm_stream_plan(static_cast<int>(nx), static_cast<int>(ny), static_cast<int>(nz),
                                ctx->sm_count, ctx->stream_bps, ctx->zc_hint);
        plan.kdev = kdev;
        e = tiles_reset(ctx);
        cudaEvent_t tend = nullptr;
        if (e == cudaSuccess && ctx->timing)
            e = timing_begin(ctx, &tend);
        if (e == cudaSuccess)
            e = afd::stream_passes(q, maps, plan, ctx->d_tiles, &ctx->tiles_base, ctx->d_err);
        if (e == cudaSuccess && tend) {
            e = cudaEventRecord(tend, ctx->stream);
            ctx->timed_passes += n_iter;
        }
    } else {
        e = afd::simple_passes(q);
    }
    if (e == cudaSuccess)
        e = afd::passes_finish(q);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    return AFD_OK;
}


bool pow2_scale_ok(float scale)
{
    if (!(scale > 0.0f) || !std::isfinite(scale))
        return false;
    int e = 0;
    return std::frexp(static_cast<double>(scale), &e) == 0.5;
}

bool storage_ok(int s) { return s == AFD_F32 || s == AFD_F16 || s == AFD_BF16 || s == AFD_I16FIX; }

// Encode a 3-D TMA map over a cube of storage kind S with the given box.
afd_status encode_box_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int box_w,
                          int box_h, int nx, int ny, int nz);

// Encode a 3-D TMA map over a cube of storage kind S for the temporally
// blocked kernel of depth T.
afd_status encode_tb_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int T, int nx,
                         int ny, int nz)
{
    const afd::TbShape sh = afd::tb_shape(S, T);
    return encode_box_map(ctx, map, ptr, S, sh.box_w, sh.box_h, nx, ny, nz);
}

afd_status encode_box_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int box_w,
                          int box_h, int nx, int ny, int nz)
{
    return encode_pitched_map(ctx, map, ptr, S, box_w, box_h, nx, ny, nz, nx);
}

afd_status encode_pitched_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int box_w,
                              int box_h, int nx, int ny, int nz, int64_t pitch)
{
    if (!resolve_encode()) {
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "cuTensorMapEncodeTiled unavailable");
        return AFD_ECUDA;
    }
    const cuuint64_t es = static_cast<cuuint64_t>(afd::store_bytes(S));
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                                static_cast<cuuint64_t>(nz)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(pitch) * es,
                                   static_cast<cuuint64_t>(pitch) * static_cast<cuuint64_t>(ny) * es};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map,
                          S == AFD_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                          3, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "cuTensorMapEncodeTiled failed (%d)",
                      static_cast<int>(r));
        return AFD_ECUDA;
    }
    return AFD_OK;
}

// One pass of depth T without the temporally blocked kernel (layout it cannot
// stage, or K = +inf): dequantise into float32 scratch, T float32
// iterations, quantise.  The same arithmetic, so the same bits.
afd_status fallback_pass(afd_ctx *ctx, int S, float units, const void *src, void *dst, int64_t nx,
                         int64_t ny, int64_t nz, const float *spacing, float K, float dt, int T,
                         afd_conductance cond)
{
    const int64_t n = nx * ny * nz;
    const size_t fbytes = static_cast<size_t>(n) * sizeof(float);
    if (S == AFD_F32)
        return filter_device(ctx, static_cast<const float *>(src), static_cast<float *>(dst), nx,
                             ny, nz, spacing, K, dt, T, cond);
    afd_status st = ensure_buffer(ctx, &ctx->fb_scratch, &ctx->fb_scratch_bytes, 2 * fbytes);
    if (st != AFD_OK)
        return st;
    float *a = ctx->fb_scratch, *b = ctx->fb_scratch + n;
    cudaError_t e = afd::launch_dequantize(S, src, a, n, units, ctx->stream);
    ctx->launches++;
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    st = filter_device(ctx, a, b, nx, ny, nz, spacing, K, dt, T, cond);
    if (st != AFD_OK)
        return st;
    e = afd::launch_quantize(S, b, dst, n, units, ctx->stream);
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status stats_device(afd_ctx *ctx, const float *cube, int64_t n, double *out4)
{
    cudaError_t e = afd::launch_stats(cube, n, ctx->d_part, ctx->part_blocks, out4, ctx->stream);
    ctx->launches += 2;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status stats_host(afd_ctx *ctx, const float *cube, int64_t n)
{
    afd_status st = stats_device(ctx, cube, n, ctx->d_out4);
    if (st != AFD_OK)
        return st;
    cudaError_t e = cudaMemcpyAsync(ctx->h_out4, ctx->d_out4, 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

}  // namespace afd_host

using namespace afd_host;

extern "C" {

afd_status afd_create(afd_ctx **out, int device, void *cuda_stream)
{
    if (!out)
        return AFD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return AFD_EINVAL;
    }
    afd_ctx *ctx = new (std::nothrow) afd_ctx();
    if (!ctx)
        return AFD_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        afd_status st = cuda_fail(ctx, e);
        delete ctx;
        return st;
    }
    ctx->part_blocks = ctx->sm_count * 4;
    const size_t small = sizeof(int) * 32 + sizeof(double) * 4 +
                         sizeof(double) * 4 * static_cast<size_t>(ctx->part_blocks) +
                         sizeof(afd::Coef);
    void *p = nullptr;
    afd_status st = device_alloc(ctx, &p, small);
    if (st != AFD_OK) {
        delete ctx;
        return st;
    }
    ctx->d_err = static_cast<int *>(p);
    ctx->d_tiles = reinterpret_cast<unsigned long long *>(ctx->d_err + 16);
    ctx->d_out4 = reinterpret_cast<double *>(static_cast<char *>(p) + sizeof(int) * 32);
    ctx->d_part = ctx->d_out4 + 4;
    ctx->d_coef = reinterpret_cast<afd::Coef *>(ctx->d_part + 4 * ctx->part_blocks);
    e = cudaMemset(ctx->d_err, 0, sizeof(int) * 32);
    if (e == cudaSuccess)
        e = cudaMallocHost(reinterpret_cast<void **>(&ctx->h_out4), 4 * sizeof(double));
    if (e != cudaSuccess) {
        st = cuda_fail(ctx, e);
        cudaFree(ctx->d_err);
        delete ctx;
        return st;
    }
    *out = ctx;
    return AFD_OK;
}

afd_status afd_destroy(afd_ctx *ctx)
{
    if (!ctx)
        return AFD_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < 2; ++i) {
        afd_ctx::HostSlot &s = ctx->host_slot[i];
        if (s.copied_out)
            cudaEventSynchronize(s.copied_out);
        if (s.buf)
            cudaFree(s.buf);
        if (s.copied_in)
            cudaEventDestroy(s.copied_in);
        if (s.filtered)
            cudaEventDestroy(s.filtered);
        if (s.copied_out)
            cudaEventDestroy(s.copied_out);
    }
    if (ctx->h2d_stream) {
        cudaStreamSynchronize(ctx->h2d_stream);
        cudaStreamDestroy(ctx->h2d_stream);
    }
    if (ctx->d2h_stream) {
        cudaStreamSynchronize(ctx->d2h_stream);
        cudaStreamDestroy(ctx->d2h_stream);
    }
    if (ctx->scratch)
        cudaFree(ctx->scratch);
    if (ctx->fd_buf)
        cudaFree(ctx->fd_buf);
    if (ctx->lp_scratch)
        cudaFree(ctx->lp_scratch);
    if (ctx->chain_f32)
        cudaFree(ctx->chain_f32);
    if (ctx->fb_scratch)
        cudaFree(ctx->fb_scratch);
    for (cudaEvent_t ev : ctx->tev)
        cudaEventDestroy(ev);
    if (ctx->d_err)
        cudaFree(ctx->d_err);
    if (ctx->h_out4)
        cudaFreeHost(ctx->h_out4);
    delete ctx;
    return AFD_OK;
}

afd_status afd_set_stream(afd_ctx *ctx, void *cuda_stream)
{
    if (!ctx)
        return AFD_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return AFD_OK;
}

afd_status afd_set_kernel(afd_ctx *ctx, afd_kernel kernel)
{
    if (!ctx || (kernel != AFD_KERNEL_AUTO && kernel != AFD_KERNEL_SIMPLE &&
                 kernel != AFD_KERNEL_STREAM && kernel != AFD_KERNEL_TWO_STAGE))
        return AFD_EINVAL;
    ctx->kernel = kernel;
    return AFD_OK;
}

afd_status afd_set_stream_zchunk(afd_ctx *ctx, int zc)
{
    if (!ctx || zc < 0)
        return AFD_EINVAL;
    ctx->zc_hint = zc;
    return AFD_OK;
}

afd_status afd_filter(afd_ctx *ctx, float *cube, int64_t nx, int64_t ny, int64_t nz,
                      const float *spacing, float K, float dt, int n_iter, afd_conductance cond)
{
    const afd_host::TraceRange trace_("afd_filter");
    if (!ctx || !cube || !dims_ok(nx, ny, nz) || !params_ok(spacing, K, dt, n_iter, cond))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    return filter_device(ctx, cube, cube, nx, ny, nz, spacing, K, dt, n_iter, cond);
}

afd_status afd_filter_out(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const float *spacing, float K, float dt, int n_iter,
                          afd_conductance cond)
{
    const afd_host::TraceRange trace_("afd_filter_out");
    if (!ctx || !in || !out || !dims_ok(nx, ny, nz) ||
        !params_ok(spacing, K, dt, n_iter, cond))
        return AFD_EINVAL;
    if (in != out) {  // partial overlap would corrupt the input mid-filter
        const size_t bytes = static_cast<size_t>(nx * ny * nz) * sizeof(float);
        const char *a = reinterpret_cast<const char *>(in);
        const char *b = reinterpret_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes)
            return AFD_EINVAL;
    }
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    return filter_device(ctx, in, out, nx, ny, nz, spacing, K, dt, n_iter, cond);
}

afd_status afd_filter_rel(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const float *spacing, float k_rms, float dt, int n_iter,
                          afd_conductance cond, float *K_out)
{
    const afd_host::TraceRange trace_("afd_filter_rel");
    if (!ctx || !in || !out || !dims_ok(nx, ny, nz) || !(k_rms > 0.0f) || !std::isfinite(k_rms) ||
        !params_ok(spacing, 1.0f, dt, n_iter, cond))
        return AFD_EINVAL;
    const int64_t n = nx * ny * nz;
    if (in != out) {
        const size_t bytes = static_cast<size_t>(n) * sizeof(float);
        const char *a = reinterpret_cast<const char *>(in);
        const char *b = reinterpret_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes)
            return AFD_EINVAL;
    }
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const bool on_device = ctx->kernel != AFD_KERNEL_SIMPLE && n_iter > 0 &&
                           stream_kernel_fits(in, out, nx);
    if (!on_device) {
        // through the host: the same rms, K and host coefficients
        double rms = 0.0;
        st = afd_noise_rms(ctx, in, n, &rms);
        if (st != AFD_OK)
            return st;
        const float K = static_cast<float>(static_cast<double>(k_rms) * rms);
        if (K_out) {
            cudaError_t e = cudaMemcpy(K_out, &K, sizeof(float), cudaMemcpyHostToDevice);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e);
        }
        return filter_device(ctx, in, out, nx, ny, nz, spacing, K, dt, n_iter, cond);
    }
    st = stats_device(ctx, in, n, ctx->d_out4);
    if (st != AFD_OK)
        return st;
    int kind = 0;
    // B terms (independent of K) and the kind from the host formulas
    const afd::Coef b = afd::make_coef(spacing, 1.0f, dt, cond == AFD_COND_EXPONENTIAL, &kind);
    const double h[3] = {spacing ? spacing[0] : 1.0, spacing ? spacing[1] : 1.0,
                         spacing ? spacing[2] : 1.0};
    cudaError_t e = afd::launch_rel_coef(ctx->d_out4, static_cast<double>(k_rms), kind,
                                         static_cast<double>(dt), h, b, ctx->d_coef, K_out,
                                         ctx->stream);
    ctx->launches++;
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    return run_passes(ctx, in, out, nx, ny, nz, kind, b, n_iter, ctx->d_coef);
}

namespace {
// The smallest float >= t (so that, for a float I, I >= t exactly when
// I >= the result).
float float_at_or_above(double t)
{
    float f = static_cast<float>(t);
    if (static_cast<double>(f) < t)
        f = std::nextafter(f, INFINITY);
    return f;
}
}  // namespace

afd_status afd_f_diagnostic(afd_ctx *ctx, const float *orig, const float *filt,
                            const float *model, int64_t nx, int64_t ny, int64_t nz,
                            const int64_t *roi, double rms_o, double rms_f, double nsig,
                            double beam, afd_fdiag *out)
{
    const afd_host::TraceRange trace_("afd_f_diagnostic");
    if (!ctx || !orig || !filt || !out || !dims_ok(nx, ny, nz) || !(nsig > 0.0) ||
        !std::isfinite(nsig) || !(beam >= 1.0) || !std::isfinite(beam) || std::isnan(rms_o) ||
        std::isnan(rms_f) || std::isinf(rms_o) || std::isinf(rms_f))
        return AFD_EINVAL;
    int64_t box[6] = {0, nx, 0, ny, 0, nz};
    if (roi)
        for (int i = 0; i < 6; ++i)
            box[i] = roi[i];
    if (box[0] < 0 || box[1] > nx || box[0] >= box[1] || box[2] < 0 || box[3] > ny ||
        box[2] >= box[3] || box[4] < 0 || box[5] > nz || box[4] >= box[5])
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const int64_t n = nx * ny * nz;
    // noise levels: given, or the estimate of each full cube (Sec. 4 assumes
    // the rms constant over the cube)
    if (rms_o <= 0.0 && (st = afd_noise_rms(ctx, orig, n, &rms_o)) != AFD_OK)
        return st;
    if (rms_f <= 0.0 && (st = afd_noise_rms(ctx, filt, n, &rms_f)) != AFD_OK)
        return st;
    const size_t part_bytes = static_cast<size_t>(ctx->part_blocks) * 6 * sizeof(double);
    st = ensure_buffer(ctx, &ctx->fd_buf, &ctx->fd_bytes, part_bytes + 6 * sizeof(double));
    if (st != AFD_OK)
        return st;
    double *part = reinterpret_cast<double *>(ctx->fd_buf);
    double *out6 = part + static_cast<size_t>(ctx->part_blocks) * 6;
    const int box32[6] = {static_cast<int>(box[0]), static_cast<int>(box[1]),
                          static_cast<int>(box[2]), static_cast<int>(box[3]),
                          static_cast<int>(box[4]), static_cast<int>(box[5])};
    const float t_o = float_at_or_above(nsig * rms_o);
    const float t_f = float_at_or_above(nsig * rms_f);
    cudaError_t e = afd::launch_fdiag(orig, filt, model, nx, ny, box32, t_o, t_f, part,
                                      ctx->part_blocks, out6, ctx->stream);
    ctx->launches += 2;
    double h[6];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, out6, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    afd_fdiag r;
    r.S_of = h[0];
    r.S_oo = h[1];
    r.S_mf = h[2];
    r.S_m = h[3];
    r.N_o = static_cast<int64_t>(h[4]);
    r.N_f = static_cast<int64_t>(h[5]);
    r.rms_o = rms_o;
    r.rms_f = rms_f;
    const double nan = std::nan("");
    r.F = r.S_oo != 0.0 ? std::fabs(r.S_of) / std::fabs(r.S_oo) : nan;
    const double sig_of = std::sqrt(static_cast<double>(r.N_f) / beam) * rms_f;
    const double sig_oo = std::sqrt(static_cast<double>(r.N_o) / beam) * rms_o;
    r.sigma_F = r.S_oo != 0.0 ? std::sqrt(sig_of * sig_of / (r.S_oo * r.S_oo) +
                                          r.S_of * r.S_of * sig_oo * sig_oo /
                                              (r.S_oo * r.S_oo * r.S_oo * r.S_oo))
                              : nan;
    r.F_M = (model && r.S_m != 0.0) ? std::fabs(r.S_mf) / std::fabs(r.S_m) : nan;
    *out = r;
    return AFD_OK;
}

namespace {
bool cubes_disjoint(const float *a, const float *b, int64_t n)
{
    const char *pa = reinterpret_cast<const char *>(a);
    const char *pb = reinterpret_cast<const char *>(b);
    const size_t bytes = static_cast<size_t>(n) * sizeof(float);
    return !(pa < pb + bytes && pb < pa + bytes);
}

constexpr double kFwhmPerSigma = 2.3548200450309493;  // 2 sqrt(2 ln 2)

// R = Rz(az) Ry(ay) Rx(ax), angles in degrees, row-major.
void euler_rotation(const float *deg, double R[3][3])
{
    const double d2r = 3.14159265358979323846 / 180.0;
    const double ax = deg[0] * d2r, ay = deg[1] * d2r, az = deg[2] * d2r;
    const double cx = std::cos(ax), sx = std::sin(ax), cy = std::cos(ay), sy = std::sin(ay);
    const double cz = std::cos(az), sz = std::sin(az);
    const double Rx[3][3] = {{1, 0, 0}, {0, cx, -sx}, {0, sx, cx}};
    const double Ry[3][3] = {{cy, 0, sy}, {0, 1, 0}, {-sy, 0, cy}};
    const double Rz[3][3] = {{cz, -sz, 0}, {sz, cz, 0}, {0, 0, 1}};
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T[i][j] = 0.0;
            for (int k = 0; k < 3; ++k)
                T[i][j] += Ry[i][k] * Rx[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            R[i][j] = 0.0;
            for (int k = 0; k < 3; ++k)
                R[i][j] += Rz[i][k] * T[k][j];
        }
}
}  // namespace

namespace {
// The separable smoothing pass: TMA-streamed when the rows are a multiple of
// 16 bytes and both cubes 16-byte aligned, else the plain-load kernel (both
// give the same floats).
afd_status smooth_separable(afd_ctx *ctx, const float *in, float *out, int nx, int ny, int nz,
                            const afd::SepWeights &w)
{
    cudaError_t e;
    if (stream_kernel_fits(in, out, nx)) {
        int bw = 0, bh = 0, hx = 0;
        afd::smooth_tma_box(w.rx, w.ry, &bw, &bh, &hx);
        CUtensorMap map;
        afd_status st = encode_box_map(ctx, &map, in, afd::STORE_F32, bw, bh, nx, ny, nz);
        if (st != AFD_OK)
            return st;
        e = afd::launch_smooth_sep_tma(map, out, nx, ny, nz, w, hx, ctx->d_err, ctx->stream);
    } else {
        e = afd::launch_smooth_sep(in, out, nx, ny, nz, w, ctx->d_err, ctx->stream);
    }
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}
}  // namespace

afd_status afd_smooth_box(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const int *N)
{
    const afd_host::TraceRange trace_("afd_smooth_box");
    if (!ctx || !in || !out || !N || !dims_ok(nx, ny, nz) || !cubes_disjoint(in, out, nx * ny * nz))
        return AFD_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (N[a] < 1 || N[a] % 2 == 0)
            return AFD_EINVAL;
    afd::SepWeights w;
    w.rx = N[0] / 2;
    w.ry = N[1] / 2;
    w.rz = N[2] / 2;
    if (w.rx > afd::kSepMaxR || w.ry > afd::kSepMaxR || w.rz > afd::kSepMaxRz)
        return AFD_EINVAL;
    for (int k = 0; k < 2 * afd::kSepMaxR + 1; ++k)
        w.wx[k] = w.wy[k] = 1.0f;
    for (int k = 0; k < 2 * afd::kSepMaxRz + 1; ++k)
        w.wz[k] = 1.0f;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    return smooth_separable(ctx, in, out, static_cast<int>(nx), static_cast<int>(ny),
                            static_cast<int>(nz), w);
}

afd_status afd_smooth_gauss(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                            int64_t nz, const float *fwhm, const float *angles_deg,
                            float truncate)
{
    const afd_host::TraceRange trace_("afd_smooth_gauss");
    if (!ctx || !in || !out || !fwhm || !dims_ok(nx, ny, nz) ||
        !cubes_disjoint(in, out, nx * ny * nz))
        return AFD_EINVAL;
    if (truncate == 0.0f)
        truncate = 3.0f;
    if (!(truncate > 0.0f) || !std::isfinite(truncate))
        return AFD_EINVAL;
    double sig[3];
    for (int a = 0; a < 3; ++a) {
        if (!(fwhm[a] > 0.0f) || !std::isfinite(fwhm[a]))
            return AFD_EINVAL;
        sig[a] = static_cast<double>(fwhm[a]) / kFwhmPerSigma;
    }
    bool rotated = false;
    if (angles_deg)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(angles_deg[a]))
                return AFD_EINVAL;
            rotated = rotated || angles_deg[a] != 0.0f;
        }
    const double t = static_cast<double>(truncate);
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const int inx = static_cast<int>(nx), iny = static_cast<int>(ny), inz = static_cast<int>(nz);
    cudaError_t e;
    if (!rotated) {
        afd::SepWeights w;
        int r[3];
        for (int a = 0; a < 3; ++a)
            r[a] = static_cast<int>(std::ceil(t * sig[a] - 1e-12));
        if (r[0] > afd::kSepMaxR || r[1] > afd::kSepMaxR || r[2] > afd::kSepMaxRz)
            return AFD_EINVAL;
        w.rx = r[0];
        w.ry = r[1];
        w.rz = r[2];
        float *dst[3] = {w.wx, w.wy, w.wz};
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k <= 2 * r[a]; ++k) {
                const double u = (k - r[a]) / sig[a];
                dst[a][k] = static_cast<float>(std::exp(-0.5 * u * u));
            }
        return smooth_separable(ctx, in, out, inx, iny, inz, w);
    } else {
        // K(p) = G(R^T p); extent of the ellipsoid along axis a:
        // sqrt(Sigma_aa), Sigma = R diag(sigma^2) R^T
        double R[3][3];
        euler_rotation(angles_deg, R);
        int r[3];
        for (int a = 0; a < 3; ++a) {
            double caa = 0.0;
            for (int b = 0; b < 3; ++b)
                caa += R[a][b] * R[a][b] * sig[b] * sig[b];
            r[a] = static_cast<int>(std::ceil(t * std::sqrt(caa) - 1e-12));
        }
        if (r[0] > 64 || r[1] > 64 || r[2] > 64 ||
            afd::smooth_direct_smem(r[0], r[1], r[2]) > 227 * 1024)
            return AFD_EINVAL;  // too large for the shared-memory ring
        const int WX = 2 * r[0] + 1, WY = 2 * r[1] + 1, WZ = 2 * r[2] + 1;
        std::vector<float> W(static_cast<size_t>(WX) * WY * WZ);
        double wsum = 0.0;
        for (int dz = -r[2]; dz <= r[2]; ++dz)
            for (int dy = -r[1]; dy <= r[1]; ++dy)
                for (int dx = -r[0]; dx <= r[0]; ++dx) {
                    const double p[3] = {static_cast<double>(dx), static_cast<double>(dy),
                                         static_cast<double>(dz)};
                    double q = 0.0;
                    for (int i = 0; i < 3; ++i) {
                        const double u = (R[0][i] * p[0] + R[1][i] * p[1] + R[2][i] * p[2]) /
                                         sig[i];  // (R^T p)_i / sigma_i
                        q += u * u;
                    }
                    const float wq = static_cast<float>(std::exp(-0.5 * q));
                    W[(dx + r[0]) + WX * ((dy + r[1]) + WY * (dz + r[2]))] = wq;
                    wsum += static_cast<double>(wq);
                }
        // FP64 prefix sums of W for the in-cube weight near a face
        const int SX1 = WX + 1, SY1 = WY + 1;
        std::vector<double> S(static_cast<size_t>(SX1) * SY1 * (WZ + 1), 0.0);
        for (int k = 1; k <= WZ; ++k)
            for (int j = 1; j < SY1; ++j)
                for (int i = 1; i < SX1; ++i) {
                    const size_t o = (static_cast<size_t>(k) * SY1 + j) * SX1 + i;
                    const size_t pz = static_cast<size_t>(SX1) * SY1;
                    S[o] = static_cast<double>(W[(i - 1) + WX * ((j - 1) + WY * (k - 1))]) +
                           S[o - 1] + S[o - SX1] + S[o - pz] - S[o - SX1 - 1] - S[o - pz - 1] -
                           S[o - pz - SX1] + S[o - pz - SX1 - 1];
                }
        const size_t w_bytes = (W.size() * sizeof(float) + 15) & ~size_t(15);
        const size_t s_bytes = S.size() * sizeof(double);
        st = ensure_buffer(ctx, &ctx->fd_buf, &ctx->fd_bytes,
                           std::max(ctx->fd_bytes, w_bytes + s_bytes));
        if (st != AFD_OK)
            return st;
        // the weights share the diagnostic's scratch: stream-ordered, copied
        // from host memory before the kernel that reads them
        char *dbuf = reinterpret_cast<char *>(ctx->fd_buf);
        e = cudaMemcpyAsync(dbuf, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dbuf + w_bytes, S.data(), s_bytes, cudaMemcpyHostToDevice,
                                ctx->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(ctx->stream);  // W and S are local buffers
        if (e == cudaSuccess)
            e = afd::launch_smooth_direct(in, out, inx, iny, inz,
                                          reinterpret_cast<const float *>(dbuf),
                                          reinterpret_cast<const double *>(dbuf + w_bytes), r[0],
                                          r[1], r[2], static_cast<float>(wsum), ctx->d_err,
                                          ctx->stream);
    }
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status afd_filter_intensity(afd_ctx *ctx, const float *in, float *out, int64_t nx,
                                int64_t ny, int64_t nz, const float *C, float K, float rms,
                                float tau, int n_iter)
{
    const afd_host::TraceRange trace_("afd_filter_intensity");
    if (!ctx || !in || !out || !dims_ok(nx, ny, nz) || !intensity_args_ok(C, K, rms, tau, n_iter))
        return AFD_EINVAL;
    if (in != out) {
        const size_t bytes = static_cast<size_t>(nx * ny * nz) * sizeof(float);
        const char *a = reinterpret_cast<const char *>(in);
        const char *b = reinterpret_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes)
            return AFD_EINVAL;
    }
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    if (n_iter == 0 || K == 0.0f || rms == 0.0f) {  // S = 0: identity
        cudaError_t e = cudaSuccess;
        if (in != out)
            e = cudaMemcpyAsync(out, in, static_cast<size_t>(nx * ny * nz) * sizeof(float),
                                cudaMemcpyDeviceToDevice, ctx->stream);
        return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
    }
    const afd::Coef k = afd::make_coef_intensity(C, K, rms, tau);
    return run_passes(ctx, in, out, nx, ny, nz, afd::COND_INT, k, n_iter);
}

namespace {

// Enqueue one host-to-host filter through staging slot `slot`: the H2D copy
// on the context's H2D stream, the passes on the context's stream, the D2H
// copy on its D2H stream, ordered by the slot's events.  A slot's input
// buffer is refilled only after the passes that read it are done, and its
// result buffer rewritten only after its copy to the host is done.
// The copy streams and a staging slot's events, created on first use; the
// slot's device buffer is two fixed halves (input, then output) of at least
// `bytes` each.  Fixed halves: a later use of the slot, whatever its size,
// writes only the input half, which never overlaps the output half that an
// earlier use's copy back may still be reading.
afd_status ensure_host_slot(afd_ctx *ctx, int slot, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);  // the output half stays 256-byte aligned
    cudaError_t e = cudaSuccess;
    if (!ctx->h2d_stream)
        e = cudaStreamCreateWithFlags(&ctx->h2d_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->d2h_stream)
        e = cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking);
    afd_ctx::HostSlot &s = ctx->host_slot[slot];
    if (e == cudaSuccess && !s.copied_in) {
        e = cudaEventCreateWithFlags(&s.copied_in, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s.filtered, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s.copied_out, cudaEventDisableTiming);
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    if (s.bytes < 2 * bytes) {
        // the slot's old buffer may still be in use: let all its work finish
        e = cudaEventSynchronize(s.copied_out);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(s.filtered);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (s.buf)
            cudaFree(s.buf);
        s.buf = nullptr;
        s.bytes = 0;
        void *p = nullptr;
        afd_status st = device_alloc(ctx, &p, 2 * bytes);
        if (st != AFD_OK)
            return st;
        s.buf = static_cast<float *>(p);
        s.bytes = 2 * bytes;
    }
    return AFD_OK;
}

// One cube (or z-slab) through staging slot `slot`: host_in -> device ->
// n_iter iterations -> planes [oz0, oz1) of the result -> host_out (which
// points at the destination of plane oz0).  Stream-ordered: the copies run on
// the copy streams and overlap the other slot's work.
afd_status enqueue_host_filter(afd_ctx *ctx, int slot, const float *host_in, float *host_out,
                               int64_t nx, int64_t ny, int64_t nz, const DeviceFilter &f,
                               int n_iter, int64_t oz0, int64_t oz1)
{
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * sizeof(float);
    afd_status st0 = ensure_host_slot(ctx, slot, bytes);
    if (st0 != AFD_OK)
        return st0;
    afd_ctx::HostSlot &s = ctx->host_slot[slot];
    cudaError_t e = cudaSuccess;
    float *d_in = s.buf;
    float *d_out = s.buf + s.bytes / 2 / sizeof(float);  // the output half
    // (waiting on an event that was never recorded returns at once)
    e = cudaStreamWaitEvent(ctx->h2d_stream, s.filtered, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_in, host_in, bytes, cudaMemcpyHostToDevice, ctx->h2d_stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(s.copied_in, ctx->h2d_stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->stream, s.copied_in, 0);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->stream, s.copied_out, 0);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    afd_status st = filter_device(ctx, d_in, d_out, nx, ny, nz, f, n_iter);
    if (st != AFD_OK)
        return st;
    e = cudaEventRecord(s.filtered, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->d2h_stream, s.filtered, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, d_out + oz0 * nx * ny,
                            static_cast<size_t>((oz1 - oz0) * nx * ny) * sizeof(float),
                            cudaMemcpyDeviceToHost, ctx->d2h_stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(s.copied_out, ctx->d2h_stream);
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

bool host_args_ok(afd_ctx *ctx, const float *host_in, float *host_out, int64_t nx, int64_t ny,
                  int64_t nz, const float *spacing, float K, float dt, int n_iter,
                  afd_conductance cond)
{
    return ctx && host_in && host_out && dims_ok(nx, ny, nz) &&
           params_ok(spacing, K, dt, n_iter, cond);
}

}  // namespace

afd_status afd_filter_host(afd_ctx *ctx, const float *host_in, float *host_out, int64_t nx,
                           int64_t ny, int64_t nz, const float *spacing, float K, float dt,
                           int n_iter, afd_conductance cond)
{
    const afd_host::TraceRange trace_("afd_filter_host");
    if (!host_args_ok(ctx, host_in, host_out, nx, ny, nz, spacing, K, dt, n_iter, cond))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    st = enqueue_host_filter(ctx, 0, host_in, host_out, nx, ny, nz,
                             per_face_filter(spacing, K, dt, cond), n_iter, 0, nz);
    if (st != AFD_OK)
        return st;
    return afd_sync(ctx);
}

afd_status afd_filter_host_async(afd_ctx *ctx, const float *host_in, float *host_out, int64_t nx,
                                 int64_t ny, int64_t nz, const float *spacing, float K, float dt,
                                 int n_iter, afd_conductance cond)
{
    const afd_host::TraceRange trace_("afd_filter_host_async");
    if (!host_args_ok(ctx, host_in, host_out, nx, ny, nz, spacing, K, dt, n_iter, cond))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const int slot = static_cast<int>(ctx->host_calls & 1ull);
    st = enqueue_host_filter(ctx, slot, host_in, host_out, nx, ny, nz,
                             per_face_filter(spacing, K, dt, cond), n_iter, 0, nz);
    if (st == AFD_OK)
        ctx->host_calls++;
    return st;
}

namespace {
// The z-slab rounds of afd_filter_slabs and afd_filter_intensity_slabs, for
// any filter whose iteration reaches one plane (arguments checked by the
// callers).
afd_status run_slabs(afd_ctx *ctx, const float *host_in, float *host_out, float *host_tmp,
                     int64_t nx, int64_t ny, int64_t nz, const DeviceFilter &f, int n_iter,
                     int64_t slab_nz, int halo)
{
    const int rounds = n_iter == 0 ? 1 : (n_iter + halo - 1) / halo;
    if (rounds > 1 && (!host_tmp || host_tmp == host_in || host_tmp == host_out))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const int64_t plane = nx * ny;
    // both slots and the pass scratch at the largest slab (slab_nz + 2 halo
    // planes), so that nothing is reallocated between slabs
    const int64_t max_nz = std::min<int64_t>(nz, slab_nz + 2 * static_cast<int64_t>(halo));
    const size_t max_bytes = static_cast<size_t>(max_nz * plane) * sizeof(float);
    for (int slot = 0; slot < 2 && st == AFD_OK; ++slot)
        st = ensure_host_slot(ctx, slot, max_bytes);
    if (st == AFD_OK)
        st = ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, max_bytes);
    if (st != AFD_OK)
        return st;
    cudaEvent_t round_done = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&round_done, cudaEventDisableTiming);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    const float *src = host_in;
    int k = 0;  // slabs enqueued: they alternate between the two slots
    for (int r = 0; r < rounds && st == AFD_OK; ++r) {
        const int its = std::min(halo, n_iter - r * halo);  // iterations this round (>= 0)
        // the last round writes host_out; the rounds before alternate
        float *dst = ((rounds - 1 - r) % 2 == 0) ? host_out : host_tmp;
        for (int64_t z0 = 0; z0 < nz && st == AFD_OK; z0 += slab_nz, ++k) {
            const int64_t z1 = std::min(nz, z0 + slab_nz);
            // a voxel moves `its` planes in `its` iterations: planes [z0, z1)
            // of the slab grown by `its` (clamped to the cube, whose faces
            // are the true zero-flux faces) are the whole cube's
            const int64_t lo = std::max<int64_t>(0, z0 - its), hi = std::min(nz, z1 + its);
            st = enqueue_host_filter(ctx, k & 1, src + lo * plane, dst + z0 * plane, nx, ny,
                                     hi - lo, f, its, z0 - lo, z1 - lo);
        }
        // the next round reads what this round wrote: its copies in wait for
        // every copy out of this one (in order on the copy-out stream)
        if (st == AFD_OK) {
            e = cudaEventRecord(round_done, ctx->d2h_stream);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(ctx->h2d_stream, round_done, 0);
            if (e != cudaSuccess)
                st = cuda_fail(ctx, e);
        }
        src = dst;
    }
    if (st == AFD_OK)
        st = afd_sync(ctx);
    cudaEventDestroy(round_done);
    return st;
}
}  // namespace

afd_status afd_filter_slabs(afd_ctx *ctx, const float *host_in, float *host_out, float *host_tmp,
                            int64_t nx, int64_t ny, int64_t nz, const float *spacing, float K,
                            float dt, int n_iter, afd_conductance cond, int64_t slab_nz, int halo)
{
    const afd_host::TraceRange trace_("afd_filter_slabs");
    if (!host_args_ok(ctx, host_in, host_out, nx, ny, nz, spacing, K, dt, n_iter, cond) ||
        slab_nz < 1 || halo < 1 || host_out == host_in)
        return AFD_EINVAL;
    return run_slabs(ctx, host_in, host_out, host_tmp, nx, ny, nz,
                     per_face_filter(spacing, K, dt, cond), n_iter, slab_nz, halo);
}

afd_status afd_filter_intensity_slabs(afd_ctx *ctx, const float *host_in, float *host_out,
                                      float *host_tmp, int64_t nx, int64_t ny, int64_t nz,
                                      const float *C, float K, float rms, float tau, int n_iter,
                                      int64_t slab_nz, int halo)
{
    const afd_host::TraceRange trace_("afd_filter_intensity_slabs");
    if (!ctx || !host_in || !host_out || !dims_ok(nx, ny, nz) ||
        !intensity_args_ok(C, K, rms, tau, n_iter) || slab_nz < 1 || halo < 1 ||
        host_out == host_in)
        return AFD_EINVAL;
    return run_slabs(ctx, host_in, host_out, host_tmp, nx, ny, nz,
                     intensity_filter(C, K, rms, tau), n_iter, slab_nz, halo);
}

afd_status afd_quantize(afd_ctx *ctx, const float *in, void *out, int64_t n, afd_storage storage,
                        float scale)
{
    const afd_host::TraceRange trace_("afd_quantize");
    if (!ctx || !in || !out || n < 1 || !storage_ok(storage) || storage == AFD_F32 ||
        !pow2_scale_ok(scale))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const float units = static_cast<float>(afd::store_units_per_value(storage, scale));
    cudaError_t e = afd::launch_quantize(storage, in, out, n, units, ctx->stream);
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status afd_dequantize(afd_ctx *ctx, const void *in, float *out, int64_t n,
                          afd_storage storage, float scale)
{
    const afd_host::TraceRange trace_("afd_dequantize");
    if (!ctx || !in || !out || n < 1 || !storage_ok(storage) || storage == AFD_F32 ||
        !pow2_scale_ok(scale))
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    const float units = static_cast<float>(afd::store_units_per_value(storage, scale));
    cudaError_t e = afd::launch_dequantize(storage, in, out, n, units, ctx->stream);
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

namespace {
// One afd_filter_ex call's launches: programmatic dependent launches chain
// the streaming kernels, and the tile counter is reset once per call.
struct ExLaunch {
    afd_ctx *ctx;
    int kind;
    afd::Coef k;
    int nx, ny, nz;
    bool prev_stream = false;  // the previous launch was a streaming-kernel launch
    bool tiles_zeroed = false;
};

// Plan bookkeeping shared by the streaming launches: PDL after a streaming
// launch, the tile counter's reset, and its base for the next launch.
cudaError_t ex_stream_begin(ExLaunch &L, afd::StreamPlan &plan)
{
    plan.pdl = L.prev_stream;
    L.prev_stream = true;
    cudaError_t e = cudaSuccess;
    if (!L.tiles_zeroed) {
        e = tiles_reset(L.ctx);
        L.tiles_zeroed = true;
    }
    return e;
}

afd_status ex_stream_end(ExLaunch &L, const afd::StreamPlan &plan, cudaError_t e)
{
    L.ctx->tiles_base += static_cast<unsigned long long>(plan.ntiles);
    L.ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(L.ctx, e);
}

// One iteration on the 8 x 2-voxel kernel, format s_in to s_out (equal, or
// one of them float32: the ends of a chain).
afd_status ex_wide(ExLaunch &L, int s_in, int s_out, const void *src, void *dst)
{
    afd_ctx *ctx = L.ctx;
    if (ctx->wide_bps == 0) {
        cudaError_t e = afd::pm_wide_prepare();
        if (e == cudaSuccess)
            e = afd::pm_wide_occupancy(&ctx->wide_bps);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (ctx->wide_bps < 1)
            ctx->wide_bps = 1;
    }
    int bw = 0, bh = 0;
    afd::pm_wide_box(s_in, &bw, &bh);
    CUtensorMap map;
    const afd_status st = encode_box_map(ctx, &map, src, s_in, bw, bh, L.nx, L.ny, L.nz);
    if (st != AFD_OK)
        return st;
    afd::StreamPlan plan = afd::pm_stream_plan(L.nx, L.ny, L.nz, ctx->sm_count, ctx->wide_bps,
                                               ctx->zc_hint, afd::kWideTX, afd::kWideTY);
    cudaError_t e = ex_stream_begin(L, plan);
    if (e == cudaSuccess)
        e = s_in == s_out
                ? afd::launch_pm_wide(s_in, L.kind, map, dst, L.nx, L.ny, L.nz, L.k, plan,
                                      ctx->d_tiles, ctx->tiles_base, ctx->d_err, ctx->stream)
                : afd::launch_pm_wide_chain_end(s_in, s_out, L.kind, map, dst, L.nx, L.ny, L.nz,
                                                L.k, plan, ctx->d_tiles, ctx->tiles_base,
                                                ctx->d_err, ctx->stream);
    return ex_stream_end(L, plan, e);
}

// One iteration on the barrier-free 4 x 2-voxel streaming kernel, on the
// stored format.
afd_status ex_stream(ExLaunch &L, int S, const void *src, void *dst)
{
    afd_ctx *ctx = L.ctx;
    if (ctx->stream_bps == 0) {
        cudaError_t e = afd::pm_stream_prepare();
        if (e == cudaSuccess)
            e = afd::pm_stream_occupancy(&ctx->stream_bps);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (ctx->stream_bps < 1)
            ctx->stream_bps = 1;
    }
    int bw = 0, bh = 0, hx = 0;
    afd::pm_stream_box(S, &bw, &bh, &hx);
    CUtensorMap map;
    const afd_status st = encode_box_map(ctx, &map, src, S, bw, bh, L.nx, L.ny, L.nz);
    if (st != AFD_OK)
        return st;
    afd::StreamPlan plan = afd::pm_stream_plan(L.nx, L.ny, L.nz, ctx->sm_count, ctx->stream_bps,
                                               ctx->zc_hint);
    cudaError_t e = ex_stream_begin(L, plan);
    if (e == cudaSuccess)
        e = afd::launch_pm_stream_s(S, L.kind, map, dst, L.nx, L.ny, L.nz, L.k, plan,
                                    ctx->d_tiles, ctx->tiles_base, ctx->d_err, ctx->stream);
    return ex_stream_end(L, plan, e);
}

// Two iterations on the two-stage kernel, format s_in to s_out.
afd_status ex_wide2(ExLaunch &L, int s_in, int s_out, const void *src, void *dst)
{
    afd_ctx *ctx = L.ctx;
    if (ctx->wide2_bps == 0) {
        cudaError_t e = afd::pm_wide2_prepare();
        if (e == cudaSuccess)
            e = afd::pm_wide2_occupancy(&ctx->wide2_bps);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        if (ctx->wide2_bps < 1)
            ctx->wide2_bps = 1;
    }
    int bw = 0, bh = 0;
    afd::pm_wide2_box(&bw, &bh);
    CUtensorMap map;
    const afd_status st = encode_box_map(ctx, &map, src, s_in, bw, bh, L.nx, L.ny, L.nz);
    if (st != AFD_OK)
        return st;
    afd::StreamPlan plan = afd::pm_stream_plan(L.nx, L.ny, L.nz, ctx->sm_count, ctx->wide2_bps,
                                               ctx->zc_hint, afd::kWide2TX, afd::kWide2TY);
    cudaError_t e = ex_stream_begin(L, plan);
    if (e == cudaSuccess)
        e = afd::launch_pm_wide2(s_in, s_out, L.kind, map, dst, L.nx, L.ny, L.nz, L.k, plan,
                                 ctx->d_tiles, ctx->tiles_base, ctx->d_err, ctx->stream);
    return ex_stream_end(L, plan, e);
}

// A pass of depth T >= 2 as a chain through two float32 context cubes,
// storage -> float32 -> ... -> float32 -> storage: dequantise, T float32
// iterations, quantise, the result of one blocked pass of depth T.  Links
// of one iteration (the ends on the 8 x 2-voxel kernel, float32 -> float32
// on the streaming kernel), or of two on the two-stage kernel (two_stage).
afd_status ex_chain(ExLaunch &L, int S, int T, bool two_stage, int64_t n, const void *src,
                    void *dst)
{
    afd_ctx *ctx = L.ctx;
    afd_status st = ensure_buffer(ctx, &ctx->chain_f32, &ctx->chain_f32_bytes,
                                  2 * static_cast<size_t>(n) * sizeof(float));
    if (st != AFD_OK)
        return st;
    float *link_buf[2] = {ctx->chain_f32, ctx->chain_f32 + n};
    const int links = two_stage ? T / 2 : T;
    for (int l = 0; l < links && st == AFD_OK; ++l) {
        const int s_in = l == 0 ? S : afd::STORE_F32;
        const int s_out = l == links - 1 ? S : afd::STORE_F32;
        const void *lsrc = l == 0 ? src : link_buf[(l - 1) & 1];
        void *ldst = l == links - 1 ? dst : link_buf[l & 1];
        if (two_stage)
            st = ex_wide2(L, s_in, s_out, lsrc, ldst);
        else if (s_in == afd::STORE_F32 && s_out == afd::STORE_F32)
            st = ex_stream(L, afd::STORE_F32, lsrc, ldst);
        else
            st = ex_wide(L, s_in, s_out, lsrc, ldst);
    }
    return st;
}

// One pass of depth T on the general temporally blocked kernel.
afd_status ex_blocked(ExLaunch &L, int S, int T, const void *src, void *dst)
{
    afd_ctx *ctx = L.ctx;
    if (!ctx->tb_ready[S][T]) {
        const cudaError_t e = afd::tb_prepare(S, T);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
        ctx->tb_ready[S][T] = true;
    }
    CUtensorMap map;
    const afd_status st = encode_tb_map(ctx, &map, src, S, T, L.nx, L.ny, L.nz);
    if (st != AFD_OK)
        return st;
    const afd::TbPlan plan = afd::tb_plan(S, T, L.nx, L.ny, L.nz, ctx->sm_count, ctx->zc_hint);
    const cudaError_t e = afd::tb_launch(S, T, L.kind, map, dst, L.nx, L.ny, L.nz, L.k, plan,
                                         ctx->d_err, ctx->stream);
    L.prev_stream = false;
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}
}  // namespace

afd_status afd_filter_ex(afd_ctx *ctx, const void *in, void *out, afd_storage storage,
                         float scale, int64_t nx, int64_t ny, int64_t nz, const float *spacing,
                         float K, float dt, int n_iter, afd_conductance cond, int t_block)
{
    const afd_host::TraceRange trace_("afd_filter_ex");
    if (!ctx || !in || !out || !storage_ok(storage) || !dims_ok(nx, ny, nz) ||
        !params_ok(spacing, K, dt, n_iter, cond))
        return AFD_EINVAL;
    if (storage == AFD_F32)
        scale = 1.0f;
    if (!pow2_scale_ok(scale))
        return AFD_EINVAL;
    if (t_block == 0)
        t_block = 1;  // the streaming pass: faster on GB300 than any blocked depth
    if (!afd::tb_depth_ok(t_block))
        return AFD_EINVAL;
    const int S = storage;
    const int64_t n = nx * ny * nz;
    const size_t bytes = static_cast<size_t>(n) * static_cast<size_t>(afd::store_bytes(S));
    if (in != out) {
        const char *a = static_cast<const char *>(in);
        const char *b = static_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes)
            return AFD_EINVAL;
    }
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    cudaError_t e = cudaSuccess;
    if (n_iter == 0 || K == 0.0f) {  // identity
        if (in != out)
            e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
    }
    st = ensure_buffer(ctx, &ctx->lp_scratch, &ctx->lp_scratch_bytes, bytes);
    if (st != AFD_OK)
        return st;
    void *scr = ctx->lp_scratch;
    const double units_d = afd::store_units_per_value(S, scale);
    const float units = static_cast<float>(units_d);
    // K in storage units (exact: units is a power of two)
    const float Ks = std::isinf(K) ? K : static_cast<float>(static_cast<double>(K) * units_d);
    int kind = 0;
    const afd::Coef k = afd::make_coef(spacing, Ks, dt, cond == AFD_COND_EXPONENTIAL, &kind);

    // passes: n_iter / t_block of depth t_block, then the remainder as
    // passes of depth 4, 2 and 1 (each at most t_block)
    int npass = 0;
    {
        int left = n_iter, m = 0;
        while (left >= t_block) {
            ++m;
            left -= t_block;
        }
        for (int d = 4; d >= 1; d >>= 1)
            while (d <= t_block && left >= d) {
                ++m;
                left -= d;
            }
        npass = m;
    }
    auto depth_of = [&](int i) -> int {
        const int full = n_iter / t_block;
        if (i < full)
            return t_block;
        int left = n_iter - full * t_block, j = full;
        for (int d = 4; d >= 1; d >>= 1)
            while (d <= t_block && left >= d) {
                if (j == i)
                    return d;
                ++j;
                left -= d;
            }
        return 1;
    };
    const bool inplace = (in == out);
    auto dst_of = [&](int i) -> void * {
        if (inplace)
            return (i & 1) ? out : scr;
        return ((npass - 1 - i) & 1) ? scr : out;
    };
    auto src_of = [&](int i) -> const void * { return i == 0 ? in : dst_of(i - 1); };

    const int es = afd::store_bytes(S);
    const bool fits = ((nx * es) % 16 == 0) && (reinterpret_cast<uintptr_t>(in) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && !std::isinf(K) &&
                      (reinterpret_cast<uintptr_t>(scr) & 15u) == 0;
    ExLaunch L{ctx, kind, k, static_cast<int>(nx), static_cast<int>(ny), static_cast<int>(nz)};
    // deep passes on the fast routes: exponential or rational g, nx a multiple of 8
    const bool deep_ok = fits && nx % 8 == 0 && (kind == afd::COND_EXP || kind == afd::COND_RAT);
    for (int i = 0; i < npass; ++i) {
        const afd_host::TraceRange pass_trace("pass");
        const int T = depth_of(i);
        if (fits && T == 1 && S != afd::STORE_F32 && ctx->kernel != AFD_KERNEL_STREAM) {
            st = ex_wide(L, S, S, src_of(i), dst_of(i));   // the 8 x 2-voxel kernel
        } else if (fits && T == 1) {
            st = ex_stream(L, S, src_of(i), dst_of(i));    // the 4 x 2-voxel kernel
        } else if (deep_ok && T >= 2 && ctx->kernel != AFD_KERNEL_STREAM) {
            st = ex_chain(L, S, T, ctx->kernel == AFD_KERNEL_TWO_STAGE, n, src_of(i), dst_of(i));
        } else if (fits) {
            st = ex_blocked(L, S, T, src_of(i), dst_of(i));
        } else {
            st = fallback_pass(ctx, S, units, src_of(i), dst_of(i), nx, ny, nz, spacing, K, dt, T,
                               cond);
            L.prev_stream = false;
        }
        if (st != AFD_OK)
            return st;
    }
    if (dst_of(npass - 1) != out) {
        e = cudaMemcpyAsync(out, dst_of(npass - 1), bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e);
    }
    return AFD_OK;
}

afd_status afd_stats(afd_ctx *ctx, const float *cube, int64_t n, double *out4)
{
    const afd_host::TraceRange trace_("afd_stats");
    if (!ctx || !cube || !out4 || n < 1)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    return stats_device(ctx, cube, n, out4);
}

afd_status afd_noise_rms(afd_ctx *ctx, const float *cube, int64_t n, double *out)
{
    const afd_host::TraceRange trace_("afd_noise_rms");
    if (!ctx || !cube || !out || n < 1)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st == AFD_OK)
        st = stats_host(ctx, cube, n);
    if (st != AFD_OK)
        return st;
    const double nneg = ctx->h_out4[3];
    *out = nneg > 0.0 ? std::sqrt(ctx->h_out4[2] / nneg) : 0.0;
    return AFD_OK;
}

afd_status afd_sum(afd_ctx *ctx, const float *cube, int64_t n, double *out)
{
    const afd_host::TraceRange trace_("afd_sum");
    if (!ctx || !cube || !out || n < 1)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st == AFD_OK)
        st = stats_host(ctx, cube, n);
    if (st != AFD_OK)
        return st;
    *out = ctx->h_out4[0];
    return AFD_OK;
}

afd_status afd_sync(afd_ctx *ctx)
{
    if (!ctx)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && ctx->h2d_stream)
        e = cudaStreamSynchronize(ctx->h2d_stream);
    if (e == cudaSuccess && ctx->d2h_stream)
        e = cudaStreamSynchronize(ctx->d2h_stream);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    int code = 0;
    e = cudaMemcpy(&code, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    if (code != 0) {
        std::snprintf(ctx->errstr, sizeof(ctx->errstr), "bounded wait expired in a kernel (code %d)",
                      code);
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return AFD_ETIMEOUT;
    }
    return AFD_OK;
}

afd_status afd_check_violations(afd_ctx *ctx, int *count, int *code, int *index)
{
    if (!ctx || !count || !code || !index)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    int rec[3] = {0, 0, 0};
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(rec, ctx->d_err + afd::kCheckCount, sizeof(rec), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->d_err + afd::kCheckCount, 0, sizeof(rec));
    if (e != cudaSuccess)
        return cuda_fail(ctx, e);
    *count = rec[0];
    *code = rec[1];
    *index = rec[2];
    return AFD_OK;
}

int afd_checked_build(void) { return afd::kChecked ? 1 : 0; }

afd_status afd_pass_timing(afd_ctx *ctx, int on)
{
    if (!ctx)
        return AFD_EINVAL;
    ctx->timing = on != 0;
    return AFD_OK;
}

afd_status afd_pass_timing_read(afd_ctx *ctx, double *ms, int64_t *passes)
{
    if (!ctx || !ms || !passes)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    double total = 0.0;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i + 1 < ctx->tev.size(); i += 2) {
        float t = 0.0f;
        if (e == cudaSuccess)
            e = cudaEventSynchronize(ctx->tev[i + 1]);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&t, ctx->tev[i], ctx->tev[i + 1]);
        total += static_cast<double>(t);
    }
    for (cudaEvent_t ev : ctx->tev)
        cudaEventDestroy(ev);
    ctx->tev.clear();
    *ms = total;
    *passes = ctx->timed_passes;
    ctx->timed_passes = 0;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status afd_selftest_wait(afd_ctx *ctx, int64_t limit_ns)
{
    if (!ctx)
        return AFD_EINVAL;
    afd_status st = set_device(ctx);
    if (st != AFD_OK)
        return st;
    if (limit_ns < 1000)
        limit_ns = 1000;
    if (limit_ns > 5000000000ll)
        limit_ns = 5000000000ll;
    cudaError_t e =
        afd::launch_selftest_wait(static_cast<uint64_t>(limit_ns), ctx->d_err, ctx->stream);
    ctx->launches++;
    return e == cudaSuccess ? AFD_OK : cuda_fail(ctx, e);
}

afd_status afd_launch_count(afd_ctx *ctx, uint64_t *out)
{
    if (!ctx || !out)
        return AFD_EINVAL;
    *out = ctx->launches;
    return AFD_OK;
}

const char *afd_status_str(afd_status s)
{
    switch (s) {
    case AFD_OK:
        return "AFD_OK";
    case AFD_EINVAL:
        return "AFD_EINVAL: invalid argument";
    case AFD_ENOMEM:
        return "AFD_ENOMEM: out of device memory";
    case AFD_ECUDA:
        return "AFD_ECUDA: CUDA error";
    case AFD_ETIMEOUT:
        return "AFD_ETIMEOUT: a kernel's bounded wait expired";
    case AFD_EBUSY:
        return "AFD_EBUSY: resource busy";
    }
    return "unknown afd_status";
}

const char *afd_last_error_string(afd_ctx *ctx)
{
    return ctx ? ctx->errstr : "";
}

}  // extern "C"
