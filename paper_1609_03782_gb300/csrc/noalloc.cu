// afd_filter_noalloc: the filter for callers that cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// application's own memory budget with every device byte already pooled by
// that application, real-time loops where an allocation (and the device
// synchronisation it may cause) is not allowed, and plug-ins that are not
// given an allocator.  They cannot create an afd_ctx either, since a context
// owns device memory.  This entry point needs neither: its ping-pong scratch
// and its error word are file-scope __device__ arrays of a fixed size, and it
// calls no cudaMalloc, cudaFree or allocating library routine.  The caller
// still passes the input and output cubes.
//
// The arrays are part of this library's device image: a GPU holds them from
// the moment the image is loaded on it (at the first call of this entry point
// on that device, CUDA loading modules lazily by default) until the process
// exits.  In host code their names are host-side stand-ins, not device
// addresses, so the first call on each device, with that device current,
// looks up their device addresses with cudaGetSymbolAddress and keeps them.
//
// The filter itself is the same as afd_filter_out's: the same pass sequence
// (passes.cu), kernels and per-face arithmetic, so the results are
// bit-identical.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/afd.h"
#include "afd_internal.h"
#include "afd_trace.h"

namespace {

constexpr int64_t kMaxVoxels = AFD_NOALLOC_MAX_VOXELS;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps the last call's contents.
__device__ __align__(256) float g_noalloc_scratch[kMaxVoxels];
__device__ __align__(256) int g_noalloc_err[64];
__device__ __align__(8) unsigned long long g_noalloc_tiles[1];  // streaming kernel tile counter

struct DeviceSetup {
    bool ready = false;
    float *scratch = nullptr;  // device address of g_noalloc_scratch
    int *err = nullptr;        // device address of g_noalloc_err
    unsigned long long *tiles = nullptr;  // device address of g_noalloc_tiles
    int sm_count = 0;
    int stream_bps = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];
PFN_cuTensorMapEncodeTiled_v12000 g_encode_fn = nullptr;

// Once per device, with that device current: resolve the arrays' device
// addresses and the streaming kernel's occupancy.
afd_status setup_device(int dev, DeviceSetup *out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess)
            return AFD_ECUDA;
        s.scratch = static_cast<float *>(p);
        if (cudaGetSymbolAddress(&p, g_noalloc_err) != cudaSuccess)
            return AFD_ECUDA;
        s.err = static_cast<int *>(p);
        if (cudaGetSymbolAddress(&p, g_noalloc_tiles) != cudaSuccess)
            return AFD_ECUDA;
        s.tiles = static_cast<unsigned long long *>(p);
        if (cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess)
            return AFD_ECUDA;
        if (afd::pm_stream_prepare() != cudaSuccess ||
            afd::pm_stream_occupancy(&s.stream_bps) != cudaSuccess)
            return AFD_ECUDA;
        if (s.stream_bps < 1)
            s.stream_bps = 1;
        if (!g_encode_fn) {
            cudaDriverEntryPointQueryResult q;
            void *fn = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                 cudaEnableDefault, &q) == cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                g_encode_fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
        s.ready = true;
    }
    *out = s;
    return AFD_OK;
}

bool encode_map(CUtensorMap *map, const float *ptr, int nx, int ny, int nz)
{
    if (!g_encode_fn)
        return false;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                                static_cast<cuuint64_t>(nz)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(nx) * 4,
                                   static_cast<cuuint64_t>(nx) * static_cast<cuuint64_t>(ny) * 4};
    const cuuint32_t box[3] = {afd::kStreamTX + 8, afd::kStreamTY + 2, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return g_encode_fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" afd_status afd_filter_noalloc(const float *in, float *out, int64_t nx, int64_t ny,
                                         int64_t nz, const float *spacing, float K, float dt,
                                         int n_iter, afd_conductance cond, void *cuda_stream)
{
    const afd_host::TraceRange trace_("afd_filter_noalloc");
    // ---- arguments (the same rules as afd_filter_out) ----
    if (!in || !out || nx < 1 || ny < 1 || nz < 1)
        return AFD_EINVAL;
    if (nx > kMaxVoxels || ny > kMaxVoxels || nz > kMaxVoxels || nx * ny > kMaxVoxels ||
        nx * ny * nz > kMaxVoxels)
        return AFD_EINVAL;  // larger than the fixed scratch
    if (cond != AFD_COND_EXPONENTIAL && cond != AFD_COND_RATIONAL)
        return AFD_EINVAL;
    if (spacing)
        for (int a = 0; a < 3; ++a)
            if (!(spacing[a] > 0.0f) || !std::isfinite(spacing[a]))
                return AFD_EINVAL;
    if (std::isnan(K) || K < 0.0f || !(dt > 0.0f) || !std::isfinite(dt) || n_iter < 0)
        return AFD_EINVAL;
    const int64_t n = nx * ny * nz;
    const size_t bytes = static_cast<size_t>(n) * sizeof(float);
    if (in != out) {
        const char *a = reinterpret_cast<const char *>(in);
        const char *b = reinterpret_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes)
            return AFD_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return AFD_ECUDA;
    DeviceSetup s;
    afd_status st = setup_device(dev, &s);
    if (st != AFD_OK)
        return st;

    cudaError_t e = cudaSuccess;
    if (n_iter == 0 || K == 0.0f) {  // identity
        if (in != out)
            e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
        return e == cudaSuccess ? AFD_OK : AFD_ECUDA;
    }

    // ---- coefficients: those of afd_filter ----
    int kind = 0;
    const afd::Coef k = afd::make_coef(spacing, K, dt, cond == AFD_COND_EXPONENTIAL, &kind);

    // the error word must start at zero; the scratch is fully overwritten
    e = cudaMemsetAsync(s.err, 0, sizeof(int), stream);
    if (e != cudaSuccess)
        return AFD_ECUDA;

    // ---- passes: in -> ... -> out, alternating with the static scratch; the
    // same pass sequence as the context entry points (passes.cu) ----
    const int inx = static_cast<int>(nx), iny = static_cast<int>(ny), inz = static_cast<int>(nz);
    const afd::PassSeq q{kind, in, out, s.scratch, inx, iny, inz, k, n_iter, stream, nullptr};
    const bool use_stream = (nx % 4) == 0 && (reinterpret_cast<uintptr_t>(in) & 15u) == 0 &&
                            (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
    if (use_stream) {
        const float *bufs[3] = {in, out, s.scratch};
        CUtensorMap maps[3];
        for (int b = 0; b < 3; ++b)
            if (!encode_map(&maps[b], bufs[b], inx, iny, inz))
                return AFD_ECUDA;
        const afd::StreamPlan plan = afd::pm_stream_plan(inx, iny, inz, s.sm_count,
                                                         s.stream_bps, 0);
        e = cudaMemsetAsync(s.tiles, 0, sizeof(unsigned long long), stream);
        unsigned long long base = 0;
        if (e == cudaSuccess)
            e = afd::stream_passes(q, maps, plan, s.tiles, &base, s.err);
    } else {
        e = afd::simple_passes(q);
    }
    if (e == cudaSuccess)
        e = afd::passes_finish(q);

    // ---- synchronous: report a bounded-wait expiry of this call ----
    int code = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&code, s.err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return AFD_ECUDA;
    return code != 0 ? AFD_ETIMEOUT : AFD_OK;
}
