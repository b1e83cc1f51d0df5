// Storage conversion kernels: float32 <-> 2-byte cube (precision line, a2 and
// a7).  q = RN_format(v * units) and v = load(q) / units, units a power of two
// (storage units per value unit), so scaling is exact and the only rounding is
// the one into the 2-byte format (nearest, ties to even; int16 clamps to
// +-32767).  HBM-bound elementwise passes: 4 values per thread per step.
#include "afd_internal.h"
#include "afd_store.cuh"

namespace afd {
namespace {

template <int S>
__global__ void __launch_bounds__(256)
    quantize_kernel(const float *__restrict__ in, typename Store<S>::T *__restrict__ out,
                    int64_t n, float units, int vec)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (!vec) {  // input not 16-byte aligned
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
             i += stride)
            out[i] = Store<S>::store(__fmul_rn(in[i], units));
        return;
    }
    const int64_t n4 = n / 4;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4;
         i += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(in) + i);
        typename Store<S>::T q[4] = {Store<S>::store(__fmul_rn(v.x, units)),
                                     Store<S>::store(__fmul_rn(v.y, units)),
                                     Store<S>::store(__fmul_rn(v.z, units)),
                                     Store<S>::store(__fmul_rn(v.w, units))};
        for (int j = 0; j < 4; ++j)
            out[4 * i + j] = q[j];
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        const int64_t i = n4 * 4 + threadIdx.x;
        if (i < n)
            out[i] = Store<S>::store(__fmul_rn(in[i], units));
    }
}

template <int S>
__global__ void __launch_bounds__(256)
    dequantize_kernel(const typename Store<S>::T *__restrict__ in, float *__restrict__ out,
                      int64_t n, float inv_units)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride)
        out[i] = __fmul_rn(Store<S>::load(in[i]), inv_units);
}

int grid_for(int64_t n)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n / 4 + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    return static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_quantize(int S, const float *in, void *out, int64_t n, float units,
                            cudaStream_t stream)
{
    const int grid = grid_for(n);
    const int vec = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
    switch (S) {
    case STORE_F16:
        quantize_kernel<STORE_F16><<<grid, 256, 0, stream>>>(
            in, static_cast<unsigned short *>(out), n, units, vec);
        break;
    case STORE_BF16:
        quantize_kernel<STORE_BF16><<<grid, 256, 0, stream>>>(
            in, static_cast<unsigned short *>(out), n, units, vec);
        break;
    case STORE_I16:
        quantize_kernel<STORE_I16><<<grid, 256, 0, stream>>>(in, static_cast<short *>(out), n,
                                                             units, vec);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dequantize(int S, const void *in, float *out, int64_t n, float units,
                              cudaStream_t stream)
{
    const int grid = grid_for(n);
    const float inv = 1.0f / units;  // exact: units is a power of two
    switch (S) {
    case STORE_F16:
        dequantize_kernel<STORE_F16><<<grid, 256, 0, stream>>>(
            static_cast<const unsigned short *>(in), out, n, inv);
        break;
    case STORE_BF16:
        dequantize_kernel<STORE_BF16><<<grid, 256, 0, stream>>>(
            static_cast<const unsigned short *>(in), out, n, inv);
        break;
    case STORE_I16:
        dequantize_kernel<STORE_I16><<<grid, 256, 0, stream>>>(static_cast<const short *>(in),
                                                               out, n, inv);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace afd
