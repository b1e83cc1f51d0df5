// FP64 statistics of an FP32 cube: sum I, sum I^2, sum over I<0 of I^2 and
// the number of negative voxels.
//
// They give the noise level "rms" that K is expressed in (arXiv:1609.03782
// Sec. 3.3; read here as the rms of the negative voxels) and the conservation
// check of the per-face scheme (the voxel sum is invariant).
//
// Each thread reads 16 consecutive values (four 16-byte loads), sums them
// pairwise in float32 (error <= 4 ulp of the chunk's absolute sum) and adds
// the chunk sums to double accumulators: one FP64 add per 16 values keeps the
// kernel bound by HBM on GB300, whose FP64 rate is low.  Warps, blocks and the
// final pass combine in a fixed order, so results are bit-reproducible for a
// given grid size.
#include "afd_internal.h"

namespace afd {
namespace {

template <bool VEC>
__global__ void __launch_bounds__(kStatsThreads)
    stats_partial(const float *__restrict__ x, int64_t n, double *__restrict__ part)
{
    double s = 0.0, s2 = 0.0, ns2 = 0.0;
    long long cnt = 0;
    const int64_t nchunk = n / 16;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < nchunk;
         c += stride) {
        float a[16], b[16], d[16];
        if (VEC) {
            const float4 *p = reinterpret_cast<const float4 *>(x + c * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = __ldcs(p + i);
                a[4 * i + 0] = v.x;
                a[4 * i + 1] = v.y;
                a[4 * i + 2] = v.z;
                a[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                a[i] = x[c * 16 + i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            b[i] = __fmul_rn(a[i], a[i]);
            const bool neg = a[i] < 0.0f;
            d[i] = neg ? b[i] : 0.0f;
            cnt += neg ? 1 : 0;
        }
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1) {
#pragma unroll
            for (int i = 0; i < w; ++i) {
                a[i] = __fadd_rn(a[i], a[i + w]);
                b[i] = __fadd_rn(b[i], b[i + w]);
                d[i] = __fadd_rn(d[i], d[i + w]);
            }
        }
        s += static_cast<double>(a[0]);
        s2 += static_cast<double>(b[0]);
        ns2 += static_cast<double>(d[0]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int64_t i = nchunk * 16; i < n; ++i) {
            const double v = static_cast<double>(x[i]);
            s += v;
            s2 += v * v;
            if (v < 0.0) {
                ns2 += v * v;
                cnt += 1;
            }
        }
    }
    double c = static_cast<double>(cnt);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, off);
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
        ns2 += __shfl_down_sync(0xffffffffu, ns2, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
    }
    __shared__ double red[kStatsThreads / 32][4];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[warp][0] = s;
        red[warp][1] = s2;
        red[warp][2] = ns2;
        red[warp][3] = c;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < kStatsThreads / 32; ++w)
            acc += red[w][threadIdx.x];
        part[static_cast<int64_t>(blockIdx.x) * 4 + threadIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(kStatsThreads)
    stats_final(const double *__restrict__ part, int nblocks, double *__restrict__ out4)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int q = 0; q < 4; ++q)
            v[q] += part[static_cast<int64_t>(b) * 4 + q];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        for (int q = 0; q < 4; ++q)
            v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    __shared__ double red[kStatsThreads / 32][4];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q)
            red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < kStatsThreads / 32; ++w)
            acc += red[w][threadIdx.x];
        out4[threadIdx.x] = acc;
    }
}

}  // namespace

cudaError_t launch_stats(const float *x, int64_t n, double *partials, int nblocks, double *out4,
                         cudaStream_t stream)
{
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    if (vec)
        stats_partial<true><<<nblocks, kStatsThreads, 0, stream>>>(x, n, partials);
    else
        stats_partial<false><<<nblocks, kStatsThreads, 0, stream>>>(x, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    stats_final<<<1, kStatsThreads, 0, stream>>>(partials, nblocks, out4);
    return cudaGetLastError();
}

}  // namespace afd
