// FP64 statistics of an FP32 cube: sum I, sum I^2, sum over I<0 of I^2 and
// the number of negative voxels.
//
// They give the noise level "rms" that K is expressed in (arXiv:1609.03782
// Sec. 3.3; read here as the rms of the negative voxels) and the conservation
// check of the per-face scheme (the voxel sum is invariant).
//
// Each thread reads 16 consecutive values (four 16-byte loads), sums them
// pairwise in float32 (error <= 4 ulp of the chunk's absolute sum) and adds
// the chunk sums to float-float (TwoSum) accumulators, converted to double
// once per thread: no FP64 arithmetic in the loop, whose rate on GB300 is
// far too low for HBM speed.  Warps, blocks and the
// final pass combine in a fixed order, so results are bit-reproducible for a
// given grid size.
#include "afd_internal.h"

namespace afd {
namespace {

// A float32 pair (hi, lo) holding hi + lo: the running sum of a thread's
// chunk sums.  Each addition is Knuth's TwoSum, exact in (hi, lo) up to the
// rounding of lo, so the pair carries ~48 significant bits with float32
// arithmetic only (GB300's FP64 rate is too low for one double add per 16
// values to keep up with HBM).
struct FF {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(hi, x);
        const float bp = __fsub_rn(t, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        hi = t;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const
    {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

// One chunk of 16 values: pairwise float32 sums of I, I^2 and I^2 over I < 0,
// added to the thread's accumulators, and the count of negative values.
__device__ __forceinline__ void chunk_sums(float (&a)[16], FF &s, FF &s2, FF &ns2, int &cnt)
{
    float b[16], d[16];
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
    s.add(a[0]);
    s2.add(b[0]);
    ns2.add(d[0]);
}

template <bool VEC>
__device__ __forceinline__ void load_chunk(const float *__restrict__ x, int64_t c, float (&a)[16])
{
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
}

template <bool VEC>
__global__ void __launch_bounds__(kStatsThreads)
    stats_partial(const float *__restrict__ x, int64_t n, double *__restrict__ part)
{
    FF fs, fs2, fns2;
    int icnt = 0;  // a thread sees far fewer than 2^31 values
    const int64_t nchunk = n / 16;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    // a thread's chunks are c, c + stride, ...; two are loaded before either
    // is summed (eight 16-byte loads in flight), and they are summed in that
    // order
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < nchunk;
         c += 2 * stride) {
        float a0[16], a1[16];
        const bool two = c + stride < nchunk;
        load_chunk<VEC>(x, c, a0);
        if (two)
            load_chunk<VEC>(x, c + stride, a1);
        chunk_sums(a0, fs, fs2, fns2, icnt);
        if (two)
            chunk_sums(a1, fs, fs2, fns2, icnt);
    }
    double s = fs.value(), s2 = fs2.value(), ns2 = fns2.value();
    long long cnt = icnt;
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

namespace {
// One thread: rms of the negative voxels from the statistics (as
// afd_noise_rms computes it on the host), K = k_rms x rms rounded to float,
// and the coefficients for K (A on the device, B from the host).
__global__ void rel_coef_kernel(const double *__restrict__ out4, double k_rms, int kind, double dt,
                                double h0, double h1, double h2, float b0, float b1, float b2,
                                Coef *__restrict__ coef, float *__restrict__ K_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    const double nneg = out4[3];
    const double rms = nneg > 0.0 ? sqrt(out4[2] / nneg) : 0.0;
    const float K = static_cast<float>(k_rms * rms);
    const double Kd = static_cast<double>(K);
    Coef k;
    k.ax = static_cast<float>(coef_a_device(Kd, kind, dt, h0));
    k.ay = static_cast<float>(coef_a_device(Kd, kind, dt, h1));
    k.az = static_cast<float>(coef_a_device(Kd, kind, dt, h2));
    k.bx = b0;
    k.by = b1;
    k.bz = b2;
    if (K == 0.0f) {
        // no negative voxel (rms 0): zero conductance, every flux exactly 0
        // (rational: delta / (A delta^2 + inf); exponential: delta 2^(... - inf))
        const float b = kind == COND_EXP ? -INFINITY : INFINITY;
        k.bx = k.by = k.bz = b;
    }
    k.nz = -0.0f;
    k.ai = 0.0f;
    *coef = k;
    if (K_out)
        *K_out = K;
}
}  // namespace

cudaError_t launch_rel_coef(const double *out4, double k_rms, int kind, double dt, const double h[3],
                            const Coef &b, Coef *coef, float *K_out, cudaStream_t stream)
{
    rel_coef_kernel<<<1, 32, 0, stream>>>(out4, k_rms, kind, dt, h[0], h[1], h[2], b.bx, b.by,
                                          b.bz, coef, K_out);
    return cudaGetLastError();
}

}  // namespace afd
