// The smoothing-quality diagnostic of arXiv:1609.03782 Sec. 4 (eqs. "F_equa",
// "Sequa", "Mfequa") and the recovered-signal fraction of Sec. 5 (eq.
// "sums_equa"): masked sums over a ROI box of the original, filtered and
// (optionally) noiseless model cubes, in one pass.
//
//   S_of = sum I_o [I_f >= t_f]    S_oo = sum I_o [I_o >= t_o]
//   S_mf = sum I_m [I_f >= t_f]    S_m  = sum I_m
//   N_o  = sum [I_o >= t_o]        N_f  = sum [I_f >= t_f]
//
// The thresholds arrive as floats already rounded up from nsig x rms (the
// smallest float >= the exact threshold), so a float comparison takes the
// same mask decision as the exact one.  Each warp walks rows of the box
// (lanes along x, four elements per lane per step, all loads issued before
// they are used); a lane's four values are summed in float32 and the sums
// added to float-float (TwoSum) accumulators, converted to double once per
// thread.  Warps and blocks combine in double in a fixed order, so a result
// is reproducible for a given grid.  HBM-bound: 8 (12 with the model) bytes
// per ROI voxel.
#include "afd_internal.h"

namespace afd {
namespace {

constexpr int kFdThreads = 256;

struct FFsum {
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

template <bool MODEL>
__global__ void __launch_bounds__(kFdThreads)
    fdiag_partial(const float *__restrict__ io_, const float *__restrict__ if_,
                  const float *__restrict__ im_, int64_t nx, int64_t ny, int x0, int x1, int y0,
                  int y1, int z0, int z1, float t_o, float t_f, double *__restrict__ part)
{
    FFsum s_of, s_oo, s_mf, s_m;
    int n_o = 0, n_f = 0;
    const int L = x1 - x0;
    const int64_t nyr = y1 - y0;
    const int64_t nrows = nyr * (z1 - z0);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t r = warp0; r < nrows; r += nwarps) {
        const int64_t z = z0 + r / nyr;
        const int64_t y = y0 + (r - (r / nyr) * nyr);
        const int64_t base = x0 + nx * (y + ny * z);
        for (int x = lane; x < L; x += 128) {
            float vo[4], vf[4], vm[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int xx = x + 32 * k;
                const bool in = xx < L;
                vo[k] = in ? __ldcs(io_ + base + xx) : 0.0f;
                vf[k] = in ? __ldcs(if_ + base + xx) : -INFINITY;  // outside: no mask
                if (MODEL)
                    vm[k] = in ? __ldcs(im_ + base + xx) : 0.0f;
            }
            float a_of = 0.0f, a_oo = 0.0f, a_mf = 0.0f, a_m = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool in = x + 32 * k < L;
                const bool mo = in && vo[k] >= t_o;
                const bool mf = in && vf[k] >= t_f;
                a_oo = __fadd_rn(a_oo, mo ? vo[k] : 0.0f);
                a_of = __fadd_rn(a_of, mf ? vo[k] : 0.0f);
                n_o += mo ? 1 : 0;
                n_f += mf ? 1 : 0;
                if (MODEL) {
                    a_m = __fadd_rn(a_m, vm[k]);
                    a_mf = __fadd_rn(a_mf, mf ? vm[k] : 0.0f);
                }
            }
            s_of.add(a_of);
            s_oo.add(a_oo);
            if (MODEL) {
                s_mf.add(a_mf);
                s_m.add(a_m);
            }
        }
    }
    double v[6] = {s_of.value(), s_oo.value(), s_mf.value(), s_m.value(),
                   static_cast<double>(n_o), static_cast<double>(n_f)};
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    __shared__ double red[kFdThreads / 32][6];
    const int warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < kFdThreads / 32; ++w)
            acc += red[w][threadIdx.x];
        part[static_cast<int64_t>(blockIdx.x) * 6 + threadIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(kFdThreads)
    fdiag_final(const double *__restrict__ part, int nblocks, double *__restrict__ out6)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            v[q] += part[static_cast<int64_t>(b) * 6 + q];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    __shared__ double red[kFdThreads / 32][6];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < kFdThreads / 32; ++w)
            acc += red[w][threadIdx.x];
        out6[threadIdx.x] = acc;
    }
}

}  // namespace

cudaError_t launch_fdiag(const float *io, const float *iff, const float *im, int64_t nx,
                         int64_t ny, const int roi[6], float t_o, float t_f, double *part,
                         int nblocks, double *out6, cudaStream_t stream)
{
    if (im)
        fdiag_partial<true><<<nblocks, kFdThreads, 0, stream>>>(
            io, iff, im, nx, ny, roi[0], roi[1], roi[2], roi[3], roi[4], roi[5], t_o, t_f, part);
    else
        fdiag_partial<false><<<nblocks, kFdThreads, 0, stream>>>(
            io, iff, im, nx, ny, roi[0], roi[1], roi[2], roi[3], roi[4], roi[5], t_o, t_f, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    fdiag_final<<<1, kFdThreads, 0, stream>>>(part, nblocks, out6);
    return cudaGetLastError();
}

}  // namespace afd
