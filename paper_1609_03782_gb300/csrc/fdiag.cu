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
// (lanes along x; four float4 loads per cube per lane per step when the rows
// are 16-byte aligned, else four scalars; all loads issued before they are
// used); a
// lane's four values are summed in float32 and the sums
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

// One element's contribution to the four partial sums and two counts.
template <bool MODEL>
__device__ __forceinline__ void fd_term(bool in, float vo, float vf, float vm, float t_o,
                                        float t_f, float &a_of, float &a_oo, float &a_mf,
                                        float &a_m, int &n_o, int &n_f)
{
    const bool mo = in && vo >= t_o;
    const bool mf = in && vf >= t_f;
    a_oo = __fadd_rn(a_oo, mo ? vo : 0.0f);
    a_of = __fadd_rn(a_of, mf ? vo : 0.0f);
    n_o += mo ? 1 : 0;
    n_f += mf ? 1 : 0;
    if (MODEL) {
        a_m = __fadd_rn(a_m, in ? vm : 0.0f);
        a_mf = __fadd_rn(a_mf, mf ? vm : 0.0f);
    }
}

// VEC: rows start 16-byte aligned and hold a multiple of 4 elements; each
// lane then loads float4s (two per cube per step), else four scalars.
template <bool MODEL, bool VEC>
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
        if (VEC) {
            const float4 *po = reinterpret_cast<const float4 *>(io_ + base);
            const float4 *pf = reinterpret_cast<const float4 *>(if_ + base);
            const float4 *pm = MODEL ? reinterpret_cast<const float4 *>(im_ + base) : nullptr;
            const int L4 = L / 4;
            for (int q = lane; q < L4; q += 128) {
                float4 vo[4], vf[4], vm[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool in = q + 32 * k < L4;
                    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    vo[k] = in ? __ldcs(po + q + 32 * k) : zero;
                    vf[k] = in ? __ldcs(pf + q + 32 * k) : zero;
                    if (MODEL)
                        vm[k] = in ? __ldcs(pm + q + 32 * k) : zero;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool in = q + 32 * k < L4;
                    float a_of = 0.0f, a_oo = 0.0f, a_mf = 0.0f, a_m = 0.0f;
                    fd_term<MODEL>(in, vo[k].x, vf[k].x, vm[k].x, t_o, t_f, a_of, a_oo, a_mf, a_m,
                                   n_o, n_f);
                    fd_term<MODEL>(in, vo[k].y, vf[k].y, vm[k].y, t_o, t_f, a_of, a_oo, a_mf, a_m,
                                   n_o, n_f);
                    fd_term<MODEL>(in, vo[k].z, vf[k].z, vm[k].z, t_o, t_f, a_of, a_oo, a_mf, a_m,
                                   n_o, n_f);
                    fd_term<MODEL>(in, vo[k].w, vf[k].w, vm[k].w, t_o, t_f, a_of, a_oo, a_mf, a_m,
                                   n_o, n_f);
                    s_of.add(a_of);
                    s_oo.add(a_oo);
                    if (MODEL) {
                        s_mf.add(a_mf);
                        s_m.add(a_m);
                    }
                }
            }
            continue;
        }
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
            for (int k = 0; k < 4; ++k)
                fd_term<MODEL>(x + 32 * k < L, vo[k], vf[k], MODEL ? vm[k] : 0.0f, t_o, t_f, a_of,
                               a_oo, a_mf, a_m, n_o, n_f);
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
    auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec = (nx % 4) == 0 && (roi[0] % 4) == 0 && ((roi[1] - roi[0]) % 4) == 0 &&
                     al16(io) && al16(iff) && (!im || al16(im));
#define FD_LAUNCH(M, V)                                                                     \
    fdiag_partial<M, V><<<nblocks, kFdThreads, 0, stream>>>(io, iff, im, nx, ny, roi[0], roi[1], \
                                                             roi[2], roi[3], roi[4], roi[5], t_o, \
                                                             t_f, part)
    if (im) {
        if (vec)
            FD_LAUNCH(true, true);
        else
            FD_LAUNCH(true, false);
    } else {
        if (vec)
            FD_LAUNCH(false, true);
        else
            FD_LAUNCH(false, false);
    }
#undef FD_LAUNCH
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    fdiag_final<<<1, kFdThreads, 0, stream>>>(part, nblocks, out6);
    return cudaGetLastError();
}

}  // namespace afd
