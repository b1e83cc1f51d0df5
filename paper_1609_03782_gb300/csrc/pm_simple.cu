// One explicit per-face Perona-Malik iteration, one voxel per thread.
//
// arXiv:1609.03782 Sec. 3.3 (eq. "perona", per-face discretisation with the
// gradient conductance).  Every thread reads its voxel and six face neighbours
// straight from global memory (the L1/L2 caches supply the reuse) and writes
// one voxel.  It handles any nx and any alignment; the streaming kernel is the
// fast path.  The arithmetic is the canonical one of afd_math.cuh (scalar
// form), so the result is bit-identical to every other kernel.
#include "afd_internal.h"

namespace afd {

template <int C>
__global__ void __launch_bounds__(256)
    pm_step_simple(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
                   Coef k)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z * blockDim.z + threadIdx.z;
    if (x >= nx || y >= ny || z >= nz)
        return;
    const int64_t sx = 1, sy = nx, sz = static_cast<int64_t>(nx) * ny;
    const int64_t p = x + sy * y + sz * z;
    const float c = in[p];
    // a missing neighbour is replaced by the voxel itself: zero flux
    const float xm = x > 0 ? in[p - sx] : c;
    const float xp = x + 1 < nx ? in[p + sx] : c;
    const float ym = y > 0 ? in[p - sy] : c;
    const float yp = y + 1 < ny ? in[p + sy] : c;
    const float zm = z > 0 ? in[p - sz] : c;
    const float zp = z + 1 < nz ? in[p + sz] : c;
    const float gxm = face_flux<C>(__fsub_rn(c, xm), k.ax, k.bx, k.nz);
    const float gxp = face_flux<C>(__fsub_rn(xp, c), k.ax, k.bx, k.nz);
    const float gym = face_flux<C>(__fsub_rn(c, ym), k.ay, k.by, k.nz);
    const float gyp = face_flux<C>(__fsub_rn(yp, c), k.ay, k.by, k.nz);
    const float gzm = face_flux<C>(__fsub_rn(c, zm), k.az, k.bz, k.nz);
    const float gzp = face_flux<C>(__fsub_rn(zp, c), k.az, k.bz, k.nz);
    if constexpr (C == COND_INT)
        out[p] = pm_update_int(c, gxm, gxp, gym, gyp, gzm, gzp, k.ai);
    else
        out[p] = pm_update(c, gxm, gxp, gym, gyp, gzm, gzp);
}

cudaError_t launch_pm_simple(int cond, const float *in, float *out, int nx, int ny, int nz,
                             const Coef &k, cudaStream_t stream)
{
    const dim3 block(32, 4, 2);
    const dim3 grid((nx + 31) / 32, (ny + 3) / 4, (nz + 1) / 2);
    if (grid.y > 65535u || grid.z > 65535u)
        return cudaErrorInvalidConfiguration;
    switch (cond) {
    case COND_EXP:
        pm_step_simple<COND_EXP><<<grid, block, 0, stream>>>(in, out, nx, ny, nz, k);
        break;
    case COND_RAT:
        pm_step_simple<COND_RAT><<<grid, block, 0, stream>>>(in, out, nx, ny, nz, k);
        break;
    case COND_INT:
        pm_step_simple<COND_INT><<<grid, block, 0, stream>>>(in, out, nx, ny, nz, k);
        break;
    default:
        pm_step_simple<COND_LIN><<<grid, block, 0, stream>>>(in, out, nx, ny, nz, k);
        break;
    }
    return cudaGetLastError();
}

}  // namespace afd
