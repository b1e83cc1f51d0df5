// Box and Gaussian smoothing of arXiv:1609.03782 Sec. 3.1 and 3.2 as a
// normalised correlation: out(p) = sum W(q-p) I(q) / sum W(q-p), q over the
// window around p inside the cube (the mean of the existing neighbours for
// the box; constants stay constant).
//
// Separable kernels (the box, and the Gaussian without rotation):
// W = wx (x) wy (x) wz, and the in-cube weight factorises into per-axis sums,
// so out = (wz * (wy * (wx * I))) / (Dx(x) Dy(y) Dz(z)) with zero outside the
// cube.  One fused pass streams z: a CTA owns a 64 x 16 column of the cube
// over a z-chunk; for every input plane it loads the tile and its x/y halo
// into shared memory (zero outside), convolves along x (a register sliding
// window per 4 outputs) into a second buffer, then along y, and pushes the
// result into a register ring of the last 2 RZ + 1 planes per voxel, from
// which each output plane takes its z sum.  HBM traffic: one read of the
// input (the halo rows come from L2) and one write.
//
// Rotated Gaussians are not separable: a direct 3-D correlation keeps the
// last 2 rz + 1 input planes (tile + halo) in a shared-memory ring and sums
// all taps per output voxel, four voxels per thread along x.
#include <cmath>

#include "afd_internal.h"

namespace afd {
namespace {

constexpr int SX = 64;         // tile width (16 threads x 4 voxels)
constexpr int SY = 16;         // tile height (16 thread rows)
constexpr int kSmThreads = 256;

template <int RZ>
__global__ void __launch_bounds__(kSmThreads)
    smooth_sep(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
               int tiles_x, int tiles_y, int zc, const __grid_constant__ SepWeights w)
{
    extern __shared__ float sm[];
    const int rx = w.rx, ry = w.ry;
    const int PW = SX + 2 * rx + 4;  // raw plane row width (+ 4: the window's last read)
    const int PH = SY + 2 * ry;      // rows convolved along x (even, so X is 16-byte aligned)
    float *P = sm;                   // PH x PW raw plane
    float *X = sm + PH * PW;         // PH x SX, x-convolved

    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int x0 = bx * SX, y0 = by * SY;
    const int zs = bz * zc, ze = min(zs + zc, nz);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qx = tid & 15, ty = tid >> 4;
    const int xq = x0 + 4 * qx, yr = y0 + ty;

    // per-axis normalisation of the voxels this thread writes
    float den_xy[4];  // in-cube weight of x times y
    {
        float dy = 0.0f;
        for (int k = 0; k <= 2 * ry; ++k) {
            const int q = yr + k - ry;
            if (q >= 0 && q < ny)
                dy = __fadd_rn(dy, w.wy[k]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float dx = 0.0f;
            for (int k = 0; k <= 2 * rx; ++k) {
                const int q = xq + j + k - rx;
                if (q >= 0 && q < nx)
                    dx = __fadd_rn(dx, w.wx[k]);
            }
            den_xy[j] = __fmul_rn(dx, dy);
        }
    }

    float ring[2 * RZ + 1][4];
#pragma unroll
    for (int m = 0; m < 2 * RZ + 1; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            ring[m][j] = 0.0f;

    for (int zi = zs - RZ; zi < ze + RZ; ++zi) {
        // ---- 1: the raw plane zi (tile + halo), zero outside the cube
        const bool zin = zi >= 0 && zi < nz;
        const float *src = in + static_cast<int64_t>(zi) * nx * ny;
        for (int r = warp; r < PH; r += kSmThreads / 32) {
            const int gy = y0 - ry + r;
            const bool yin = zin && gy >= 0 && gy < ny;
            for (int c = lane; c < PW; c += 32) {
                const int gx = x0 - rx + c;
                P[r * PW + c] = (yin && gx >= 0 && gx < nx)
                                    ? __ldg(src + static_cast<int64_t>(gy) * nx + gx)
                                    : 0.0f;
            }
        }
        __syncthreads();
        // ---- 2: x convolution of every row, 4 outputs per task
        for (int task = tid; task < PH * 16; task += kSmThreads) {
            const int r = task >> 4, q = task & 15;
            const float *row = P + r * PW + 4 * q;
            float v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3];
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
            for (int k = 0; k <= 2 * rx; ++k) {
                const float wk = w.wx[k];
                a0 = __fmaf_rn(wk, v0, a0);
                a1 = __fmaf_rn(wk, v1, a1);
                a2 = __fmaf_rn(wk, v2, a2);
                a3 = __fmaf_rn(wk, v3, a3);
                v0 = v1;
                v1 = v2;
                v2 = v3;
                v3 = row[k + 4];  // 4q + k + 4 <= 64 + 2 rx < PW
            }
            float4 *dst = reinterpret_cast<float4 *>(X + r * SX + 4 * q);
            *dst = make_float4(a0, a1, a2, a3);
        }
        __syncthreads();
        // ---- 3: y convolution, into the z ring
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int k = 0; k <= 2 * ry; ++k) {
            const float wk = w.wy[k];
            const float4 v = *reinterpret_cast<const float4 *>(X + (ty + k) * SX + 4 * qx);
            c[0] = __fmaf_rn(wk, v.x, c[0]);
            c[1] = __fmaf_rn(wk, v.y, c[1]);
            c[2] = __fmaf_rn(wk, v.z, c[2]);
            c[3] = __fmaf_rn(wk, v.w, c[3]);
        }
#pragma unroll
        for (int m = 0; m < 2 * RZ; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                ring[m][j] = ring[m + 1][j];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            ring[2 * RZ][j] = c[j];
        // ---- 4: the output plane zo = zi - RZ: z sum, normalise, store
        const int zo = zi - RZ;
        if (zo >= zs && yr < ny) {
            float dz = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RZ; ++k) {
                const int q = zo + k - RZ;
                if (q >= 0 && q < nz)
                    dz = __fadd_rn(dz, w.wz[k]);
            }
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RZ; ++k)
                    s = __fmaf_rn(w.wz[k], ring[k][j], s);
                o[j] = __fdiv_rn(s, __fmul_rn(den_xy[j], dz));
            }
            float *dst = out + (static_cast<int64_t>(zo) * ny + yr) * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx)
                    dst[xq + j] = o[j];
        }
        // the next iteration rewrites P right away: every read of P happened
        // before the second barrier above; it rewrites X only after its first
        // barrier, which follows these reads of X
    }
}

// Direct correlation with a full (2rx+1) x (2ry+1) x (2rz+1) weight array
// (rotated Gaussian).  Shared memory: the weights, then a ring of 2 rz + 1
// raw planes of PH x PW (tile + halo).
__global__ void __launch_bounds__(kSmThreads)
    smooth_direct(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
                  int tiles_x, int tiles_y, int zc, const float *__restrict__ W, int rx, int ry,
                  int rz)
{
    extern __shared__ float sm[];
    const int WX = 2 * rx + 1, WY = 2 * ry + 1, WZ = 2 * rz + 1;
    const int PW = SX + 2 * rx + 4;  // + 4: the sliding window reads 4 past its last tap
    const int PH = SY + 2 * ry;
    float *Ws = sm;
    float *ring = sm + WX * WY * WZ;

    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int x0 = bx * SX, y0 = by * SY;
    const int zs = bz * zc, ze = min(zs + zc, nz);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qx = tid & 15, ty = tid >> 4;
    const int xq = x0 + 4 * qx, yr = y0 + ty;

    for (int i = tid; i < WX * WY * WZ; i += kSmThreads)
        Ws[i] = W[i];

    // normalisation: the in-cube weight of each output voxel depends on z;
    // it is summed with the same loops as the numerator, from a ones plane
    for (int zi = zs - rz; zi < ze + rz; ++zi) {
        // ---- load plane zi into its ring slot (the slot last read for the
        // output plane zi - 2 rz - 1, finished before the barrier below)
        float *P = ring + ((zi - (zs - rz)) % WZ) * PH * PW;
        const bool zin = zi >= 0 && zi < nz;
        const float *src = in + static_cast<int64_t>(zi) * nx * ny;
        for (int r = warp; r < PH; r += kSmThreads / 32) {
            const int gy = y0 - ry + r;
            const bool yin = zin && gy >= 0 && gy < ny;
            for (int c = lane; c < PW; c += 32) {
                const int gx = x0 - rx + c;
                P[r * PW + c] = (yin && gx >= 0 && gx < nx)
                                    ? __ldg(src + static_cast<int64_t>(gy) * nx + gx)
                                    : 0.0f;
            }
        }
        __syncthreads();
        const int zo = zi - rz;  // every plane of its window is now in the ring
        if (zo >= zs && yr < ny) {
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int dz = 0; dz < WZ; ++dz) {
                const int qz = zo - rz + dz;
                if (qz < 0 || qz >= nz)
                    continue;
                const float *Pz = ring + ((qz - (zs - rz)) % WZ) * PH * PW;
                for (int dy = 0; dy < WY; ++dy) {
                    const int qy = yr - ry + dy;
                    if (qy < 0 || qy >= ny)
                        continue;
                    const float *row = Pz + (ty + dy) * PW + 4 * qx;
                    const float *wrow = Ws + (dz * WY + dy) * WX;
                    float v0 = row[0], v1 = row[1], v2 = row[2], v3 = row[3];
                    for (int dx = 0; dx < WX; ++dx) {
                        const float wk = wrow[dx];
                        const int gx = xq - rx + dx;
                        a[0] = __fmaf_rn(wk, v0, a[0]);
                        a[1] = __fmaf_rn(wk, v1, a[1]);
                        a[2] = __fmaf_rn(wk, v2, a[2]);
                        a[3] = __fmaf_rn(wk, v3, a[3]);
                        d[0] = (gx >= 0 && gx < nx) ? __fadd_rn(d[0], wk) : d[0];
                        d[1] = (gx + 1 >= 0 && gx + 1 < nx) ? __fadd_rn(d[1], wk) : d[1];
                        d[2] = (gx + 2 >= 0 && gx + 2 < nx) ? __fadd_rn(d[2], wk) : d[2];
                        d[3] = (gx + 3 >= 0 && gx + 3 < nx) ? __fadd_rn(d[3], wk) : d[3];
                        v0 = v1;
                        v1 = v2;
                        v2 = v3;
                        v3 = row[dx + 4];
                    }
                }
            }
            float *dst = out + (static_cast<int64_t>(zo) * ny + yr) * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx)
                    dst[xq + j] = __fdiv_rn(a[j], d[j]);
        }
        __syncthreads();  // the ring slot of plane zi - 2 rz is refilled next
    }
}

template <int RZ>
cudaError_t sep_launch(const float *in, float *out, int nx, int ny, int nz, const SepWeights &w,
                       int zc, cudaStream_t stream)
{
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int tiles_z = (nz + zc - 1) / zc;
    const size_t smem = static_cast<size_t>((SY + 2 * w.ry) * (SX + 2 * w.rx + 4) +
                                            (SY + 2 * w.ry) * SX) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(smooth_sep<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    smooth_sep<RZ><<<tiles_x * tiles_y * tiles_z, kSmThreads, smem, stream>>>(
        in, out, nx, ny, nz, tiles_x, tiles_y, zc, w);
    return cudaGetLastError();
}

template <int... R>
struct SepTable;
template <>
struct SepTable<> {
    static cudaError_t run(int, const float *, float *, int, int, int, const SepWeights &, int,
                           cudaStream_t)
    {
        return cudaErrorInvalidValue;
    }
};
template <int R0, int... R>
struct SepTable<R0, R...> {
    static cudaError_t run(int rz, const float *in, float *out, int nx, int ny, int nz,
                           const SepWeights &w, int zc, cudaStream_t s)
    {
        if (rz == R0)
            return sep_launch<R0>(in, out, nx, ny, nz, w, zc, s);
        return SepTable<R...>::run(rz, in, out, nx, ny, nz, w, zc, s);
    }
};

}  // namespace

size_t smooth_direct_smem(int rx, int ry, int rz)
{
    const size_t wts = static_cast<size_t>(2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1);
    const size_t ring = static_cast<size_t>(2 * rz + 1) * (SY + 2 * ry) * (SX + 2 * rx + 4);
    return (wts + ring) * sizeof(float);
}

cudaError_t launch_smooth_sep(const float *in, float *out, int nx, int ny, int nz,
                              const SepWeights &w, cudaStream_t stream)
{
    if (w.rx < 0 || w.rx > kSepMaxR || w.ry < 0 || w.ry > kSepMaxR || w.rz < 0 ||
        w.rz > kSepMaxRz)
        return cudaErrorInvalidValue;
    const int zc = nz < 64 ? nz : 64;
    return SepTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::run(w.rz, in, out, nx, ny, nz, w,
                                                                  zc, stream);
}

cudaError_t launch_smooth_direct(const float *in, float *out, int nx, int ny, int nz,
                                 const float *W, int rx, int ry, int rz, cudaStream_t stream)
{
    const size_t smem = smooth_direct_smem(rx, ry, rz);
    cudaError_t e = cudaFuncSetAttribute(smooth_direct, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int zc = nz < 32 ? nz : 32;
    const int tiles_z = (nz + zc - 1) / zc;
    smooth_direct<<<tiles_x * tiles_y * tiles_z, kSmThreads, smem, stream>>>(
        in, out, nx, ny, nz, tiles_x, tiles_y, zc, W, rx, ry, rz);
    return cudaGetLastError();
}

}  // namespace afd
