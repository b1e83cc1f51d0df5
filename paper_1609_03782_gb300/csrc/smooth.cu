// Box and Gaussian smoothing of arXiv:1609.03782 Sec. 3.1 and 3.2 as a
// normalised correlation: out(p) = sum W(q-p) I(q) / sum W(q-p), q over the
// window around p inside the cube (the mean of the existing neighbours for
// the box; constants stay constant).
//
// Separable kernels (the box, and the Gaussian without rotation):
// W = wx (x) wy (x) wz, and the in-cube weight factorises into per-axis sums,
// so out = (wz * (wy * (wx * I))) / (Dx(x) Dy(y) Dz(z)) with zero outside the
// cube, applied as two products with the rounded reciprocals of Dx Dy (per
// voxel column) and Dz (per plane).  One fused pass streams z: a CTA owns a
// 64 x 16 column of the cube over a z-chunk; for every input plane it loads
// the tile and its x/y halo into shared memory (zero outside), convolves
// along x (a register sliding window per 4 outputs) into a second buffer,
// then along y, and pushes the result into a register ring of the last
// 2 RZ + 1 planes per voxel, from which each output plane takes its z sum.
// HBM traffic: one read of the input (the halo rows come from L2) and one
// write.
//
// Rotated Gaussians are not separable: their direct 3-D correlation is in
// smooth_direct.cu.
#include <cmath>

#include "afd_internal.h"
#include "afd_ptx.cuh"
#include "afd_check.cuh"

namespace afd {
namespace {

constexpr int SX = 64;         // tile width (16 threads x 4 voxels)
constexpr int SY = 16;         // tile height (16 thread rows)
constexpr int kSmThreads = 256;

template <int RZ>
__global__ void __launch_bounds__(kSmThreads)
    smooth_sep(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
               int tiles_x, int tiles_y, int zc, const __grid_constant__ SepWeights w, int *err)
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
    float inv_xy[4];
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
            inv_xy[j] = __frcp_rn(__fmul_rn(dx, dy));  // 1 / (in-cube weight of x times y)
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
            if (!check_range(err, r * PW + 4 * q + 2 * rx + 4, 0, PH * PW, kChkSmoothSmem))
                continue;
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
        const bool y_ok = check_range(err, (ty + 2 * ry) * SX + 4 * qx + 3, 0, PH * SX,
                                      kChkSmoothSmem);
        for (int k = 0; k <= 2 * ry && y_ok; ++k) {
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
            const float inv_z = __frcp_rn(dz);
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RZ; ++k)
                    s = __fmaf_rn(w.wz[k], ring[k][j], s);
                o[j] = __fmul_rn(__fmul_rn(s, inv_xy[j]), inv_z);
            }
            float *dst = out + (static_cast<int64_t>(zo) * ny + yr) * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx &&
                    check_range(err, dst + xq + j - out, 0, static_cast<int64_t>(nz) * ny * nx,
                                kChkSmoothStore))
                    dst[xq + j] = o[j];
        }
        // the next iteration rewrites P right away: every read of P happened
        // before the second barrier above; it rewrites X only after its first
        // barrier, which follows these reads of X
    }
}

// The separable pass with its planes streamed by TMA (rows of a multiple of
// 16 bytes): warp 8 issues one 3-D load per plane (tile + halo, zero outside
// the cube) into a ring of kSmSlots slots.  Warps 0-7 convolve the slot's
// rows along x into a double-buffered shared-memory plane, release the slot,
// meet at one named barrier, convolve along y and keep the z window in
// registers: the same products and sums, in the same order, as smooth_sep.
// Every mbarrier wait is bounded (kWaitLimitNs); a thread whose wait expires
// records the error and keeps stepping without waiting again, so every
// consumer reaches every named barrier and the CTA ends.
constexpr int kSmSlots = 4;
constexpr int kSmTmaThreads = kSmThreads + 32;

__device__ __forceinline__ void consumer_barrier()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kSmThreads) : "memory");
}

template <int RZ>
__global__ void __launch_bounds__(kSmTmaThreads)
    smooth_sep_tma(const __grid_constant__ CUtensorMap tmap, float *__restrict__ out, int nx,
                   int ny, int nz, int tiles_x, int tiles_y, int zc, int hx,
                   const __grid_constant__ SepWeights w, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((128u - (base & 127u)) & 127u);
    const int rx = w.rx, ry = w.ry;
    const int SW = SX + 2 * hx, SH = SY + 2 * ry;  // slot: SH rows of SW floats
    const uint32_t slot_bytes = static_cast<uint32_t>(SW * SH) * 4u;
    const uint32_t slot_stride = (slot_bytes + 127u) & ~127u;
    float *X = reinterpret_cast<float *>(smem + kSmSlots * slot_stride);  // 2 x SH x SX
    uint64_t *full = reinterpret_cast<uint64_t *>(X + 2 * SH * SX);
    uint64_t *empty = full + kSmSlots;

    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int x0 = bx * SX, y0 = by * SY;
    const int zs = bz * zc, ze = min(zs + zc, nz);
    const int zlo = max(zs - RZ, 0), zhi = min(ze + RZ, nz) - 1;  // planes loaded

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kSmSlots; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kSmThreads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kSmThreads / 32) {  // ---- producer
        if (lane == 0) {
            for (int j = 0; j <= zhi - zlo; ++j) {
                const int slot = j % kSmSlots, use = j / kSmSlots;
                if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u, err, kErrWaitEmpty))
                    return;
                mbar_arrive_expect_tx(&full[slot], slot_bytes);
                tma_load_3d(smem + slot * slot_stride, &tmap, x0 - hx, y0 - ry, zlo + j,
                            &full[slot]);
            }
        }
        return;
    }

    // ---- consumers: thread (qx, ty) owns 4 voxels of row ty
    const int qx = tid & 15, ty = tid >> 4;
    const int xq = x0 + 4 * qx, yr = y0 + ty;
    float inv_xy[4];
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
            inv_xy[j] = __frcp_rn(__fmul_rn(dx, dy));  // 1 / (in-cube weight of x times y)
        }
    }
    float ring[2 * RZ + 1][4];
#pragma unroll
    for (int m = 0; m < 2 * RZ + 1; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            ring[m][j] = 0.0f;

    bool waiting = true;  // false after an expired wait: no more waits
    for (int zi = zs - RZ; zi < ze + RZ; ++zi) {
        const bool have = zi >= zlo && zi <= zhi;  // the same for the whole CTA
        float *Xb = X + (zi & 1) * SH * SX;
        if (have) {
            const int j = zi - zlo, slot = j % kSmSlots;
            if (waiting && !mbar_wait(&full[slot], (j / kSmSlots) & 1u, err, kErrWaitFull))
                waiting = false;
            const float *S = reinterpret_cast<const float *>(smem + slot * slot_stride);
            // x sums of every slot row: 4 outputs per task; the window of
            // output column 4q starts at column hx + 4q - rx >= 0 and the last
            // read is column hx + 4q + rx + 3 <= SW - 1 (hx >= rx)
            for (int task = tid; task < SH * 16; task += kSmThreads) {
                const int r = task >> 4, q = task & 15;
                if (!(check_range(err, r * SW + hx + 4 * q - rx, 0, SH * SW, kChkSmoothSmem) &&
                      check_range(err, r * SW + hx + 4 * q + rx + 3, 0, SH * SW, kChkSmoothSmem)))
                    continue;
                const float *row = S + r * SW + hx + 4 * q - rx;
                float v0 = row[0], v1 = row[1], v2 = row[2];
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
                for (int k = 0; k <= 2 * rx; ++k) {
                    const float v3 = row[k + 3];
                    const float wk = w.wx[k];
                    a0 = __fmaf_rn(wk, v0, a0);
                    a1 = __fmaf_rn(wk, v1, a1);
                    a2 = __fmaf_rn(wk, v2, a2);
                    a3 = __fmaf_rn(wk, v3, a3);
                    v0 = v1;
                    v1 = v2;
                    v2 = v3;
                }
                *reinterpret_cast<float4 *>(Xb + r * SX + 4 * q) = make_float4(a0, a1, a2, a3);
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[slot]);
        }
        // Xb is complete; the other buffer, written next plane, was last read
        // before this barrier
        consumer_barrier();
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (have && check_range(err, (ty + 2 * ry) * SX + 4 * qx + 3, 0, SH * SX, kChkSmoothSmem)) {
            for (int k = 0; k <= 2 * ry; ++k) {
                const float wk = w.wy[k];
                const float4 v = *reinterpret_cast<const float4 *>(Xb + (ty + k) * SX + 4 * qx);
                c[0] = __fmaf_rn(wk, v.x, c[0]);
                c[1] = __fmaf_rn(wk, v.y, c[1]);
                c[2] = __fmaf_rn(wk, v.z, c[2]);
                c[3] = __fmaf_rn(wk, v.w, c[3]);
            }
        }
#pragma unroll
        for (int m = 0; m < 2 * RZ; ++m)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                ring[m][jj] = ring[m + 1][jj];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
            ring[2 * RZ][jj] = c[jj];
        const int zo = zi - RZ;
        if (zo >= zs && yr < ny && xq < nx) {
            float dz = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RZ; ++k) {
                const int q = zo + k - RZ;
                if (q >= 0 && q < nz)
                    dz = __fadd_rn(dz, w.wz[k]);
            }
            const float inv_z = __frcp_rn(dz);
            float o[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                float sum = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RZ; ++k)
                    sum = __fmaf_rn(w.wz[k], ring[k][jj], sum);
                o[jj] = __fmul_rn(__fmul_rn(sum, inv_xy[jj]), inv_z);
            }
            // nx % 4 == 0 and xq % 4 == 0: the quad is inside the row
            const int64_t oi = (static_cast<int64_t>(zo) * ny + yr) * nx + xq;
            if (check_range(err, oi, 0, static_cast<int64_t>(nz) * ny * nx - 3, kChkSmoothStore))
                *reinterpret_cast<float4 *>(out + oi) = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

template <int RZ>
cudaError_t sep_launch(const float *in, float *out, int nx, int ny, int nz, const SepWeights &w,
                       int zc, int *err, cudaStream_t stream)
{
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int tiles_z = (nz + zc - 1) / zc;
    const size_t smem = static_cast<size_t>((SY + 2 * w.ry) * (SX + 2 * w.rx + 4) +
                                            (SY + 2 * w.ry) * SX) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(smooth_sep<RZ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    smooth_sep<RZ><<<tiles_x * tiles_y * tiles_z, kSmThreads, smem, stream>>>(
        in, out, nx, ny, nz, tiles_x, tiles_y, zc, w, err);
    return cudaGetLastError();
}

template <int RZ>
cudaError_t sep_tma_launch(const CUtensorMap &tmap, float *out, int nx, int ny, int nz,
                           const SepWeights &w, int hx, int *err, cudaStream_t stream)
{
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int zc = nz < 64 ? nz : 64;
    const int tiles_z = (nz + zc - 1) / zc;
    const size_t smem = smooth_tma_smem(w.ry, hx);
    cudaError_t e = cudaFuncSetAttribute(smooth_sep_tma<RZ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    smooth_sep_tma<RZ><<<tiles_x * tiles_y * tiles_z, kSmTmaThreads, smem, stream>>>(
        tmap, out, nx, ny, nz, tiles_x, tiles_y, zc, hx, w, err);
    return cudaGetLastError();
}

template <int... R>
struct SepTmaTable;
template <>
struct SepTmaTable<> {
    static cudaError_t run(int, const CUtensorMap &, float *, int, int, int, const SepWeights &,
                           int, int *, cudaStream_t)
    {
        return cudaErrorInvalidValue;
    }
};
template <int R0, int... R>
struct SepTmaTable<R0, R...> {
    static cudaError_t run(int rz, const CUtensorMap &m, float *out, int nx, int ny, int nz,
                           const SepWeights &w, int hx, int *err, cudaStream_t s)
    {
        if (rz == R0)
            return sep_tma_launch<R0>(m, out, nx, ny, nz, w, hx, err, s);
        return SepTmaTable<R...>::run(rz, m, out, nx, ny, nz, w, hx, err, s);
    }
};

template <int... R>
struct SepTable;
template <>
struct SepTable<> {
    static cudaError_t run(int, const float *, float *, int, int, int, const SepWeights &, int,
                           int *, cudaStream_t)
    {
        return cudaErrorInvalidValue;
    }
};
template <int R0, int... R>
struct SepTable<R0, R...> {
    static cudaError_t run(int rz, const float *in, float *out, int nx, int ny, int nz,
                           const SepWeights &w, int zc, int *err, cudaStream_t s)
    {
        if (rz == R0)
            return sep_launch<R0>(in, out, nx, ny, nz, w, zc, err, s);
        return SepTable<R...>::run(rz, in, out, nx, ny, nz, w, zc, err, s);
    }
};

}  // namespace

size_t smooth_tma_smem(int ry, int hx)
{
    const size_t slot = (static_cast<size_t>(SX + 2 * hx) * (SY + 2 * ry) * 4 + 127) / 128 * 128;
    const size_t xbuf = 2 * static_cast<size_t>(SY + 2 * ry) * SX * sizeof(float);
    return kSmSlots * slot + xbuf + 2 * kSmSlots * sizeof(uint64_t) + 128;
}

void smooth_tma_box(int rx, int ry, int *box_w, int *box_h, int *hx)
{
    *hx = (rx + 3) / 4 * 4;  // x halo: >= rx, a multiple of 4 floats (16-byte TMA x)
    *box_w = SX + 2 * *hx;
    *box_h = SY + 2 * ry;
}

cudaError_t launch_smooth_sep_tma(const CUtensorMap &tmap, float *out, int nx, int ny, int nz,
                                  const SepWeights &w, int hx, int *err, cudaStream_t stream)
{
    if (w.rx < 0 || w.rx > kSepMaxR || w.ry < 0 || w.ry > kSepMaxR || w.rz < 0 ||
        w.rz > kSepMaxRz || hx < w.rx || (nx % 4) != 0)
        return cudaErrorInvalidValue;
    return SepTmaTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::run(w.rz, tmap, out, nx, ny, nz,
                                                                     w, hx, err, stream);
}

cudaError_t launch_smooth_sep(const float *in, float *out, int nx, int ny, int nz,
                              const SepWeights &w, int *err, cudaStream_t stream)
{
    if (w.rx < 0 || w.rx > kSepMaxR || w.ry < 0 || w.ry > kSepMaxR || w.rz < 0 ||
        w.rz > kSepMaxRz)
        return cudaErrorInvalidValue;
    const int zc = nz < 64 ? nz : 64;
    return SepTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::run(w.rz, in, out, nx, ny, nz, w,
                                                                  zc, err, stream);
}

}  // namespace afd
