// Smoothing with a rotated Gaussian (arXiv:1609.03782 Sec. 3.2, the
// anisotropic kernel turned by Euler angles) as a normalised correlation,
// out(p) = sum W(q-p) I(q) / sum W(q-p) over the taps inside the cube.  The
// rotated kernel is not separable: a direct 3-D correlation keeps the last
// input planes (tile + halo) in a shared-memory ring and sums every tap of
// every output voxel in FP32 multiply-adds.  The pass is bound by those
// multiply-adds, not by HBM.
#include <cmath>

#include "afd_internal.h"
#include "afd_check.cuh"

namespace afd {
namespace {

constexpr int SX = 64;         // tile width (16 threads x 4 voxels)
constexpr int SY = 16;         // tile height of smooth_direct (16 thread rows)
constexpr int kSmThreads = 256;

// In-cube weight of the window around voxel (x, y, z): the taps inside the
// cube form a box of the kernel ([lx, hx) x [ly, hy) x [lz, hz) in tap
// indices), summed by inclusion-exclusion over the FP64 prefix sums
// S[k][j][i] = sum of W over dz < k, dy < j, dx < i (a (WZ+1) x (WY+1) x
// (WX+1) table) and rounded once.  Eight loads per voxel, for voxels within
// a radius of a face only.
__device__ __forceinline__ float face_weight(const double *__restrict__ S, int x, int y, int z,
                                             int nx, int ny, int nz, int rx, int ry, int rz)
{
    const int WX1 = 2 * rx + 2, WY1 = 2 * ry + 2;
    const int lx = max(0, rx - x), hx = min(2 * rx + 1, nx - x + rx);
    const int ly = max(0, ry - y), hy = min(2 * ry + 1, ny - y + ry);
    const int lz = max(0, rz - z), hz = min(2 * rz + 1, nz - z + rz);
    auto at = [&](int k, int j, int i) { return __ldg(S + (k * WY1 + j) * WX1 + i); };
    const double d = at(hz, hy, hx) - at(lz, hy, hx) - at(hz, ly, hx) - at(hz, hy, lx) +
                     at(lz, ly, hx) + at(lz, hy, lx) + at(hz, ly, lx) - at(lz, ly, lx);
    return __double2float_rn(d);
}

// Direct correlation with a full (2rx+1) x (2ry+1) x (2rz+1) weight array
// (rotated Gaussian).  Shared memory: the weights, then a ring of 2 rz + 1
// raw planes of PH x PW (tile + halo).  A voxel whose window lies inside the
// cube divides by the kernel's total weight wsum (summed in double on the
// host, rounded once); one within a radius of a face by face_weight().
__global__ void __launch_bounds__(kSmThreads)
    smooth_direct(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
                  int tiles_x, int tiles_y, int zc, const float *__restrict__ W,
                  const double *__restrict__ S, int rx, int ry, int rz, float wsum, int *err)
{
    extern __shared__ float sm[];
    const int WX = 2 * rx + 1, WY = 2 * ry + 1, WZ = 2 * rz + 1;
    const int PW = SX + 2 * rx + 4;  // + 4: room for the sliding window's reads
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
    const bool xy_inside = xq - rx >= 0 && xq + 3 + rx < nx && yr - ry >= 0 && yr + ry < ny;

    for (int i = tid; i < WX * WY * WZ; i += kSmThreads)
        Ws[i] = W[i];

    for (int zi = zs - rz; zi < ze + rz; ++zi) {
        // ---- load plane zi into its ring slot (the slot's previous plane,
        // zi - 2 rz - 1, was last read before the barrier ending the
        // previous iteration)
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
        // the farthest ring read of this thread: row ty + 2 ry, column 4 qx + 2 rx + 3
        if (zo >= zs && yr < ny &&
            check_range(err, (ty + 2 * ry) * PW + 4 * qx + 2 * rx + 3, 0, PH * PW,
                        kChkSmoothSmem)) {
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int dz = 0; dz < WZ; ++dz) {
                const int qz = zo - rz + dz;
                if (qz < 0 || qz >= nz)
                    continue;  // zero plane
                const float *Pz = ring + ((qz - (zs - rz)) % WZ) * PH * PW;
                for (int dy = 0; dy < WY; ++dy) {
                    // row ty + dy of the slot; the window's last read is
                    // column 4 qx + 2 rx + 3 < PW
                    const float *row = Pz + (ty + dy) * PW + 4 * qx;
                    const float *wrow = Ws + (dz * WY + dy) * WX;
                    float v0 = row[0], v1 = row[1], v2 = row[2];
                    for (int dx = 0; dx < WX; ++dx) {
                        const float v3 = row[dx + 3];
                        const float wk = wrow[dx];
                        a[0] = __fmaf_rn(wk, v0, a[0]);
                        a[1] = __fmaf_rn(wk, v1, a[1]);
                        a[2] = __fmaf_rn(wk, v2, a[2]);
                        a[3] = __fmaf_rn(wk, v3, a[3]);
                        v0 = v1;
                        v1 = v2;
                        v2 = v3;
                    }
                }
            }
            float d[4] = {wsum, wsum, wsum, wsum};
            if (!(xy_inside && zo - rz >= 0 && zo + rz < nz)) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (xq + j < nx)
                        d[j] = face_weight(S, xq + j, yr, zo, nx, ny, nz, rx, ry, rz);
            }
            float *dst = out + (static_cast<int64_t>(zo) * ny + yr) * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx &&
                    check_range(err, dst + xq + j - out, 0, static_cast<int64_t>(nz) * ny * nx,
                                kChkSmoothStore))
                    dst[xq + j] = __fdiv_rn(a[j], d[j]);
        }
        __syncthreads();  // the ring slot of plane zi - 2 rz is refilled next
    }
}

// The direct correlation, register-blocked: a 64 x 32 tile, each thread 4
// voxels of two rows, compiled per x radius.  Weight rows are zero-padded
// to 4 NG taps and the input window moves in aligned 16-byte loads, four
// taps per load; the padding taps are skipped, never multiplied.  Every
// input row a thread loads feeds both of its output rows (weight rows dy
// and dy - 1), so a tap costs a quarter of a shared-memory float per
// product.  Ring planes are PH x PW with PH = 32 + 2 ry and PW = 64 + 4 NG,
// the first column at x0 - rx; the ring holds 2 rz + 2 planes, and the next
// input plane is copied (cp.async, zero-filled outside the cube in x and y)
// into the spare one while the current output plane is summed.  A voxel
// whose window lies inside the cube divides by wsum; one near a face by
// face_weight().
constexpr int SY2 = 32;
constexpr int kDirectMaxRx = 15;

__device__ __forceinline__ void cp_async_f32(float *dst, const float *src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// acc[j] += sum over the row's taps of w[dx] d[j + dx]; d holds NG + 1
// float4 of the input row from the thread's first column on.
template <int NG, int LAST>
__device__ __forceinline__ void direct_row(float (&acc)[4], const float4 (&d)[NG + 1],
                                           const float4 (&wr)[NG])
{
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const float4 w4 = wr[g];
        const float v[8] = {d[g].x, d[g].y, d[g].z, d[g].w,
                            d[g + 1].x, d[g + 1].y, d[g + 1].z, d[g + 1].w};
        const float wk[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            if (g == NG - 1 && tt >= LAST)
                break;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                acc[j] = __fmaf_rn(wk[tt], v[j + tt], acc[j]);
        }
    }
}

// Both output rows from one input row: a0 with weight row wa, a1 with
// weight row wb, interleaved (eight independent chains).
template <int NG, int LAST>
__device__ __forceinline__ void direct_row2(float (&a0)[4], float (&a1)[4],
                                            const float4 (&d)[NG + 1], const float4 (&wa)[NG],
                                            const float4 (&wb)[NG])
{
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const float v[8] = {d[g].x, d[g].y, d[g].z, d[g].w,
                            d[g + 1].x, d[g + 1].y, d[g + 1].z, d[g + 1].w};
        const float ka[4] = {wa[g].x, wa[g].y, wa[g].z, wa[g].w};
        const float kb[4] = {wb[g].x, wb[g].y, wb[g].z, wb[g].w};
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            if (g == NG - 1 && tt >= LAST)
                break;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                a0[j] = __fmaf_rn(ka[tt], v[j + tt], a0[j]);
                a1[j] = __fmaf_rn(kb[tt], v[j + tt], a1[j]);
            }
        }
    }
}

template <int NG>
__device__ __forceinline__ void load_row(float4 (&d)[NG + 1], const float *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int g = 0; g <= NG; ++g)
        d[g] = q[g];
}

template <int NG>
__device__ __forceinline__ void load_wrow(float4 (&w)[NG], const float4 *q)
{
#pragma unroll
    for (int g = 0; g < NG; ++g)
        w[g] = q[g];
}

template <int RX>
__global__ void __launch_bounds__(kSmThreads, 1)
    smooth_direct2(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
                   int tiles_x, int tiles_y, int zc, const float *__restrict__ W,
                   const double *__restrict__ S, int ry, int rz, float wsum, int *err)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int rx = RX, WX = 2 * RX + 1;
    constexpr int NG = (WX + 3) / 4;          // groups of four x taps
    constexpr int LAST = WX - 4 * (NG - 1);   // taps in the last group
    const int WY = 2 * ry + 1, WZ = 2 * rz + 1;
    constexpr int WXP = 4 * NG;
    constexpr int PW = SX + WXP;   // a multiple of 4: rows stay 16-byte aligned
    const int PH = SY2 + 2 * ry;
    const int NS = WZ + 1;         // ring slots
    float *Ws = sm;                // WZ x WY rows of WXP taps
    float *ring = sm + WZ * WY * WXP;

    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int x0 = bx * SX, y0 = by * SY2;
    const int zs = bz * zc, ze = min(zs + zc, nz);
    const int zb = zs - rz;        // first ring plane

    const int tid = threadIdx.x;
    const int qx = tid & 15, ry2 = tid >> 4;
    const int xq = x0 + 4 * qx, ya = y0 + 2 * ry2, yb = ya + 1;
    const bool xy_inside = xq - rx >= 0 && xq + 3 + rx < nx && ya - ry >= 0 && yb + ry < ny;

    for (int i = tid; i < WZ * WY * WXP; i += kSmThreads) {
        const int kx = i % WXP, row = i / WXP;
        Ws[i] = kx < WX ? W[row * WX + kx] : 0.0f;
    }

    // copy input plane zi (inside the cube in z) into its ring slot
    auto fetch = [&](int zi) {
        float *P = ring + ((zi - zb) % NS) * PH * PW;
        const float *src = in + static_cast<int64_t>(zi) * nx * ny;
        for (int i = tid; i < PH * PW; i += kSmThreads) {
            const int r = i / PW, c = i - r * PW;
            const int gy = y0 - ry + r, gx = x0 - rx + c;
            const bool ok = gy >= 0 && gy < ny && gx >= 0 && gx < nx;
            cp_async_f32(P + i, ok ? src + static_cast<int64_t>(gy) * nx + gx : in, ok);
        }
        cp_async_commit();
    };

    const int zlast = min(ze + rz, nz);   // one past the last input plane
    const int zfirst = max(zb, 0);
    if (zfirst < zlast)
        fetch(zfirst);
    for (int zi = zfirst; zi < ze + rz; ++zi) {
        cp_async_wait_all();
        __syncthreads();   // plane zi landed; the slot of zi + 1 is free
        if (zi + 1 < zlast)
            fetch(zi + 1);
        const int zo = zi - rz;
        // farthest read: row 2 ry2 + 2 ry + 1, columns up to 4 qx + WXP + 3
        if (zo < zs || ya >= ny ||
            !check_range(err, (2 * ry2 + 1 + 2 * ry) * PW + 4 * qx + WXP + 3, 0, PH * PW,
                         kChkSmoothSmem))
            continue;
        float a0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int dz = 0; dz < WZ; ++dz) {
            const int qz = zo - rz + dz;
            if (qz < 0 || qz >= nz)
                continue;  // zero plane
            const float *Pz = ring + ((qz - zb) % NS) * PH * PW + 2 * ry2 * PW + 4 * qx;
            const float4 *wz = reinterpret_cast<const float4 *>(Ws + dz * WY * WXP);
            // input row r of the thread's window: output row a takes weight
            // row r, output row b weight row r - 1.  The next input row is
            // loaded while the current one is summed; rows go in pairs so
            // that the two register buffers swap roles without copies.
            float4 d[NG + 1], dn[NG + 1], wc[NG], wp[NG];
            load_row<NG>(d, Pz);
            load_wrow<NG>(wp, wz);
            load_row<NG>(dn, Pz + PW);
            direct_row<NG, LAST>(a0, d, wp);
            // here: dn = input row r, wp = weight row r - 1
            int r = 1;
            for (; r + 1 < WY; r += 2) {
                load_row<NG>(d, Pz + (r + 1) * PW);
                load_wrow<NG>(wc, wz + r * NG);
                direct_row2<NG, LAST>(a0, a1, dn, wc, wp);
                load_row<NG>(dn, Pz + (r + 2) * PW);
                load_wrow<NG>(wp, wz + (r + 1) * NG);
                direct_row2<NG, LAST>(a0, a1, d, wp, wc);
            }
            if (r < WY) {  // r = WY - 1: one interior row left, then row WY
                load_row<NG>(d, Pz + (r + 1) * PW);
                load_wrow<NG>(wc, wz + r * NG);
                direct_row2<NG, LAST>(a0, a1, dn, wc, wp);
                direct_row<NG, LAST>(a1, d, wc);
            } else {       // r = WY: row WY only
                direct_row<NG, LAST>(a1, dn, wp);
            }
        }
        float d0[4] = {wsum, wsum, wsum, wsum}, d1[4] = {wsum, wsum, wsum, wsum};
        if (!(xy_inside && zo - rz >= 0 && zo + rz < nz)) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx) {
                    d0[j] = face_weight(S, xq + j, ya, zo, nx, ny, nz, rx, ry, rz);
                    if (yb < ny)
                        d1[j] = face_weight(S, xq + j, yb, zo, nx, ny, nz, rx, ry, rz);
                }
        }
        const int64_t oext = static_cast<int64_t>(nz) * ny * nx;
        float *dst0 = out + (static_cast<int64_t>(zo) * ny + ya) * nx;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (xq + j < nx && check_range(err, dst0 + xq + j - out, 0, oext, kChkSmoothStore))
                dst0[xq + j] = __fdiv_rn(a0[j], d0[j]);
            if (xq + j < nx && yb < ny &&
                check_range(err, dst0 + nx + xq + j - out, 0, oext, kChkSmoothStore))
                dst0[nx + xq + j] = __fdiv_rn(a1[j], d1[j]);
        }
    }
}

using DirectKernel = void (*)(const float *, float *, int, int, int, int, int, int, const float *,
                              const double *, int, int, float, int *);
constexpr DirectKernel kDirect2[kDirectMaxRx + 1] = {
    smooth_direct2<0>,  smooth_direct2<1>,  smooth_direct2<2>,  smooth_direct2<3>,
    smooth_direct2<4>,  smooth_direct2<5>,  smooth_direct2<6>,  smooth_direct2<7>,
    smooth_direct2<8>,  smooth_direct2<9>,  smooth_direct2<10>, smooth_direct2<11>,
    smooth_direct2<12>, smooth_direct2<13>, smooth_direct2<14>, smooth_direct2<15>};

}  // namespace

size_t smooth_direct_smem(int rx, int ry, int rz)
{
    const size_t wts = static_cast<size_t>(2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1);
    const size_t ring = static_cast<size_t>(2 * rz + 1) * (SY + 2 * ry) * (SX + 2 * rx + 4);
    return (wts + ring) * sizeof(float);
}

size_t smooth_direct2_smem(int rx, int ry, int rz)
{
    const size_t wxp = static_cast<size_t>((2 * rx + 1 + 3) & ~3);
    const size_t wts = wxp * (2 * ry + 1) * (2 * rz + 1);
    const size_t ring = static_cast<size_t>(2 * rz + 2) * (SY2 + 2 * ry) * (SX + wxp);
    return (wts + ring) * sizeof(float);
}

cudaError_t launch_smooth_direct(const float *in, float *out, int nx, int ny, int nz,
                                 const float *W, const double *S, int rx, int ry, int rz,
                                 float wsum, int *err, cudaStream_t stream)
{
    const size_t smem2 = smooth_direct2_smem(rx, ry, rz);
    if (rx <= kDirectMaxRx && smem2 <= 227 * 1024) {
        const DirectKernel k = kDirect2[rx];
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem2));
        if (e != cudaSuccess)
            return e;
        const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY2 - 1) / SY2;
        const int zc = nz < 32 ? nz : 32;
        const int tiles_z = (nz + zc - 1) / zc;
        k<<<tiles_x * tiles_y * tiles_z, kSmThreads, smem2, stream>>>(
            in, out, nx, ny, nz, tiles_x, tiles_y, zc, W, S, ry, rz, wsum, err);
        return cudaGetLastError();
    }
    const size_t smem = smooth_direct_smem(rx, ry, rz);
    cudaError_t e = cudaFuncSetAttribute(smooth_direct, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int zc = nz < 32 ? nz : 32;
    const int tiles_z = (nz + zc - 1) / zc;
    smooth_direct<<<tiles_x * tiles_y * tiles_z, kSmThreads, smem, stream>>>(
        in, out, nx, ny, nz, tiles_x, tiles_y, zc, W, S, rx, ry, rz, wsum, err);
    return cudaGetLastError();
}

}  // namespace afd
