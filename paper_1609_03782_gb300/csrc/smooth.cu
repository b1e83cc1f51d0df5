// Box and Gaussian smoothing of arXiv:1609.03782 Sec. 3.1 and 3.2 as a
// normalised correlation: out(p) = sum W(q-p) I(q) / sum W(q-p), q over the
// window around p inside the cube (the mean of the existing neighbours for
// the box; constants stay constant).
//
// Separable kernels (the box, and the Gaussian without rotation):
// W = wx (x) wy (x) wz, and the in-cube weight factorises into per-axis sums,
// so out = (wz * (wx * (wy * I))) / (Dx(x) Dy(y) Dz(z)) with zero outside the
// cube (each output sums its taps y first, then x, then z, each in tap
// order), applied as two products with the rounded reciprocals of Dx Dy (per
// voxel column) and Dz (per plane).  One fused pass streams z: a CTA owns a
// 64 x 16 column of the cube over a z-chunk; for every input plane it has
// the tile and its x/y halo in shared memory (zero outside), takes the y
// sums of the tile's rows over every column (two rows per loaded row), then
// the x sums of each thread's 4 voxels (a register sliding window), and
// keeps the last 2 RZ + 1 planes' sums per voxel (in registers for small
// RZ, in shared memory from kSepSmemRingRz on), from which each output plane
// takes its z sum.  HBM traffic: one read of the input (the halo rows come
// from L2) and one write.
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

// ---- the arithmetic shared by both separable passes (same products and
// sums, in the same order, whichever way the planes arrive)

// 1 / (in-cube weight along x times along y) of the thread's four voxels
__device__ __forceinline__ void sep_inv_xy(const SepWeights &w, int xq, int yr, int nx, int ny,
                                           float (&inv_xy)[4])
{
    float dy = 0.0f;
    for (int k = 0; k <= 2 * w.ry; ++k) {
        const int q = yr + k - w.ry;
        if (q >= 0 && q < ny)
            dy = __fadd_rn(dy, w.wy[k]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float dx = 0.0f;
        for (int k = 0; k <= 2 * w.rx; ++k) {
            const int q = xq + j + k - w.rx;
            if (q >= 0 && q < nx)
                dx = __fadd_rn(dx, w.wx[k]);
        }
        inv_xy[j] = __frcp_rn(__fmul_rn(dx, dy));
    }
}

// 1 / (in-cube weight along z) of output plane zo; inv_full is that of a
// plane whose window lies inside the cube (the same sum, taken once)
template <int RZ>
__device__ __forceinline__ float sep_inv_z(const SepWeights &w, int zo, int nz, float inv_full)
{
    if (zo - RZ >= 0 && zo + RZ < nz)
        return inv_full;
    float dz = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * RZ; ++k) {
        const int q = zo + k - RZ;
        if (q >= 0 && q < nz)
            dz = __fadd_rn(dz, w.wz[k]);
    }
    return __frcp_rn(dz);
}

template <int RZ>
__device__ __forceinline__ float sep_inv_z_full(const SepWeights &w)
{
    float dz = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * RZ; ++k)
        dz = __fadd_rn(dz, w.wz[k]);
    return __frcp_rn(dz);
}

// y sums of four columns of one row: Y(r, c..c+3) = sum_k wy[k] P(r+k, c..c+3),
// k ascending; P rows of pp floats (pp % 4 == 0, c % 4 == 0), Y rows of yp
// (even) floats
__device__ __forceinline__ void sep_y_quad(const float *__restrict__ P, int pp,
                                           float *__restrict__ Y, int yp, int r, int c,
                                           const SepWeights &w)
{
    const float *p = P + r * pp + c;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 4
    for (int k = 0; k <= 2 * w.ry; ++k) {
        const float4 v = *reinterpret_cast<const float4 *>(p + k * pp);
        const float wk = w.wy[k];
        a0 = __fmaf_rn(wk, v.x, a0);
        a1 = __fmaf_rn(wk, v.y, a1);
        a2 = __fmaf_rn(wk, v.z, a2);
        a3 = __fmaf_rn(wk, v.w, a3);
    }
    float2 *d = reinterpret_cast<float2 *>(Y + r * yp + c);
    d[0] = make_float2(a0, a1);
    d[1] = make_float2(a2, a3);
}

// y sums of two rows r, r + 1 (the products and sums of sep_y_quad, k
// ascending for each): every loaded row feeds both, with weights k and k - 1
__device__ __forceinline__ void sep_y_pair(const float *__restrict__ P, int pp,
                                           float *__restrict__ Y, int yp, int r, int c,
                                           const SepWeights &w)
{
    const float *p = P + r * pp + c;
    const int ry2 = 2 * w.ry;
    float4 v = *reinterpret_cast<const float4 *>(p);
    float wp = w.wy[0];
    float a0 = __fmaf_rn(wp, v.x, 0.0f), a1 = __fmaf_rn(wp, v.y, 0.0f);
    float a2 = __fmaf_rn(wp, v.z, 0.0f), a3 = __fmaf_rn(wp, v.w, 0.0f);
    float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f, b3 = 0.0f;
#pragma unroll 2
    for (int i = 1; i <= ry2; ++i) {  // row r + i: tap i of row r, tap i - 1 of row r + 1
        v = *reinterpret_cast<const float4 *>(p + i * pp);
        const float wc = w.wy[i];
        a0 = __fmaf_rn(wc, v.x, a0);
        a1 = __fmaf_rn(wc, v.y, a1);
        a2 = __fmaf_rn(wc, v.z, a2);
        a3 = __fmaf_rn(wc, v.w, a3);
        b0 = __fmaf_rn(wp, v.x, b0);
        b1 = __fmaf_rn(wp, v.y, b1);
        b2 = __fmaf_rn(wp, v.z, b2);
        b3 = __fmaf_rn(wp, v.w, b3);
        wp = wc;
    }
    v = *reinterpret_cast<const float4 *>(p + (ry2 + 1) * pp);  // tap 2 ry of row r + 1
    b0 = __fmaf_rn(wp, v.x, b0);
    b1 = __fmaf_rn(wp, v.y, b1);
    b2 = __fmaf_rn(wp, v.z, b2);
    b3 = __fmaf_rn(wp, v.w, b3);
    float2 *d = reinterpret_cast<float2 *>(Y + r * yp + c);
    d[0] = make_float2(a0, a1);
    d[1] = make_float2(a2, a3);
    d = reinterpret_cast<float2 *>(Y + (r + 1) * yp + c);
    d[0] = make_float2(b0, b1);
    d[1] = make_float2(b2, b3);
}

// x sums of the thread's quad: a_j = sum_k wx[k] row[j + k], k ascending;
// row points at the first tap of voxel 0 (2 rx + 4 floats are read)
__device__ __forceinline__ void sep_x_quad(const float *__restrict__ row, const SepWeights &w,
                                           float (&a)[4])
{
    float v0 = row[0], v1 = row[1], v2 = row[2];
    a[0] = a[1] = a[2] = a[3] = 0.0f;
#pragma unroll 4
    for (int k = 0; k <= 2 * w.rx; ++k) {
        const float v3 = row[k + 3];
        const float wk = w.wx[k];
        a[0] = __fmaf_rn(wk, v0, a[0]);
        a[1] = __fmaf_rn(wk, v1, a[1]);
        a[2] = __fmaf_rn(wk, v2, a[2]);
        a[3] = __fmaf_rn(wk, v3, a[3]);
        v0 = v1;
        v1 = v2;
        v2 = v3;
    }
}

// The z window of the thread's quad: the xy sums of the last planes.  Small
// windows live in registers (shifted by one per plane); from kSepSmemRingRz
// on, in shared memory, one float4 per plane and thread in slots taken
// modulo 2 RZ + 1, so that registers stay few.  step() takes plane zi's sums
// and hands each output plane zo >= zs that is complete to put(zo, sums);
// every output sums its planes oldest first.
constexpr int kSepSmemRingRz = 3;

template <int RZ, bool SMEM = (RZ >= kSepSmemRingRz)>
struct SepRing;

template <int RZ>
struct SepRing<RZ, false> {
    float v[2 * RZ + 1][4];
    __device__ __forceinline__ SepRing(float4 *, int)
    {
#pragma unroll
        for (int m = 0; m < 2 * RZ + 1; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[m][j] = 0.0f;
    }
    template <class Put>
    __device__ __forceinline__ void step(int zi, int zs, int, const float (&c)[4],
                                         const SepWeights &w, Put &&put)
    {
#pragma unroll
        for (int m = 0; m < 2 * RZ; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[m][j] = v[m + 1][j];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            v[2 * RZ][j] = c[j];
        const int zo = zi - RZ;
        if (zo < zs)
            return;
        float s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s[j] = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RZ; ++k)
                s[j] = __fmaf_rn(w.wz[k], v[k][j], s[j]);
        }
        put(zo, s);
    }
};

// Output planes leave in pairs (zo - 1, zo), formed before plane zi = zo + RZ
// is stored: one pass over the 2 RZ + 1 stored planes zi - 2 RZ - 1 .. zi - 1
// and the new plane's sums in registers serves both, half the loads of two
// single sums.  A chunk with an odd number of outputs ends with a single one.
template <int RZ>
struct SepRing<RZ, true> {
    static constexpr int W = 2 * RZ + 1;
    float4 *base;  // slot m of this thread: base[m * stride]
    int stride;
    __device__ __forceinline__ SepRing(float4 *ring, int nthreads) : base(ring), stride(nthreads)
    {
    }
    template <class Put>
    __device__ __forceinline__ void step(int zi, int zs, int ze, const float (&c)[4],
                                         const SepWeights &w, Put &&put)
    {
        const int zo = zi - RZ, q = zo - zs;
        if (q >= 0 && ((q & 1) || zo == ze - 1)) {
            const bool pair = (q & 1) != 0;  // the same for the whole CTA
            float a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            int m = (zi - 2 * RZ - 1 + W) % W;  // plane zo - 1 - RZ >= -RZ - 1
            if (pair) {  // tap 0 of zo - 1
                const float4 v = base[m * stride];
                const float wk = w.wz[0];
                a[0] = __fmaf_rn(wk, v.x, a[0]);
                a[1] = __fmaf_rn(wk, v.y, a[1]);
                a[2] = __fmaf_rn(wk, v.z, a[2]);
                a[3] = __fmaf_rn(wk, v.w, a[3]);
            }
#pragma unroll
            for (int i = 1; i <= 2 * RZ; ++i) {  // plane zo - 1 - RZ + i
                m = m + 1 == W ? 0 : m + 1;
                const float4 v = base[m * stride];
                if (pair) {  // tap i of zo - 1
                    const float wa = w.wz[i];
                    a[0] = __fmaf_rn(wa, v.x, a[0]);
                    a[1] = __fmaf_rn(wa, v.y, a[1]);
                    a[2] = __fmaf_rn(wa, v.z, a[2]);
                    a[3] = __fmaf_rn(wa, v.w, a[3]);
                }
                const float wb = w.wz[i - 1];  // tap i - 1 of zo
                b[0] = __fmaf_rn(wb, v.x, b[0]);
                b[1] = __fmaf_rn(wb, v.y, b[1]);
                b[2] = __fmaf_rn(wb, v.z, b[2]);
                b[3] = __fmaf_rn(wb, v.w, b[3]);
            }
            const float wl = w.wz[2 * RZ];  // tap 2 RZ of zo: plane zi
#pragma unroll
            for (int j = 0; j < 4; ++j)
                b[j] = __fmaf_rn(wl, c[j], b[j]);
            if (pair)
                put(zo - 1, a);
            put(zo, b);
        }
        base[((zi + W) % W) * stride] = make_float4(c[0], c[1], c[2], c[3]);  // zi >= -RZ
    }
};

// bytes of shared memory the ring of one CTA of nthreads consumers takes
__host__ __device__ constexpr size_t sep_ring_bytes(int rz, int nthreads)
{
    return rz >= kSepSmemRingRz ? static_cast<size_t>(2 * rz + 1) * nthreads * 16 : 0;
}

__device__ __forceinline__ void sep_norm(const float (&sum)[4], const float (&inv_xy)[4],
                                         float inv_z, float (&o)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j)
        o[j] = __fmul_rn(__fmul_rn(sum[j], inv_xy[j]), inv_z);
}

// Plane geometry of both passes: P = the raw plane, SH = 16 + 2 ry rows of
// SW = 64 + 2 hx floats (hx = rx rounded up to a multiple of 4), column 0
// at x = x0 - hx, row 0 at y = y0 - ry, zero outside the cube; Y = its y
// sums, 16 rows of YP = SW + 2 floats (the odd pair of floats puts the two
// rows a warp reads in the x pass on different banks).
__host__ __device__ constexpr int sep_hx(int rx) { return (rx + 3) / 4 * 4; }
__host__ __device__ constexpr int sep_yp(int sw) { return sw + 2; }

template <int RZ>
__global__ void __launch_bounds__(kSmThreads, 1)
    smooth_sep(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz,
               int tiles_x, int tiles_y, int zc, const __grid_constant__ SepWeights w, int *err)
{
    extern __shared__ float sm[];
    const int rx = w.rx, ry = w.ry, hx = sep_hx(rx);
    const int SW = SX + 2 * hx, SH = SY + 2 * ry, YP = sep_yp(SW);
    float *P = sm;             // SH x SW raw plane
    float *Y = sm + SH * SW;   // SY x YP y sums
    // z ring (large windows): after Y, 16-byte aligned
    float4 *zr = reinterpret_cast<float4 *>(sm + ((SH * SW + SY * YP + 3) & ~3));

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

    float inv_xy[4];
    sep_inv_xy(w, xq, yr, nx, ny, inv_xy);
    const float inv_zf = sep_inv_z_full<RZ>(w);
    SepRing<RZ> ring(zr + tid, kSmThreads);
    const int nhq = 16 * (hx / 2);  // halo y tasks: 16 rows x hx/2 quads
    const bool x_ok =
        check_range(err, ty * YP + (hx - rx) + 4 * qx + 2 * rx + 3, 0, SY * YP, kChkSmoothSmem);

    for (int zi = zs - RZ; zi < ze + RZ; ++zi) {
        // ---- 1: the raw plane zi (tile + halo), zero outside the cube
        const bool zin = zi >= 0 && zi < nz;
        const float *src = in + static_cast<int64_t>(zi) * nx * ny;
        for (int r = warp; r < SH; r += kSmThreads / 32) {
            const int gy = y0 - ry + r;
            const bool yin = zin && gy >= 0 && gy < ny;
            for (int c = lane; c < SW; c += 32) {
                const int gx = x0 - hx + c;
                P[r * SW + c] = (yin && gx >= 0 && gx < nx)
                                    ? __ldg(src + static_cast<int64_t>(gy) * nx + gx)
                                    : 0.0f;
            }
        }
        __syncthreads();
        // ---- 2: y sums of the tile's rows over every column of the plane,
        // by row pairs: threads 0-127 the 8 x 16 under the tile, 128-255
        // the x halo's 8 x hx/2
        if (tid < kSmThreads / 2) {
            const int r = 2 * (tid >> 4), c = hx + 4 * qx;
            if (check_range(err, (r + 1 + 2 * ry) * SW + c + 3, 0, SH * SW, kChkSmoothSmem))
                sep_y_pair(P, SW, Y, YP, r, c, w);
        } else {
            for (int h = tid - kSmThreads / 2; h < nhq / 2; h += kSmThreads / 2) {
                const int r = 2 * (h & 7), hq = h >> 3;  // hq < hx/4: left, else right
                const int c = 4 * hq + (hq < hx / 4 ? 0 : SX);
                if (check_range(err, (r + 1 + 2 * ry) * SW + c + 3, 0, SH * SW, kChkSmoothSmem))
                    sep_y_pair(P, SW, Y, YP, r, c, w);
            }
        }
        __syncthreads();
        // ---- 3: x sums of the thread's quad, into the z ring
        float c4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (x_ok)
            sep_x_quad(Y + ty * YP + (hx - rx) + 4 * qx, w, c4);
        // ---- 4: z sums of the output planes now complete; normalise, store
        ring.step(zi, zs, ze, c4, w, [&](int zo, const float (&sz)[4]) {
            if (yr >= ny)
                return;
            float o[4];
            sep_norm(sz, inv_xy, sep_inv_z<RZ>(w, zo, nz, inv_zf), o);
            float *dst = out + (static_cast<int64_t>(zo) * ny + yr) * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (xq + j < nx &&
                    check_range(err, dst + xq + j - out, 0, static_cast<int64_t>(nz) * ny * nx,
                                kChkSmoothStore))
                    dst[xq + j] = o[j];
        });
        // the next iteration rewrites P right away: every read of P happened
        // before the second barrier above; it rewrites Y only after its first
        // barrier, which follows these reads of Y
    }
}

// The separable pass with its planes streamed by TMA (rows of a multiple of
// 16 bytes) into a ring of kSmSlots slots, kSmSlots - 1 planes ahead.  All
// nine warps take the y sums of a slot into a double-buffered Y plane: warps
// 0-7 the 16 x 16 quads under the tile, warp 8 (whose lane 0 also issues the
// loads) the 16 x hx/2 quads of the x halo, one per lane when hx = 4.  They
// release the slot, meet at one named barrier, and warps 0-7 take the x sums
// and keep the z window in registers: the same products and sums, in the
// same order, as smooth_sep.  Every mbarrier wait is bounded (kWaitLimitNs);
// a thread whose wait expires records the error and keeps stepping without
// waiting again (lane 0 of warp 8 stops loading), so every warp reaches every
// named barrier and the CTA ends.
constexpr int kSmSlots = 3;
constexpr int kSmTmaThreads = kSmThreads + 32;

__device__ __forceinline__ void all_warps_barrier()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kSmTmaThreads) : "memory");
}

// Register budget: 3 CTAs per SM while the z ring is in registers (RZ <= 2),
// else 2 (shared memory allows no more)
template <int RZ>
__global__ void __launch_bounds__(kSmTmaThreads, RZ <= 4 ? 3 : 2)
    smooth_sep_tma(const __grid_constant__ CUtensorMap tmap, float *__restrict__ out, int nx,
                   int ny, int nz, int tiles_x, int tiles_y, int zc, int hx,
                   const __grid_constant__ SepWeights w, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((128u - (base & 127u)) & 127u);
    const int rx = w.rx, ry = w.ry;
    const int SW = SX + 2 * hx, SH = SY + 2 * ry, YP = sep_yp(SW);  // slot: SH rows of SW floats
    const uint32_t slot_bytes = static_cast<uint32_t>(SW * SH) * 4u;
    const uint32_t slot_stride = (slot_bytes + 127u) & ~127u;
    float *Yb2 = reinterpret_cast<float *>(smem + kSmSlots * slot_stride);  // 2 x SY x YP
    float4 *zr = reinterpret_cast<float4 *>(Yb2 + ((2 * SY * YP + 3) & ~3));  // z ring (large RZ)
    uint64_t *full = reinterpret_cast<uint64_t *>(
        reinterpret_cast<unsigned char *>(zr) + sep_ring_bytes(RZ, kSmThreads));
    uint64_t *empty = full + kSmSlots;

    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int x0 = bx * SX, y0 = by * SY;
    const int zs = bz * zc, ze = min(zs + zc, nz);
    const int zlo = max(zs - RZ, 0), zhi = min(ze + RZ, nz) - 1;  // planes loaded
    const int np = zhi - zlo + 1;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const bool loader = tid == kSmThreads;  // lane 0 of warp 8
    if (tid == 0) {
        for (int i = 0; i < kSmSlots; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kSmTmaThreads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    bool waiting = true;  // false after an expired wait: no more waits (and no more loads)
    // plane j of the chunk into slot j % kSmSlots, once every warp released
    // its previous plane (j - kSmSlots)
    auto load = [&](int j) {
        const int slot = j % kSmSlots, use = j / kSmSlots;
        if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u, err, kErrWaitEmpty)) {
            waiting = false;
            return;
        }
        mbar_arrive_expect_tx(&full[slot], slot_bytes);
        tma_load_3d(smem + slot * slot_stride, &tmap, x0 - hx, y0 - ry, zlo + j, &full[slot]);
    };
    if (loader)
        for (int j = 0; j < kSmSlots - 1 && j < np; ++j)
            load(j);

    // consumers: thread (qx, ty) owns 4 voxels of row ty
    const int qx = tid & 15, ty = (tid >> 4) & 15;
    const int xq = x0 + 4 * qx, yr = y0 + ty;
    const bool cons = warp < kSmThreads / 32;
    float inv_xy[4] = {1.0f, 1.0f, 1.0f, 1.0f};
    if (cons)
        sep_inv_xy(w, xq, yr, nx, ny, inv_xy);
    const float inv_zf = sep_inv_z_full<RZ>(w);
    SepRing<RZ> ring(zr + (tid & (kSmThreads - 1)), kSmThreads);
    const int nhq = 16 * (hx / 2);  // halo y tasks: 16 rows x hx/2 quads
    const bool x_ok =
        check_range(err, ty * YP + (hx - rx) + 4 * qx + 2 * rx + 3, 0, SY * YP, kChkSmoothSmem);

    for (int zi = zs - RZ; zi < ze + RZ; ++zi) {
        const bool have = zi >= zlo && zi <= zhi;  // the same for the whole CTA
        float *Y = Yb2 + (zi & 1) * SY * YP;
        if (have) {
            const int j = zi - zlo, slot = j % kSmSlots;
            if (loader && waiting && j + kSmSlots - 1 < np)
                load(j + kSmSlots - 1);
            if (waiting && !mbar_wait(&full[slot], (j / kSmSlots) & 1u, err, kErrWaitFull))
                waiting = false;
            const float *S = reinterpret_cast<const float *>(smem + slot * slot_stride);
            // by row pairs: warps 0-3 the 8 x 16 under the tile, warp 8 the
            // x halo's 8 x hx/2 (warps 4-7 have none)
            if (tid < kSmThreads / 2) {
                const int r = 2 * (tid >> 4), c = hx + 4 * qx;
                if (check_range(err, (r + 1 + 2 * ry) * SW + c + 3, 0, SH * SW, kChkSmoothSmem))
                    sep_y_pair(S, SW, Y, YP, r, c, w);
            } else if (!cons) {
                for (int h = lane; h < nhq / 2; h += 32) {
                    const int r = 2 * (h & 7), hq = h >> 3;  // hq < hx/4: left, else right
                    const int c = 4 * hq + (hq < hx / 4 ? 0 : SX);
                    if (check_range(err, (r + 1 + 2 * ry) * SW + c + 3, 0, SH * SW,
                                    kChkSmoothSmem))
                        sep_y_pair(S, SW, Y, YP, r, c, w);
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[slot]);
        }
        // Y is complete; the other buffer, written next plane, was last read
        // before this barrier
        all_warps_barrier();
        if (!cons)
            continue;
        float c4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (have && x_ok)
            sep_x_quad(Y + ty * YP + (hx - rx) + 4 * qx, w, c4);
        ring.step(zi, zs, ze, c4, w, [&](int zo, const float (&sz)[4]) {
            if (yr >= ny || xq >= nx)
                return;
            float o[4];
            sep_norm(sz, inv_xy, sep_inv_z<RZ>(w, zo, nz, inv_zf), o);
            // nx % 4 == 0 and xq % 4 == 0: the quad is inside the row
            const int64_t oi = (static_cast<int64_t>(zo) * ny + yr) * nx + xq;
            if (check_range(err, oi, 0, static_cast<int64_t>(nz) * ny * nx - 3, kChkSmoothStore))
                *reinterpret_cast<float4 *>(out + oi) = make_float4(o[0], o[1], o[2], o[3]);
        });
    }
}

template <int RZ>
cudaError_t sep_launch(const float *in, float *out, int nx, int ny, int nz, const SepWeights &w,
                       int zc, int *err, cudaStream_t stream)
{
    const int tiles_x = (nx + SX - 1) / SX, tiles_y = (ny + SY - 1) / SY;
    const int tiles_z = (nz + zc - 1) / zc;
    const int sw = SX + 2 * sep_hx(w.rx);
    const size_t smem =
        (static_cast<size_t>((SY + 2 * w.ry) * sw + SY * sep_yp(sw) + 3) & ~size_t(3)) *
            sizeof(float) +
        sep_ring_bytes(RZ, kSmThreads);
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
    const size_t smem = smooth_tma_smem(w.ry, hx, RZ);
    cudaError_t e = cudaFuncSetAttribute(smooth_sep_tma<RZ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess)  // several CTAs per SM: all of the carveout as shared memory
        e = cudaFuncSetAttribute(smooth_sep_tma<RZ>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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

size_t smooth_tma_smem(int ry, int hx, int rz)
{
    const size_t slot = (static_cast<size_t>(SX + 2 * hx) * (SY + 2 * ry) * 4 + 127) / 128 * 128;
    const size_t ybuf =
        ((2 * static_cast<size_t>(SY) * sep_yp(SX + 2 * hx) + 3) & ~size_t(3)) * sizeof(float);
    return kSmSlots * slot + ybuf + sep_ring_bytes(rz, kSmThreads) +
           2 * kSmSlots * sizeof(uint64_t) + 128;
}

void smooth_tma_box(int rx, int ry, int *box_w, int *box_h, int *hx)
{
    *hx = sep_hx(rx);  // x halo: >= rx, a multiple of 4 floats (16-byte TMA x)
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
