// Two explicit per-face Perona-Malik iterations per pass (temporal blocking;
// arXiv:1609.03782 Sec. 3.3, the per-face discretisation of eq. "perona"
// with the gradient conductance, evaluated twice per HBM pass), from an
// input in format SI to an output in format SO (float32 or 2-byte storage).
// A pass reads the cube once and writes it once for two iterations.  Every
// value is the canonical per-face arithmetic (afd_math.cuh) and the
// intermediate iteration stays float32, so a pass equals dequantise -> two
// float32 iterations -> quantise, bit for bit the temporally blocked kernel
// of the same depth (pm_tb.cuh), and with float32 storage two
// single-iteration passes.  A chain SI -> float32 -> ... -> float32 -> SO of
// these passes is therefore T = 2 x (links) float32 iterations between one
// dequantisation and one quantisation: the temporally blocked kernel of
// depth T, bit for bit.
//
// Design (sm_103a), per persistent CTA (TY = kWide2TY output rows):
//   * The last warp is the TMA producer: for a 128 x TY output tile and a
//     z-chunk it loads, plane by plane, the 144 x (TY + 4) box around the
//     tile (a 2-voxel halo in y, a 16-byte aligned 8-voxel halo in x) in the
//     storage format into a ring of slots.
//   * Stage 1 (the first kWide2S1Warps warps): the first iteration over the
//     tile grown by one voxel on each side (17 x (TY/2 + 1) blocks of 8 x 2
//     voxels from x0-4, y0-1), for the chunk's planes and one plane below and
//     above; each result plane goes to a ring of float32 planes in shared
//     memory.  With 2-byte storage its rows start 8 bytes into a 16-byte
//     word, so they are read as two 8-byte loads.
//   * Stage 2 (the next kWide2S2Warps warps): the second iteration over the
//     tile from those planes, rounded to the output format and stored to
//     global memory.
//   * The stages hand planes over through mbarriers (full / empty per ring
//     plane), so neither waits for the other except on the data itself.
//   * Zero flux at the cube's faces as in the single-iteration kernels:
//     neighbours across a face point at the own voxel; blocks of the grown
//     tile that straddle an x face give their outside voxels the nearest
//     inside value; outside rows take the inside row's values.
// Requirements checked by the host: nx a multiple of 8, 16-byte aligned
// pointers.  Every mbarrier wait is bounded (afd_ptx.cuh).
#include "afd_internal.h"
#include "afd_ptx.cuh"
#include "afd_check.cuh"
#include "afd_store.cuh"
#include "pm_block.cuh"

namespace afd {
namespace {

constexpr int TX2 = kWide2TX;               // 128
constexpr int TY2 = kWide2TY;               // 24
constexpr int S1W = kWide2S1Warps;          // stage-1 warps
constexpr int S2W = kWide2S2Warps;          // stage-2 warps
constexpr int S1T = S1W * 32, S2T = S2W * 32;
constexpr int NQ1 = TX2 / 8 + 1;            // 17 stage-1 column blocks (from x0 - 4)
constexpr int RP1 = TY2 / 2 + 1;            // 9 stage-1 row pairs (from y0 - 1)
static_assert(NQ1 * RP1 <= S1T && (TX2 / 8) * (TY2 / 2) == S2T, "thread mapping");
constexpr int IN_W = TX2 + 16;              // input box: x0 - 8 .. x0 + TX2 + 8
constexpr int IN_H = TY2 + 4;               // y0 - 2 .. y0 + TY2 + 2
template <int S>
struct In {
    static constexpr int ES = static_cast<int>(sizeof(typename Store<S>::T));
    static constexpr uint32_t BOX = IN_W * IN_H * ES;  // bytes of one TMA box
    static constexpr int SLOT = (BOX + 127) / 128 * 128;
    static_assert((IN_W * ES) % 16 == 0, "16-byte rows");
};
constexpr uint32_t NIN = kWide2Slots;       // input ring
constexpr int P1_W = TX2 + 8;               // stage-1 plane: x0 - 4 .. x0 + TX2 + 4
constexpr int P1_H = TY2 + 2;               // y0 - 1 .. y0 + TY2 + 1
constexpr int P1_SLOT = (P1_W * P1_H * 4 + 127) / 128 * 128;
constexpr uint32_t NP1 = kWide2P1;          // stage-1 plane ring
static_assert((NIN & (NIN - 1)) == 0 && (NP1 & (NP1 - 1)) == 0, "ring sizes");
static_assert((P1_W * 4) % 16 == 0, "16-byte rows");

// A ring of shared-memory planes guarded by full / empty mbarriers.
struct PRing {
    const unsigned char *base;
    uint32_t full, empty;  // shared-memory addresses of the barrier arrays
    uint32_t n, bytes;     // planes, bytes per plane
    int *err;
    __device__ __forceinline__ const unsigned char *slot(uint32_t r) const
    {
        return base + (r & (n - 1)) * bytes;
    }
    __device__ __forceinline__ bool wait_full(uint32_t r) const
    {
        return mbar_wait_sleep(full + (r & (n - 1)) * 8, (r / n) & 1u, err, kErrWaitFull);
    }
    __device__ __forceinline__ bool wait_empty(uint32_t r) const
    {
        // the use before this one must have been released (no wait the first time)
        return r < n || mbar_wait_sleep(empty + (r & (n - 1)) * 8, ((r / n) - 1) & 1u, err,
                                        kErrWaitEmpty);
    }
    __device__ __forceinline__ void arrive_full(uint32_t r) const
    {
        mbar_arrive_u32(full + (r & (n - 1)) * 8);
    }
    __device__ __forceinline__ void release(uint32_t r) const
    {
        mbar_arrive_u32(empty + (r & (n - 1)) * 8);
    }
};

struct Tile2 {
    int x0, y0, z0, z1;
};

__device__ __forceinline__ Tile2 decode2(int t, int tiles_x, int txy, const ZLevels &lv)
{
    const int tz = t / txy;
    const int r = t - tz * txy;
    const int ty = r / tiles_x;
    Tile2 w;
    w.x0 = (r - ty * tiles_x) * TX2;
    w.y0 = ty * TY2;
    zchunk(lv, tz, w.z0, w.z1);
    return w;
}

// Offsets of a block in a plane of es-byte elements with row pitch pitch_b
// bytes whose first row is y_first and whose first column is x_first;
// zero-flux substitutions at the cube's faces (rows outside the cube take the
// inside row's values).
__device__ __forceinline__ Offs block_offs(int x, int ya, int nx, int ny, int x_first,
                                           int y_first, int pitch_b, int es)
{
    const int yb = ya + 1;
    Offs o;
    o.r0 = (ya - y_first) * pitch_b + (x - x_first) * es;
    o.r1 = (yb < ny) ? o.r0 + pitch_b : o.r0;  // row 1 outside: zero flux to row 0
    if (ya < 0)
        o.r0 = o.r1;                           // row 0 outside: zero flux to row 1
    o.dn = (ya <= 0) ? o.r0 : o.r0 - pitch_b;
    o.up = (yb + 1 >= ny) ? o.r1 : o.r1 + pitch_b;
    o.xl0 = (x <= 0) ? o.r0 : o.r0 - es;
    o.xl1 = (x <= 0) ? o.r1 : o.r1 - es;
    o.xr0 = (x + 8 >= nx) ? o.r0 + 7 * es : o.r0 + 8 * es;
    o.xr1 = (x + 8 >= nx) ? o.r1 + 7 * es : o.r1 + 8 * es;
    return o;
}

// Checked builds: every read of a block (rows of 8 es-byte elements, the x
// neighbours) lies inside a plane of `box` bytes.  Always true in release
// builds.
__device__ __forceinline__ bool offs_ok(const Offs &o, int box, int es, int *err)
{
    const int row = box - 8 * es + 1;
    return check_range(err, o.r0, 0, row, kChkStreamSlot) &&
           check_range(err, o.r1, 0, row, kChkStreamSlot) &&
           check_range(err, o.dn, 0, row, kChkStreamSlot) &&
           check_range(err, o.up, 0, row, kChkStreamSlot) &&
           check_range(err, o.xl0, 0, box - es + 1, kChkStreamSlot) &&
           check_range(err, o.xl1, 0, box - es + 1, kChkStreamSlot) &&
           check_range(err, o.xr0, 0, box - es + 1, kChkStreamSlot) &&
           check_range(err, o.xr1, 0, box - es + 1, kChkStreamSlot);
}

// A block that is read in place of one whose offsets failed offs_ok: the
// start of the plane's third row (16-byte aligned), its results unused.
__device__ __forceinline__ Offs safe_offs(int pitch_b)
{
    const int a = 2 * pitch_b;
    return Offs{a, a, a, a, a, a, a, a};
}

// The two rows of a block at ring entry r, as packed pairs, clamped at the
// cube's x faces (positions before a and from b on take the nearest inside
// value) when the block straddles one.
template <int S, bool A8>
__device__ __forceinline__ void rows(const unsigned char *slot, const Offs &o, bool clamp, int a,
                                     int b, f2_t (&r0)[4], f2_t (&r1)[4])
{
    cvt8<S>(ld_raw8<S, A8>(slot + o.r0), r0);
    cvt8<S>(ld_raw8<S, A8>(slot + o.r1), r1);
    if (clamp) {
        clamp8_ab(r0, a, b);
        clamp8_ab(r1, a, b);
    }
}

// One plane of one stage: the update of the block's 16 voxels of plane z
// (ring entry r) from the plane's x and y neighbours, plane z+1 (entry r+1,
// own values at the top face) and the flux through plane z's lower faces.
// In: plane z (c0, c1), lower z-face flux (fb0, fb1).  Out: plane z+1
// (n0, n1), the flux between them (fa0, fa1) and the results (o0, o1).
// Releases entry r after its last read.  S, A8: the ring's element format
// and row alignment.
template <int S, int C, bool A8>
__device__ __forceinline__ bool stage_step(const PRing &ring, const Offs &o, const Kp &k,
                                           uint32_t r, bool has_next, bool clamp, int a, int b,
                                           const f2_t (&c0)[4], const f2_t (&c1)[4],
                                           const f2_t (&fb0)[4], const f2_t (&fb1)[4],
                                           f2_t (&n0)[4], f2_t (&n1)[4], f2_t (&fa0)[4],
                                           f2_t (&fa1)[4], f2_t (&o0)[4], f2_t (&o1)[4])
{
    f2_t s0[4], s1[4];
    xy_sums<S, C, A8>(ring.slot(r), o, k, c0, c1, s0, s1);
    if (has_next) {
        if (!ring.wait_full(r + 1))
            return false;
        rows<S, A8>(ring.slot(r + 1), o, clamp, a, b, n0, n1);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            n0[i] = c0[i];
            n1[i] = c1[i];
        }
    }
    ring.release(r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        fa0[i] = face_flux2<C>(f2_sub(n0[i], c0[i]), k.az, k.bz, k.z);
        fa1[i] = face_flux2<C>(f2_sub(n1[i], c1[i]), k.az, k.bz, k.z);
        // I' = I + ((s_x + s_y) + s_z)
        o0[i] = f2_add(c0[i], f2_add(s0[i], f2_sub(fa0[i], fb0[i])));
        o1[i] = f2_add(c1[i], f2_add(s1[i], f2_sub(fa1[i], fb1[i])));
    }
    return true;
}

__device__ __forceinline__ void sts8x2(unsigned char *p, int pitch_b, const f2_t (&v0)[4],
                                       const f2_t (&v1)[4], bool on)
{
    if (!on)
        return;
    uint4 *q0 = reinterpret_cast<uint4 *>(p);
    uint4 *q1 = reinterpret_cast<uint4 *>(p + pitch_b);
    unsigned w[8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm("mov.b64 {%0, %1}, %2;" : "=r"(w[2 * i]), "=r"(w[2 * i + 1]) : "l"(v0[i]));
    q0[0] = make_uint4(w[0], w[1], w[2], w[3]);
    q0[1] = make_uint4(w[4], w[5], w[6], w[7]);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm("mov.b64 {%0, %1}, %2;" : "=r"(w[2 * i]), "=r"(w[2 * i + 1]) : "l"(v1[i]));
    q1[0] = make_uint4(w[0], w[1], w[2], w[3]);
    q1[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

template <int S, int SO, int C>
__global__ void __maxnreg__(kWide2MaxRegs)
    pm_step_wide2(const __grid_constant__ CUtensorMap tmap,
                  typename Store<SO>::T *__restrict__ out, int nx, int ny, int nz, int tiles_x,
                  int txy, const __grid_constant__ ZLevels lv, int ntiles,
                  unsigned long long *ctr, unsigned long long base, Coef kc, int *err)
{
    typedef In<S> IS;
    grid_dep_launch_dependents();  // the next pass may take SMs as this one frees them
    extern __shared__ unsigned char smem_raw[];
    const uint32_t sb = smem_u32(smem_raw);
    unsigned char *in_slots = smem_raw + ((128u - (sb & 127u)) & 127u);
    unsigned char *p1_slots = in_slots + NIN * IS::SLOT;
    uint64_t *in_full = reinterpret_cast<uint64_t *>(p1_slots + NP1 * P1_SLOT);
    uint64_t *in_empty = in_full + NIN;
    uint64_t *p1_full = in_empty + NIN;
    uint64_t *p1_empty = p1_full + NP1;
    int *tile_of = reinterpret_cast<int *>(p1_empty + NP1);  // per input slot
    int *p1_tile = tile_of + NIN;                             // per stage-1 plane

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < NIN; ++i) {
            mbar_init(&in_full[i], 1);
            mbar_init(&in_empty[i], S1T);
        }
        for (uint32_t i = 0; i < NP1; ++i) {
            mbar_init(&p1_full[i], S1T);
            mbar_init(&p1_empty[i], S2T);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const PRing in{in_slots, smem_u32(in_full), smem_u32(in_empty), NIN, IS::SLOT, err};
    const PRing p1{p1_slots, smem_u32(p1_full), smem_u32(p1_empty), NP1, P1_SLOT, err};

    if (warp == S1W + S2W) {
        // ---------------- producer ----------------
        if (lane == 0) {
            grid_dep_wait();  // the previous pass's writes are visible from here on
            uint32_t kk = 0;
            int64_t t = blockIdx.x;
            for (;;) {
                const bool more = t >= 0 && t < ntiles;
                int np = 1, zlo0 = 0;
                Tile2 w{0, 0, 0, 0};
                if (more) {
                    w = decode2(static_cast<int>(t), tiles_x, txy, lv);
                    const int zlo1 = max(w.z0 - 1, 0), zhi1 = min(w.z1, nz - 1);
                    zlo0 = max(zlo1 - 1, 0);
                    np = min(zhi1 + 1, nz - 1) - zlo0 + 1;
                }
                for (int j = 0; j < np; ++j, ++kk) {
                    const uint32_t slot = kk & (NIN - 1);
                    if (!in.wait_empty(kk))
                        return;
                    if (j == 0)
                        tile_of[slot] = more ? static_cast<int>(t) : -1;
                    if (!more) {
                        mbar_arrive(&in_full[slot]);  // the end mark: no data
                        break;
                    }
                    mbar_arrive_expect_tx(&in_full[slot], IS::BOX);
                    tma_load_3d(in_slots + slot * IS::SLOT, &tmap, w.x0 - 8, w.y0 - 2, zlo0 + j,
                                &in_full[slot]);
                }
                if (!more)
                    break;
                t = static_cast<int64_t>(gridDim.x) +
                    static_cast<int64_t>(atomicAdd(ctr, 1ull) - base);
            }
        }
        return;
    }

    if (warp < S1W) {
        // ---------------- stage 1: the first iteration ----------------
        const int t1 = threadIdx.x;
        const bool has_block = t1 < NQ1 * RP1;
        const int kq = has_block ? t1 % NQ1 : 0, jr = has_block ? t1 / NQ1 : 0;
        uint32_t kk = 0, k1 = 0;
        for (;;) {
            if (!in.wait_full(kk))
                return;
            const int t = tile_of[kk & (NIN - 1)];
            if (t < 0) {
                // end mark for stage 2: a stage-1 plane with tile -1
                if (!p1.wait_empty(k1))
                    return;
                if (t1 == 0)
                    p1_tile[k1 & (NP1 - 1)] = -1;
                p1.arrive_full(k1);
                break;
            }
            const Tile2 w = decode2(t, tiles_x, txy, lv);
            const int zlo1 = max(w.z0 - 1, 0), zhi1 = min(w.z1, nz - 1);
            const int zlo0 = max(zlo1 - 1, 0), zhi0 = min(zhi1 + 1, nz - 1);
            const int x = w.x0 - 4 + 8 * kq, ya = w.y0 - 1 + 2 * jr;
            Offs o = block_offs(x, ya, nx, ny, w.x0 - 8, w.y0 - 2, IN_W * IS::ES, IS::ES);
            const int a = max(0, -x), b = min(8, nx - x);
            const bool clamp = (a > 0 || b < 8) && a < b;
            const Kp k = make_kp<C>(kc);
            const int p1off = (2 * jr * P1_W + 8 * kq) * 4;  // the block in a stage-1 plane
            // checked builds: reads inside the input box, both stores inside
            // the stage-1 plane (else a safe block is read and nothing stored)
            bool store_on = has_block;
            if (!(offs_ok(o, IN_W * IN_H * IS::ES, IS::ES, err) &&
                  check_range(err, p1off, 0, P1_W * P1_H * 4 - P1_W * 4 - 32 + 1,
                              kChkStreamSlot))) {
                o = safe_offs(IN_W * IS::ES);
                store_on = false;
            }
            const uint32_t kbase = kk;
            uint32_t r = kbase + static_cast<uint32_t>(zlo1 - zlo0);
            f2_t c0[4], c1[4], fb0[4], fb1[4];
            if (zlo1 > 0) {
                f2_t q0[4], q1[4];
                rows<S, true>(in.slot(kbase), o, clamp, a, b, q0, q1);
                if (!in.wait_full(r))
                    return;
                rows<S, true>(in.slot(r), o, clamp, a, b, c0, c1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    fb0[i] = face_flux2<C>(f2_sub(c0[i], q0[i]), k.az, k.bz, k.z);
                    fb1[i] = face_flux2<C>(f2_sub(c1[i], q1[i]), k.az, k.bz, k.z);
                }
                in.release(kbase);
            } else {
                rows<S, true>(in.slot(r), o, clamp, a, b, c0, c1);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    fb0[i] = fb1[i] = 0ull;  // +0: the zero flux at z = 0
            }
            f2_t n0[4], n1[4], fa0[4], fa1[4], o0[4], o1[4];
            int p = zlo1;
            // one stage-1 plane: compute it, then hand it to stage 2
#define S1_PLANE(C0, C1, FB0, FB1, N0, N1, FA0, FA1)                                         \
    {                                                                                          \
        if (!stage_step<S, C, true>(in, o, k, r, p + 1 < nz, clamp, a, b, C0, C1, FB0, FB1,   \
                                    N0, N1, FA0, FA1, o0, o1))                                 \
            return;                                                                            \
        if (!p1.wait_empty(k1))                                                                \
            return;                                                                            \
        if (p == zlo1 && t1 == 0)                                                              \
            p1_tile[k1 & (NP1 - 1)] = t;                                                       \
        sts8x2(const_cast<unsigned char *>(p1.slot(k1)) + p1off, P1_W * 4, o0, o1, store_on);  \
        p1.arrive_full(k1);                                                                    \
        ++k1;                                                                                  \
        ++r;                                                                                   \
        ++p;                                                                                   \
    }
            while (p + 1 <= zhi1) {
                S1_PLANE(c0, c1, fb0, fb1, n0, n1, fa0, fa1);
                S1_PLANE(n0, n1, fa0, fa1, c0, c1, fb0, fb1);
            }
            if (p <= zhi1)
                S1_PLANE(c0, c1, fb0, fb1, n0, n1, fa0, fa1);
#undef S1_PLANE
            if (zhi1 + 1 < nz)
                in.release(r);  // the input plane above the last stage-1 plane
            kk = kbase + static_cast<uint32_t>(zhi0 - zlo0 + 1);
        }
        return;
    }

    // ---------------- stage 2: the second iteration ----------------
    const int t2 = threadIdx.x - S1T;
    const int q = t2 % (TX2 / 8), rp = t2 / (TX2 / 8);
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    uint32_t k2 = 0;
    for (;;) {
        if (!p1.wait_full(k2))
            return;
        const int t = p1_tile[k2 & (NP1 - 1)];
        if (t < 0)
            break;
        const Tile2 w = decode2(t, tiles_x, txy, lv);
        const int zlo1 = max(w.z0 - 1, 0), zhi1 = min(w.z1, nz - 1);
        const int x = w.x0 + 8 * q, ya = w.y0 + 2 * rp, yb = ya + 1;
        Offs o = block_offs(x, ya, nx, ny, w.x0 - 4, w.y0 - 1, P1_W * 4, 4);
        const bool p1_ok = offs_ok(o, P1_W * P1_H * 4, 4, err);  // checked builds
        if (!p1_ok)
            o = safe_offs(P1_W * 4);
        const Kp k = make_kp<C>(kc);
        const bool tile_ok = check_range(err, w.z1, w.z0 + 1, static_cast<int64_t>(nz) + 1,
                                         kChkStreamTile) &&
                             check_range(err, w.x0, 0, nx, kChkStreamTile) &&
                             check_range(err, w.y0, 0, ny, kChkStreamTile);
        const bool act0 = tile_ok && p1_ok && x < nx && ya < ny;
        const bool act1 = tile_ok && p1_ok && x < nx && yb < ny;
        typename Store<SO>::T *po = out + (static_cast<int64_t>(w.z0) * ny + ya) * nx + x;
        const uint32_t kb2 = k2;
        uint32_t r = kb2 + static_cast<uint32_t>(w.z0 - zlo1);
        f2_t c0[4], c1[4], fb0[4], fb1[4];
        if (w.z0 > 0) {
            f2_t q0[4], q1[4];
            rows<STORE_F32, false>(p1.slot(kb2), o, false, 0, 8, q0, q1);
            if (!p1.wait_full(r))
                return;
            rows<STORE_F32, false>(p1.slot(r), o, false, 0, 8, c0, c1);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fb0[i] = face_flux2<C>(f2_sub(c0[i], q0[i]), k.az, k.bz, k.z);
                fb1[i] = face_flux2<C>(f2_sub(c1[i], q1[i]), k.az, k.bz, k.z);
            }
            p1.release(kb2);
        } else {
            rows<STORE_F32, false>(p1.slot(r), o, false, 0, 8, c0, c1);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                fb0[i] = fb1[i] = 0ull;
        }
        f2_t n0[4], n1[4], fa0[4], fa1[4], o0[4], o1[4];
        int z = w.z0;
#define S2_PLANE(C0, C1, FB0, FB1, N0, N1, FA0, FA1)                                          \
    {                                                                                          \
        if (!stage_step<STORE_F32, C, false>(p1, o, k, r, z + 1 < nz, false, 0, 8, C0, C1, FB0, \
                                             FB1, N0, N1, FA0, FA1, o0, o1))                   \
            return;                                                                            \
        stg8<SO>(po, o0,                                                                       \
                 act0 && check_range(err, po - out, 0, nz * plane - 7, kChkStreamStore));      \
        stg8<SO>(po + nx, o1,                                                                  \
                 act1 && check_range(err, po + nx - out, 0, nz * plane - 7, kChkStreamStore)); \
        po += plane;                                                                           \
        ++r;                                                                                   \
        ++z;                                                                                   \
    }
        while (z + 1 < w.z1) {
            S2_PLANE(c0, c1, fb0, fb1, n0, n1, fa0, fa1);
            S2_PLANE(n0, n1, fa0, fa1, c0, c1, fb0, fb1);
        }
        if (z < w.z1)
            S2_PLANE(c0, c1, fb0, fb1, n0, n1, fa0, fa1);
#undef S2_PLANE
        if (w.z1 < nz)
            p1.release(r);  // the stage-1 plane above the chunk
        k2 = kb2 + static_cast<uint32_t>(zhi1 - zlo1 + 1);
    }
}

template <int S>
size_t smem_bytes2()
{
    return static_cast<size_t>(NIN) * In<S>::SLOT + static_cast<size_t>(NP1) * P1_SLOT +
           2 * (NIN + NP1) * sizeof(uint64_t) + (NIN + NP1) * sizeof(int) + 128;
}

template <int S, int SO, int C>
cudaError_t wide2_launch(const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                         const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                         unsigned long long base, int *err, cudaStream_t stream)
{
    if (plan.ntiles > 0x7fffffff || plan.kdev)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(plan.grid));
    cfg.blockDim = dim3(kWide2Threads);
    cfg.dynamicSmemBytes = smem_bytes2<S>();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = plan.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, pm_step_wide2<S, SO, C>, tmap,
                              static_cast<typename Store<SO>::T *>(out), nx, ny, nz, plan.tiles_x,
                              plan.tiles_x * plan.tiles_y, plan.lv, static_cast<int>(plan.ntiles),
                              ctr, base, k, err);
}

template <int S, int SO>
cudaError_t prepare_pair()
{
    const int smem = static_cast<int>(smem_bytes2<S>());
    cudaError_t e = cudaFuncSetAttribute(pm_step_wide2<S, SO, COND_EXP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pm_step_wide2<S, SO, COND_RAT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <int S, int SO>
cudaError_t launch_pair(int cond, const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                        const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                        unsigned long long base, int *err, cudaStream_t stream)
{
    switch (cond) {
    case COND_EXP:
        return wide2_launch<S, SO, COND_EXP>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                             stream);
    case COND_RAT:
        return wide2_launch<S, SO, COND_RAT>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                             stream);
    default:
        return cudaErrorInvalidValue;  // the other conductance kinds have no depth-2 pass
    }
}

// A 2-byte format to and from float32, and to itself
template <int S>
cudaError_t prepare_s()
{
    cudaError_t e = prepare_pair<S, S>();
    if (e == cudaSuccess)
        e = prepare_pair<S, STORE_F32>();
    if (e == cudaSuccess)
        e = prepare_pair<STORE_F32, S>();
    return e;
}

template <int S>
cudaError_t launch_s(int SO, int cond, const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                     const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                     unsigned long long base, int *err, cudaStream_t stream)
{
    if (SO == S)
        return launch_pair<S, S>(cond, tmap, out, nx, ny, nz, k, plan, ctr, base, err, stream);
    if (SO == STORE_F32)
        return launch_pair<S, STORE_F32>(cond, tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                         stream);
    return cudaErrorInvalidValue;
}

template <int SO>
cudaError_t launch_from_f32(int cond, const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                            const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                            unsigned long long base, int *err, cudaStream_t stream)
{
    return launch_pair<STORE_F32, SO>(cond, tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                      stream);
}


}  // namespace

void pm_wide2_box(int *box_w, int *box_h)
{
    *box_w = IN_W;
    *box_h = IN_H;
}

cudaError_t pm_wide2_prepare()
{
    cudaError_t e = prepare_pair<STORE_F32, STORE_F32>();
    if (e == cudaSuccess)
        e = prepare_s<STORE_F16>();
    if (e == cudaSuccess)
        e = prepare_s<STORE_BF16>();
    if (e == cudaSuccess)
        e = prepare_s<STORE_I16>();
    return e;
}

cudaError_t pm_wide2_occupancy(int *blocks_per_sm)
{
    // float32 input slots are the largest: its occupancy bounds every pair's
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, pm_step_wide2<STORE_F32, STORE_F32, COND_RAT>, kWide2Threads,
        smem_bytes2<STORE_F32>());
}

cudaError_t launch_pm_wide2(int S, int SO, int cond, const CUtensorMap &tmap_in, void *out,
                            int nx, int ny, int nz, const Coef &k, const StreamPlan &plan,
                            unsigned long long *ctr, unsigned long long base, int *err,
                            cudaStream_t stream)
{
    switch (S) {
    case STORE_F16:
        return launch_s<STORE_F16>(SO, cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                   stream);
    case STORE_BF16:
        return launch_s<STORE_BF16>(SO, cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                    stream);
    case STORE_I16:
        return launch_s<STORE_I16>(SO, cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                   stream);
    case STORE_F32:
        switch (SO) {
        case STORE_F32:
            return launch_from_f32<STORE_F32>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base,
                                              err, stream);
        case STORE_F16:
            return launch_from_f32<STORE_F16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base,
                                              err, stream);
        case STORE_BF16:
            return launch_from_f32<STORE_BF16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base,
                                               err, stream);
        case STORE_I16:
            return launch_from_f32<STORE_I16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base,
                                              err, stream);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace afd
