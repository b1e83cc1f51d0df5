// One explicit per-face Perona-Malik iteration over an FP32 cube:
// TMA-staged x-y tiles streamed along z (arXiv:1609.03782 Sec. 3.3, the
// per-face discretisation of eq. "perona" with the gradient conductance).
//
// Design (sm_103a):
//   * Persistent CTAs walk a static list of tiles: a tile is 64 (x) x 32 (y)
//     columns over a chunk of zc planes.  Tiles are numbered x fastest, then
//     y, then z-chunk, so CTAs running at the same time share halo rows
//     through L2.
//   * Warp 8 is the producer: one lane issues a 3-D TMA load
//     (cp.async.bulk.tensor) per plane of the tile's chunk, plus one halo
//     plane below and above, into a ring of shared-memory slots guarded by
//     "full" / "empty" mbarriers.  A slot holds the plane's 64 x 32 interior
//     with a one-row halo in y and a four-float halo in x (the TMA x
//     coordinate must be a multiple of 4 floats); elements outside the cube
//     are zero-filled by the TMA unit and never used.
//   * Warps 0-7 consume: thread (qx, ry) owns a 4 (x) x 2 (y) block of
//     voxels, x0+4qx.., rows y0+2ry and y0+2ry+1.  The block's voxels of the
//     plane below and above roll through registers; x and y neighbours come
//     from the plane's slot.  Every face inside the block and every z face is
//     evaluated once for both voxels (30 conductances per 8 voxels), and the
//     arithmetic runs on packed f32x2 instructions (two voxels per
//     instruction; each lane rounds exactly like the scalar canonical form,
//     so results are bit-identical to the one-voxel-per-thread kernel).
//   * Tiles that touch no cube face take a path without boundary selects.
//   * Results go straight to global memory with 16-byte stores.
//   * The cube may be stored as float32 or in a 2-byte format
//     (afd_store.cuh): planes are converted to float32 as they are read from
//     the ring and rounded back on store, so a launch on a 2-byte cube is one
//     depth-1 pass of afd_filter_ex.
// Requirements checked by the host: nx * element size a multiple of 16
// bytes, 16-byte aligned pointers.  Every mbarrier wait is bounded
// (afd_ptx.cuh).
#include "afd_internal.h"
#include "afd_ptx.cuh"
#include "afd_check.cuh"
#include "afd_store.cuh"

namespace afd {
namespace {

constexpr int TX = kStreamTX;
constexpr int TY = kStreamTY;
constexpr int PY = TY + 2;                                 // rows per slot
constexpr uint32_t NSLOT = kStreamSlots;                   // power of two

// Slot geometry per storage kind: the x halo is 16 bytes (4 floats or 8
// 2-byte elements) each side so that the TMA x coordinate stays aligned.
template <int S>
struct Slot {
    static constexpr int ES = Store<S>::bytes;
    static constexpr int HX = 16 / ES;
    static constexpr int PX = TX + 2 * HX;                      // elements per row
    static constexpr uint32_t BOX_BYTES = PX * PY * ES;         // one TMA box
    static constexpr int BYTES = (BOX_BYTES + 127) / 128 * 128;  // 128-B aligned
};
constexpr int SLOT_BYTES_MAX = Slot<STORE_F32>::BYTES;
constexpr int NCW = kStreamConsumerWarps;
static_assert(TX == 16 * 4 && TY == 2 * 16 && NCW * 32 == 256, "thread mapping");
static_assert(Slot<STORE_F16>::BYTES <= SLOT_BYTES_MAX, "slot sizes");
static_assert((NSLOT & (NSLOT - 1)) == 0, "ring size must be a power of two");

struct TileCoord {
    int x0, y0, z0, z1, zlo, np;
};

// Tile t of a cube cut into tiles_x x tiles_y columns and z-chunks; t runs
// over the columns fastest, so the CTAs working at one time are on
// neighbouring columns at the same depth (shared halos stay in L2).  The
// first lv.nuni chunks are zlen + 1 planes long for tz < zrem and zlen planes
// after that; the chunks after them start at lv.off[tz - nuni] (the guided
// sequence of the planner, long chunks first and short ones last).
__device__ __forceinline__ TileCoord decode_tile(int t, int tiles_x, int txy, const ZLevels &lv,
                                                 int nz)
{
    const int tz = t / txy;
    const int r = t - tz * txy;
    const int ty = r / tiles_x;
    const int tx = r - ty * tiles_x;
    TileCoord c;
    c.x0 = tx * TX;
    c.y0 = ty * TY;
    if (tz < lv.nuni) {
        c.z0 = tz * lv.zlen + min(tz, lv.zrem);
        c.z1 = c.z0 + lv.zlen + (tz < lv.zrem ? 1 : 0);
    } else {
        c.z0 = lv.off[tz - lv.nuni];
        c.z1 = lv.off[tz - lv.nuni + 1];
    }
    c.zlo = max(c.z0 - 1, 0);
    const int zhi = min(c.z1, nz - 1);
    c.np = zhi - c.zlo + 1;
    return c;
}

// Four voxels of one row as two packed pairs: (x, x+1) and (x+2, x+3).
struct Q {
    f2_t a, b;
};

__device__ __forceinline__ Q lds_q(const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {f2_pack(v.x, v.y), f2_pack(v.z, v.w)};
}

__device__ __forceinline__ Q q_sub(Q u, Q v) { return {f2_sub(u.a, v.a), f2_sub(u.b, v.b)}; }

template <int C>
__device__ __forceinline__ Q q_flux(Q d, f2_t A2, f2_t B2, f2_t Z2)
{
    return {face_flux2<C>(d.a, A2, B2, Z2), face_flux2<C>(d.b, A2, B2, Z2)};
}

// Four stored elements at element offset `off` of a slot -> float32 quad.
template <int S>
__device__ __forceinline__ Q lds_qs(const unsigned char *slot, int off)
{
    if constexpr (S == STORE_F32) {
        return lds_q(reinterpret_cast<const float *>(slot) + off);
    } else {
        typedef typename Store<S>::T E;
        const uint2 w = *reinterpret_cast<const uint2 *>(slot + off * 2);
        return {f2_pack(Store<S>::load(static_cast<E>(w.x & 0xffffu)),
                        Store<S>::load(static_cast<E>(w.x >> 16))),
                f2_pack(Store<S>::load(static_cast<E>(w.y & 0xffffu)),
                        Store<S>::load(static_cast<E>(w.y >> 16)))};
    }
}

template <int S>
__device__ __forceinline__ float lds_s(const unsigned char *slot, int off)
{
    typedef typename Store<S>::T E;
    return Store<S>::load(reinterpret_cast<const E *>(slot)[off]);
}

template <int S>
__device__ __forceinline__ void stg_q(typename Store<S>::T *p, Q v)
{
    float4 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(v.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.z), "=f"(o.w) : "l"(v.b));
    if constexpr (S == STORE_F32) {
        *reinterpret_cast<float4 *>(p) = o;
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2(store2<S>(o.x, o.y), store2<S>(o.z, o.w));
    }
}

struct Packed {
    f2_t ax, ay, az, bx, by, bz, z, ai, one;
};

// A quad that straddles the cube's x face (only its first m < 4 voxels are
// inside, possible when rows are padded): the outside lanes take the last
// inside value, so the x face at the cube boundary has delta = +0 (zero
// flux); the outside lanes' own results are never used.
__device__ __forceinline__ Q clamp_quad(Q c, int m)
{
    if (m == 1) {
        const float c0 = f2_lo(c.a);
        return {f2_pack(c0, c0), f2_pack(c0, c0)};
    }
    if (m == 2) {
        const float c1 = f2_hi(c.a);
        return {c.a, f2_pack(c1, c1)};
    }
    const float c2 = f2_lo(c.b);
    return {c.a, f2_pack(c2, c2)};
}

// x fluxes of one row: voxel sums s_x = G_x+ - G_x- for the quad (c0..c3)
// given its left neighbour xl and right neighbour xr.  The x faces are
// F0 (xl|c0) F1 (c0|c1) F2 (c1|c2) F3 (c2|c3) F4 (c3|xr); F4 is passed in
// (computed for both rows in one packed op).
template <int C>
__device__ __forceinline__ Q x_sums(Q c, float xl, float f4, const Packed &k)
{
    float c0, c1, c2, c3;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(c.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c2), "=f"(c3) : "l"(c.b));
    const f2_t f01 = face_flux2<C>(f2_sub(c.a, f2_pack(xl, c0)), k.ax, k.bx, k.z);  // (F0, F1)
    const f2_t f23 = face_flux2<C>(f2_sub(c.b, f2_pack(c1, c2)), k.ax, k.bx, k.z);  // (F2, F3)
    const f2_t f12 = f2_pack(f2_hi(f01), f2_lo(f23));
    const f2_t f34 = f2_pack(f2_hi(f23), f4);
    return {f2_sub(f12, f01), f2_sub(f34, f23)};
}

// Where a tile's planes come from and where its result goes.
template <int S>
struct TileInfo {
    int x0, y0, z0, z1, zlo, np;
    int nx, ny, nz;
    int64_t px;     // output row pitch (elements)
    const void *map;  // TMA descriptor (generic address)
    typename Store<S>::T *out;
    Coef k;
};

__device__ __forceinline__ void chunk_planes(int tz, int zc, int nz, int &z0, int &z1, int &zlo,
                                             int &np)
{
    z0 = tz * zc;
    z1 = min(z0 + zc, nz);
    zlo = max(z0 - 1, 0);
    np = min(z1, nz - 1) - zlo + 1;
}

// One cube, described by kernel parameters (dense rows: pitch nx).  Tiles
// are handed out dynamically: a CTA starts on tile blockIdx.x and then takes
// gridDim.x + (the next value of the launch's tile counter - base), so CTAs
// on faster SMs take more tiles and all of them end within one short tile of
// each other.
template <int S>
struct OneCube {
    // one cube: the fixed thread mapping (its code path stays the plain one)
    static constexpr bool kRemap = false;
    const void *map;
    typename Store<S>::T *out;
    int nx, ny, nz, tiles_x, txy;
    const ZLevels *lv;
    unsigned long long *ctr;
    unsigned long long base;
    Coef k;
    const Coef *kdev;  // if set: the coefficients, in device memory (written by an earlier kernel)
    __device__ __forceinline__ void tile(int t, TileInfo<S> &ti) const
    {
        const TileCoord tc = decode_tile(t, tiles_x, txy, *lv, nz);
        ti.x0 = tc.x0;
        ti.y0 = tc.y0;
        ti.z0 = tc.z0;
        ti.z1 = tc.z1;
        ti.zlo = tc.zlo;
        ti.np = tc.np;
        ti.nx = nx;
        ti.ny = ny;
        ti.nz = nz;
        ti.px = nx;
        ti.map = map;
        ti.out = out;
        ti.k = kdev ? *kdev : k;
    }
    __device__ __forceinline__ int64_t next(int64_t) const
    {
        return static_cast<int64_t>(gridDim.x) +
               static_cast<int64_t>(atomicAdd(ctr, 1ull) - base);
    }
};

// Many cubes of a resident batch: per-cube descriptors in global memory and a
// list of (cube, tile) pairs; `src` and `dst` select the buffers (roles), or
// per descriptor `roles[c]` = (src, dst) when roles is not null.  With a tile
// counter the list is handed out dynamically as for one cube, else
// round-robin.
template <int S>
struct ManyCubes {
    // ragged cutouts: narrow edge tiles remapped, idle warps skip (stream_body)
    static constexpr bool kRemap = true;
    const BatchDesc *desc;
    const int2 *list;
    const int2 *roles;
    int src, dst;
    unsigned long long *ctr;
    unsigned long long base;
    __device__ __forceinline__ int64_t next(int64_t t) const
    {
        if (!ctr)
            return t + gridDim.x;
        return static_cast<int64_t>(gridDim.x) +
               static_cast<int64_t>(atomicAdd(ctr, 1ull) - base);
    }
    __device__ __forceinline__ void tile(int64_t t, TileInfo<S> &ti) const
    {
        const int2 ct = list[t];
        const BatchDesc &d = desc[ct.x];
        const int txy = d.tiles_x * d.tiles_y;
        const int tz = ct.y / txy;
        const int r = ct.y - tz * txy;
        const int ty = r / d.tiles_x;
        ti.x0 = (r - ty * d.tiles_x) * TX;
        ti.y0 = ty * TY;
        chunk_planes(tz, d.zc, d.nz, ti.z0, ti.z1, ti.zlo, ti.np);
        ti.nx = d.nx;
        ti.ny = d.ny;
        ti.nz = d.nz;
        ti.px = d.px;
        int sr = src, dr = dst;
        if (roles) {
            const int2 rr = roles[ct.x];
            sr = rr.x;
            dr = rr.y;
        }
        ti.map = &d.map[sr];
        ti.out = static_cast<typename Store<S>::T *>(d.buf[dr]);
        ti.k = d.coef;
    }
};

// Everything one consumer thread needs for its 4 x 2 block of a tile.
template <int S>
struct PlaneArgs {
    const unsigned char *slots;
    uint64_t *full, *empty;
    int *err;
    uint32_t kbase;
    int zlo, nx, ny, nz, cen0, cen1, x, ya, yb, lane;
    bool edge, act0, act1;
    typename Store<S>::T *out0;
    int64_t row_stride;
    const typename Store<S>::T *obase;  // the output cube and its extent in
    int64_t oext;                        // elements (bounds checks only)
};

// One plane z of the block: reads the plane above (waiting for its TMA),
// computes and stores the block's 8 results, releases plane z's slot.
// In: the current plane (cur) and the flux through its lower z face (fb).
// Out: the plane above (n) and the flux through the upper face (fa), the next
// plane's cur and fb.  Returns false if a bounded wait expired.
template <int S, int C>
__device__ __forceinline__ bool plane_step(const PlaneArgs<S> &a, const Packed &k, int z,
                                           const Q &cur0, const Q &cur1, const Q &fb0,
                                           const Q &fb1, Q &n0, Q &n1, Q &fa0, Q &fa1)
{
    typedef Slot<S> SL;
    const uint32_t rc = a.kbase + static_cast<uint32_t>(z - a.zlo);
    const unsigned char *s = a.slots + (rc & (NSLOT - 1)) * SLOT_BYTES_MAX;
    // ---- z: the plane above and the flux through the upper face
    if (z + 1 < a.nz) {
        const uint32_t rn = rc + 1;
        if (!mbar_wait(&a.full[rn & (NSLOT - 1)], (rn / NSLOT) & 1u, a.err, kErrWaitFull))
            return false;
        const unsigned char *sn = a.slots + (rn & (NSLOT - 1)) * SLOT_BYTES_MAX;
        n0 = lds_qs<S>(sn, a.cen0);
        n1 = lds_qs<S>(sn, a.cen1);
    } else {
        n0 = cur0;  // zero flux at z = nz-1
        n1 = cur1;
    }
    fa0 = q_flux<C>(q_sub(n0, cur0), k.az, k.bz, k.z);
    fa1 = q_flux<C>(q_sub(n1, cur1), k.az, k.bz, k.z);

    // ---- neighbours in the plane (own value across a cube face)
    Q dn = lds_qs<S>(s, a.cen0 - SL::PX);
    Q up = lds_qs<S>(s, a.cen1 + SL::PX);
    Q mid = cur1;
    float xl0 = lds_s<S>(s, a.cen0 - 1), xr0 = lds_s<S>(s, a.cen0 + 4);
    float xl1 = lds_s<S>(s, a.cen1 - 1), xr1 = lds_s<S>(s, a.cen1 + 4);
    Q cx0 = cur0, cx1 = cur1;
    if (a.edge) {
        const float c0a = f2_lo(cur0.a), c3a = f2_hi(cur0.b);
        const float c0b = f2_lo(cur1.a), c3b = f2_hi(cur1.b);
        if (a.ya == 0)
            dn = cur0;
        if (a.yb >= a.ny)
            mid = cur0;
        if (a.yb + 1 >= a.ny)
            up = cur1;
        if (a.x == 0) {
            xl0 = c0a;
            xl1 = c0b;
        }
        if (a.x + 4 >= a.nx) {
            xr0 = c3a;
            xr1 = c3b;
        }
        if (a.x < a.nx && a.x + 4 > a.nx) {
            cx0 = clamp_quad(cur0, a.nx - a.x);
            cx1 = clamp_quad(cur1, a.nx - a.x);
        }
    }

    // ---- y: faces (dn|row0), (row0|row1), (row1|up)
    const Q fdn = q_flux<C>(q_sub(cur0, dn), k.ay, k.by, k.z);
    const Q fmid = q_flux<C>(q_sub(mid, cur0), k.ay, k.by, k.z);
    const Q fup = q_flux<C>(q_sub(up, cur1), k.ay, k.by, k.z);

    // ---- x: F4 of both rows in one packed op, then the in-row faces
    const f2_t c3p = f2_pack(f2_hi(cur0.b), f2_hi(cur1.b));
    const f2_t f4 = face_flux2<C>(f2_sub(f2_pack(xr0, xr1), c3p), k.ax, k.bx, k.z);
    const Q sx0 = x_sums<C>(cx0, xl0, f2_lo(f4), k);
    const Q sx1 = x_sums<C>(cx1, xl1, f2_hi(f4), k);

    // ---- update: I' = I + ((s_x + s_y) + s_z)
    const Q o0 = {update2<C>(cur0.a, sx0.a, f2_sub(fmid.a, fdn.a), f2_sub(fa0.a, fb0.a), k.ai, k.one),
                  update2<C>(cur0.b, sx0.b, f2_sub(fmid.b, fdn.b), f2_sub(fa0.b, fb0.b), k.ai, k.one)};
    const Q o1 = {update2<C>(cur1.a, sx1.a, f2_sub(fup.a, fmid.a), f2_sub(fa1.a, fb1.a), k.ai, k.one),
                  update2<C>(cur1.b, sx1.b, f2_sub(fup.b, fmid.b), f2_sub(fa1.b, fb1.b), k.ai, k.one)};
    typename Store<S>::T *po = a.out0 + static_cast<int64_t>(z) * a.ny * a.row_stride;
    if (a.act0 && check_range(a.err, po - a.obase, 0, a.oext - 3, kChkStreamStore))
        stg_q<S>(po, o0);
    if (a.act1 && check_range(a.err, po + a.row_stride - a.obase, 0, a.oext - 3, kChkStreamStore))
        stg_q<S>(po + a.row_stride, o1);

    __syncwarp();
    if (a.lane == 0)
        mbar_arrive(&a.empty[rc & (NSLOT - 1)]);
    return true;
}

template <int S, int C, class Src>
__device__ __forceinline__ void stream_body(const Src &src, int64_t ntiles, int *err)
{
    typedef Slot<S> SL;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((128u - (base & 127u)) & 127u);
    unsigned char *slots = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NSLOT * SLOT_BYTES_MAX);
    uint64_t *empty = full + NSLOT;
    // tile index of the tile whose first plane a slot holds, -1: no more tiles
    int *tile_of = reinterpret_cast<int *>(empty + NSLOT);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < NSLOT; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NCW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ---------------- producer ----------------
        if (lane == 0) {
            // Launched as a programmatic dependent of the previous pass, the
            // CTA may start while that pass is still running: every global
            // access of this CTA (the producer's loads and tile fetches, and
            // the consumers' stores, which follow the loads) waits here until
            // the previous grid has completed and its writes are visible.
            grid_dep_wait();
            uint32_t kk = 0;
            int64_t t = blockIdx.x;
            for (;;) {
                const bool more = t >= 0 && t < ntiles;
                TileInfo<S> tc;
                if (more)
                    src.tile(t, tc);
                const int np = more ? tc.np : 1;
                for (int j = 0; j < np; ++j, ++kk) {
                    const uint32_t slot = kk & (NSLOT - 1);
                    const uint32_t use = kk / NSLOT;
                    if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u, err, kErrWaitEmpty))
                        return;
                    if (j == 0)
                        tile_of[slot] = more ? static_cast<int>(t) : -1;
                    if (!more) {
                        mbar_arrive(&full[slot]);  // the end mark: no data
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], SL::BOX_BYTES);
                    tma_load_3d(slots + slot * SLOT_BYTES_MAX, tc.map, tc.x0 - SL::HX, tc.y0 - 1,
                                tc.zlo + j, &full[slot]);
                }
                if (!more)
                    break;
                t = src.next(t);
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    // Thread mapping: 16 quads x 16 row pairs.  With Src::kRemap (many
    // ragged cubes), per tile: a tile with only w < 64 columns inside the
    // cube (the last tile column of a cube that ends there) takes nq =
    // ceil(w / 4) quads per row pair, thread t the quad t % nq of row pair
    // t / nq, so its 16 row pairs fill the first 16 nq threads; and a warp
    // whose rows all lie past the tile or past the cube keeps the slot
    // protocol (the same waits and releases) but skips the arithmetic.
    // Lanes of a working warp past the tile's last row pair compute on a
    // safe block and store nothing.  Every active thread computes the same
    // 4 x 2 block with the same arithmetic under any mapping.
    const int qx_d = threadIdx.x & 15;
    const int ry_d = threadIdx.x >> 4;
    int cen0_d = (1 + 2 * ry_d) * SL::PX + SL::HX + 4 * qx_d;  // quad of row 0 in a slot
    int cen1_d = cen0_d + SL::PX;                               // quad of row 1
    // the block reads slot elements [cen0 - PX, cen1 + PX + 4); a thread
    // that would leave the slot (checked builds) reads a safe block instead
    // and stores nothing
    const bool slot_ok_d =
        check_range(err, cen0_d - SL::PX, 0, SL::PX * PY, kChkStreamSlot) &&
        check_range(err, cen1_d + SL::PX + 3, 0, SL::PX * PY, kChkStreamSlot);
    if (!slot_ok_d) {
        cen0_d = SL::PX + SL::HX;
        cen1_d = cen0_d + SL::PX;
    }
    uint32_t kk = 0;

    for (;;) {
        // the next tile's first slot names the tile (or ends the loop)
        if (!mbar_wait(&full[kk & (NSLOT - 1)], (kk / NSLOT) & 1u, err, kErrWaitFull))
            return;
        const int t = tile_of[kk & (NSLOT - 1)];
        if (t < 0)
            break;
        TileInfo<S> tc;
        src.tile(t, tc);
        const int nx = tc.nx, ny = tc.ny, nz = tc.nz;
        int qx = qx_d, ry = ry_d, cen0 = cen0_d, cen1 = cen1_d;
        bool slot_ok = slot_ok_d, idle = false;
        if constexpr (Src::kRemap) {
            const int wq = (nx - tc.x0 + 3) >> 2;  // quads inside the cube
            if (wq < TX / 4) {
                const int p_first = (32 * warp) / wq;  // the warp's first row pair
                // warp-uniform: the warp's first row is past the tile or the cube
                idle = p_first >= TY / 2 || tc.y0 + 2 * p_first >= ny;
                if (!idle) {
                    const int t = threadIdx.x;
                    ry = t / wq;
                    qx = t - ry * wq;
                    const bool lane_on = ry < TY / 2;
                    if (!lane_on)
                        ry = qx = 0;
                    cen0 = (1 + 2 * ry) * SL::PX + SL::HX + 4 * qx;
                    cen1 = cen0 + SL::PX;
                    slot_ok =
                        lane_on &&
                        check_range(err, cen0 - SL::PX, 0, SL::PX * PY, kChkStreamSlot) &&
                        check_range(err, cen1 + SL::PX + 3, 0, SL::PX * PY, kChkStreamSlot);
                    if (!slot_ok) {
                        cen0 = SL::PX + SL::HX;
                        cen1 = cen0 + SL::PX;
                    }
                }
            } else {
                idle = tc.y0 + 4 * warp >= ny;  // warp-uniform
            }
        }
        Packed k;
        k.ax = f2_pack(tc.k.ax, tc.k.ax);
        k.ay = f2_pack(tc.k.ay, tc.k.ay);
        k.az = f2_pack(tc.k.az, tc.k.az);
        k.bx = f2_pack(tc.k.bx, tc.k.bx);
        k.by = f2_pack(tc.k.by, tc.k.by);
        k.bz = f2_pack(tc.k.bz, tc.k.bz);
        k.z = f2_pack(tc.k.nz, tc.k.nz);
        k.ai = f2_pack(tc.k.ai, tc.k.ai);
        k.one = f2_pack(1.0f, 1.0f);
        const int x = tc.x0 + 4 * qx;
        const int ya = tc.y0 + 2 * ry;  // row 0
        const int yb = ya + 1;          // row 1
        const bool tile_ok =
            check_range(err, tc.z1, tc.z0 + 1, static_cast<int64_t>(nz) + 1, kChkStreamTile) &&
            check_range(err, tc.x0, 0, nx, kChkStreamTile) &&
            check_range(err, tc.y0, 0, ny, kChkStreamTile) &&
            check_range(err, tc.zlo, 0, nz, kChkStreamTile);
        const bool act0 = slot_ok && tile_ok && (x < nx) && (ya < ny);
        const bool act1 = slot_ok && tile_ok && (x < nx) && (yb < ny);
        const bool edge = (tc.x0 == 0) || (tc.x0 + TX >= nx) || (tc.y0 == 0) ||
                          (tc.y0 + TY >= ny);
        const uint32_t kbase = kk;
        const int64_t row_stride = tc.px;
        typename Store<S>::T *out0 = tc.out + (static_cast<int64_t>(ya) * row_stride + x);

#define RING(z) (kbase + static_cast<uint32_t>((z) - tc.zlo))
#define SLOT_PTR(r) (slots + ((r) & (NSLOT - 1)) * SLOT_BYTES_MAX)
#define WAIT_FULL(r)                                                                     \
    if (!mbar_wait(&full[(r) & (NSLOT - 1)], ((r) / NSLOT) & 1u, err, kErrWaitFull))      \
        return;
#define RELEASE(r)                                                                       \
    do {                                                                                 \
        __syncwarp();                                                                    \
        if (lane == 0)                                                                   \
            mbar_arrive(&empty[(r) & (NSLOT - 1)]);                                      \
    } while (0)

        if (idle) {
            // every plane of the chunk: wait for it, release it, in the
            // order of the arithmetic path below
            if (tc.z0 > 0) {
                WAIT_FULL(RING(tc.z0 - 1));
                WAIT_FULL(RING(tc.z0));
                RELEASE(RING(tc.z0 - 1));
            } else {
                WAIT_FULL(RING(tc.z0));
            }
            for (int z = tc.z0; z < tc.z1; ++z) {
                if (z + 1 < nz)
                    WAIT_FULL(RING(z + 1));
                RELEASE(RING(z));
            }
            if (tc.z1 < nz)
                RELEASE(RING(tc.z1));
            kk = kbase + static_cast<uint32_t>(tc.np);
            continue;
        }

        Q cur0, cur1, fb0, fb1;  // current plane and the flux through its lower z face
        {
            const uint32_t rz = RING(tc.z0);
            if (tc.z0 > 0) {
                const uint32_t rb = RING(tc.z0 - 1);
                WAIT_FULL(rb);
                const Q p0 = lds_qs<S>(SLOT_PTR(rb), cen0);
                const Q p1 = lds_qs<S>(SLOT_PTR(rb), cen1);
                WAIT_FULL(rz);
                cur0 = lds_qs<S>(SLOT_PTR(rz), cen0);
                cur1 = lds_qs<S>(SLOT_PTR(rz), cen1);
                fb0 = q_flux<C>(q_sub(cur0, p0), k.az, k.bz, k.z);
                fb1 = q_flux<C>(q_sub(cur1, p1), k.az, k.bz, k.z);
                RELEASE(rb);
            } else {
                WAIT_FULL(rz);
                cur0 = lds_qs<S>(SLOT_PTR(rz), cen0);
                cur1 = lds_qs<S>(SLOT_PTR(rz), cen1);
                fb0 = q_flux<C>(q_sub(cur0, cur0), k.az, k.bz, k.z);  // zero flux at z = 0
                fb1 = q_flux<C>(q_sub(cur1, cur1), k.az, k.bz, k.z);
            }
        }

        const PlaneArgs<S> pa{slots, full, empty, err, kbase, tc.zlo, nx, ny, nz, cen0, cen1,
                              x, ya, yb, lane, edge, act0, act1, out0, row_stride, tc.out,
                              static_cast<int64_t>(nz) * ny * row_stride};
        // two planes per iteration with the register roles swapped: no copies
        Q n0, n1, fa0, fa1;
        int z = tc.z0;
        for (; z + 1 < tc.z1; z += 2) {
            if (!plane_step<S, C>(pa, k, z, cur0, cur1, fb0, fb1, n0, n1, fa0, fa1))
                return;
            if (!plane_step<S, C>(pa, k, z + 1, n0, n1, fa0, fa1, cur0, cur1, fb0, fb1))
                return;
        }
        if (z < tc.z1) {
            if (!plane_step<S, C>(pa, k, z, cur0, cur1, fb0, fb1, n0, n1, fa0, fa1))
                return;
        }
        if (tc.z1 < nz)
            RELEASE(RING(tc.z1));  // the halo plane above the chunk
        kk = kbase + static_cast<uint32_t>(tc.np);
#undef RING
#undef SLOT_PTR
#undef WAIT_FULL
#undef RELEASE
    }
}


template <int S, int C>
__global__ void __maxnreg__(kStreamMaxRegs)
    pm_step_stream(const __grid_constant__ CUtensorMap tmap, typename Store<S>::T *__restrict__ out,
                   int nx, int ny, int nz, int tiles_x, int txy, const __grid_constant__ ZLevels lv,
                   int ntiles, unsigned long long *ctr, unsigned long long base, Coef kc,
                   const Coef *kdev, int *err)
{
    grid_dep_launch_dependents();  // the next pass may take SMs as this one frees them
    const OneCube<S> src{&tmap, out, nx, ny, nz, tiles_x, txy, &lv, ctr, base, kc, kdev};
    stream_body<S, C>(src, ntiles, err);
}

template <int S, int C>
__global__ void __maxnreg__(kStreamMaxRegs)
    pm_step_batch(const BatchDesc *__restrict__ desc, const int2 *__restrict__ list,
                  const int2 *__restrict__ roles, int64_t ntiles, int src_role, int dst_role,
                  unsigned long long *ctr, unsigned long long base, int *err)
{
    grid_dep_launch_dependents();
    const ManyCubes<S> src{desc, list, roles, src_role, dst_role, ctr, base};
    stream_body<S, C>(src, ntiles, err);
}

}  // namespace

size_t pm_stream_smem_bytes()
{
    return static_cast<size_t>(NSLOT) * SLOT_BYTES_MAX + 2 * NSLOT * sizeof(uint64_t) +
           NSLOT * sizeof(int) + 128;
}

void pm_stream_box(int S, int *box_w, int *box_h, int *hx)
{
    const int es = S == STORE_F32 ? 4 : 2;
    *hx = 16 / es;
    *box_w = TX + 2 * *hx;
    *box_h = PY;
}

namespace {
template <int S, int C>
cudaError_t stream_attr()
{
    return cudaFuncSetAttribute(pm_step_stream<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(pm_stream_smem_bytes()));
}
template <int S, int C>
cudaError_t batch_attr()
{
    return cudaFuncSetAttribute(pm_step_batch<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(pm_stream_smem_bytes()));
}
template <int S>
cudaError_t stream_attr_all()
{
    cudaError_t e = cudaSuccess;
    if constexpr (S == STORE_F32)
        e = stream_attr<S, COND_INT>();
    if (e == cudaSuccess)
        e = stream_attr<S, COND_EXP>();
    if (e == cudaSuccess)
        e = stream_attr<S, COND_RAT>();
    if (e == cudaSuccess)
        e = stream_attr<S, COND_LIN>();
    if (e == cudaSuccess)
        e = batch_attr<S, COND_EXP>();
    if (e == cudaSuccess)
        e = batch_attr<S, COND_RAT>();
    if (e == cudaSuccess)
        e = batch_attr<S, COND_LIN>();
    return e;
}
}  // namespace

cudaError_t pm_stream_prepare()
{
    cudaError_t e = stream_attr_all<STORE_F32>();
    if (e == cudaSuccess)
        e = stream_attr_all<STORE_F16>();
    if (e == cudaSuccess)
        e = stream_attr_all<STORE_BF16>();
    if (e == cudaSuccess)
        e = stream_attr_all<STORE_I16>();
    return e;
}

cudaError_t pm_stream_occupancy(int *blocks_per_sm)
{
    int a = 0, b = 0, c = 0;
    const size_t smem = pm_stream_smem_bytes();
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, pm_step_stream<STORE_F32, COND_EXP>, kStreamThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pm_step_stream<STORE_F32, COND_RAT>,
                                                          kStreamThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, pm_step_stream<STORE_F16, COND_RAT>,
                                                          kStreamThreads, smem);
    *blocks_per_sm = min(a, min(b, c));
    return e;
}

namespace {
// Guided z-chunks: each chunk is at most the share of the remaining work that
// keeps every CTA busy while the CTAs that took the chunk's tiles finish them
// (length <= remaining x txy / (grid + txy)), between lmin and zmax planes; the
// last chunks are the shortest, so the CTAs end within one short tile of each
// other.  Returns the number of chunks (-1: more than kStreamMaxLevels).
int guided_levels(int nz, int64_t txy, int64_t grid, int lmin, int *off, int zmax)
{
    int n = 0, z = 0;
    while (z < nz) {
        if (n >= kStreamMaxLevels)
            return -1;
        const int64_t left = nz - z;
        int64_t len = left * txy / (grid + txy);
        if (len < lmin)
            len = lmin;
        if (len > zmax)
            len = zmax;
        if (len > left || left - len < (lmin + 1) / 2)
            len = left;
        off[n++] = z;
        z += static_cast<int>(len);
    }
    off[n] = nz;
    return n;
}
}  // namespace

StreamPlan pm_stream_plan(int nx, int ny, int nz, int sm_count, int blocks_per_sm, int zc_hint,
                          int tile_x, int tile_y, int zmax)
{
    StreamPlan p;
    p.tiles_x = (nx + tile_x - 1) / tile_x;
    p.tiles_y = (ny + tile_y - 1) / tile_y;
    const int64_t txy = static_cast<int64_t>(p.tiles_x) * p.tiles_y;
    const int64_t gmax = static_cast<int64_t>(sm_count) * (blocks_per_sm > 0 ? blocks_per_sm : 1);
    ZLevels &lv = p.lv;
    lv.nuni = 0;
    lv.zlen = 1;
    lv.zrem = 0;
    lv.nlev = 0;
    lv.off[0] = 0;
    int n = -1;
    if (zc_hint <= 0)
        for (int lmin = 4; n < 0; lmin *= 2)
            n = guided_levels(nz, txy, gmax, lmin, lv.off, zmax);
    if (n > 0) {
        lv.nlev = n;
        p.zc = 0;
        for (int i = 0; i < n; ++i)
            p.zc = max(p.zc, lv.off[i + 1] - lv.off[i]);
    } else {
        // a fixed z-chunk: chunks of equal length (+-1), none above zc_hint
        const int zc = zc_hint > 0 ? zc_hint : nz;
        lv.nuni = (nz + zc - 1) / zc;
        lv.zlen = nz / lv.nuni;
        lv.zrem = nz % lv.nuni;
        lv.off[0] = nz;
        p.zc = lv.zlen + (lv.zrem ? 1 : 0);
    }
    p.tiles_z = lv.nuni + lv.nlev;
    p.ntiles = txy * p.tiles_z;
    p.grid = static_cast<int>(p.ntiles < gmax ? p.ntiles : gmax);
    p.pdl = false;
    p.kdev = nullptr;
    return p;
}

namespace {
template <int S, int C>
cudaError_t stream_launch(const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                          const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                          unsigned long long base, int *err, cudaStream_t stream)
{
    if (plan.ntiles > 0x7fffffff)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(plan.grid));
    cfg.blockDim = dim3(kStreamThreads);
    cfg.dynamicSmemBytes = pm_stream_smem_bytes();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = plan.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, pm_step_stream<S, C>, tmap,
                              static_cast<typename Store<S>::T *>(out), nx, ny, nz, plan.tiles_x,
                              plan.tiles_x * plan.tiles_y, plan.lv, static_cast<int>(plan.ntiles),
                              ctr, base, k, plan.kdev, err);
}
template <int S>
cudaError_t stream_launch_c(int cond, const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                            const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                            unsigned long long base, int *err, cudaStream_t stream)
{
    if constexpr (S == STORE_F32) {
        if (cond == COND_INT)
            return stream_launch<S, COND_INT>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                              stream);
    }
    switch (cond) {
    case COND_EXP:
        return stream_launch<S, COND_EXP>(tmap, out, nx, ny, nz, k, plan, ctr, base, err, stream);
    case COND_RAT:
        return stream_launch<S, COND_RAT>(tmap, out, nx, ny, nz, k, plan, ctr, base, err, stream);
    default:
        return stream_launch<S, COND_LIN>(tmap, out, nx, ny, nz, k, plan, ctr, base, err, stream);
    }
}
}  // namespace

cudaError_t launch_pm_stream_s(int S, int cond, const CUtensorMap &tmap_in, void *out, int nx,
                               int ny, int nz, const Coef &k, const StreamPlan &plan,
                               unsigned long long *ctr, unsigned long long base, int *err,
                               cudaStream_t stream)
{
    switch (S) {
    case STORE_F32:
        return stream_launch_c<STORE_F32>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                          stream);
    case STORE_F16:
        return stream_launch_c<STORE_F16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                          stream);
    case STORE_BF16:
        return stream_launch_c<STORE_BF16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base,
                                           err, stream);
    default:
        return stream_launch_c<STORE_I16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                          stream);
    }
}

namespace {
template <int S>
cudaError_t batch_launch_c(int cond, const BatchDesc *desc, const int2 *list, const int2 *roles,
                           int64_t ntiles, int src, int dst, int grid, unsigned long long *ctr,
                           unsigned long long base, bool pdl, int *err, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kStreamThreads);
    cfg.dynamicSmemBytes = pm_stream_smem_bytes();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (cond) {
    case COND_EXP:
        return cudaLaunchKernelEx(&cfg, pm_step_batch<S, COND_EXP>, desc, list, roles, ntiles, src,
                                  dst, ctr, base, err);
    case COND_RAT:
        return cudaLaunchKernelEx(&cfg, pm_step_batch<S, COND_RAT>, desc, list, roles, ntiles, src,
                                  dst, ctr, base, err);
    default:
        return cudaLaunchKernelEx(&cfg, pm_step_batch<S, COND_LIN>, desc, list, roles, ntiles, src,
                                  dst, ctr, base, err);
    }
}
}  // namespace

cudaError_t launch_pm_batch(int S, int cond, const BatchDesc *desc, const int2 *list,
                            const int2 *roles, int64_t ntiles, int src_role, int dst_role, int grid,
                            unsigned long long *ctr, unsigned long long base, bool pdl, int *err,
                            cudaStream_t stream)
{
    switch (S) {
    case STORE_F32:
        return batch_launch_c<STORE_F32>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                         ctr, base, pdl, err, stream);
    case STORE_F16:
        return batch_launch_c<STORE_F16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                         ctr, base, pdl, err, stream);
    case STORE_BF16:
        return batch_launch_c<STORE_BF16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                          ctr, base, pdl, err, stream);
    default:
        return batch_launch_c<STORE_I16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                         ctr, base, pdl, err, stream);
    }
}

cudaError_t launch_pm_stream(int cond, const CUtensorMap &tmap_in, float *out, int nx, int ny,
                             int nz, const Coef &k, const StreamPlan &plan,
                             unsigned long long *ctr, unsigned long long base, int *err,
                             cudaStream_t stream)
{
    return launch_pm_stream_s(STORE_F32, cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                              stream);
}

}  // namespace afd
