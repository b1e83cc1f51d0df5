// One explicit per-face Perona-Malik iteration over a cube stored in a 2-byte
// format (float16, bfloat16 or int16 counts; afd_store.cuh): the depth-1 pass
// of the precision line (arXiv:1609.03782 Sec. 3.3, the per-face
// discretisation of eq. "perona" with the gradient conductance; the 2-byte
// storage follows the float-precision argument of Sec. 6).
//
// The arithmetic is the library's canonical per-face form (afd_math.cuh), so
// a pass equals dequantise -> one float32 iteration -> quantise bit for bit,
// exactly like the 4 x 2-voxel streaming kernel (pm_stream.cu).  This kernel
// is organised to issue fewer instructions per voxel, because with 2-byte
// storage the pass is bound by instruction issue, not by HBM:
//
//   * Persistent CTAs of 4 consumer warps and 1 producer warp, three per SM
//     (128 registers per thread: more independent work per warp served this
//     issue-bound pass better than more warps), take 128 (x) x 16 (y) column
//     tiles over z-chunks from a device tile counter (as the streaming kernel
//     does).  The producer issues one 3-D TMA load per plane
//     into a ring of shared-memory slots (a slot is the tile with a one-row
//     y halo and an 8-element x halo, 16 bytes, the TMA alignment unit).
//   * A consumer thread owns 8 (x) x 2 (y) voxels: one 16-byte shared-memory
//     load per row, 16 voxels per plane to share the per-plane costs (the
//     slot wait and release, pointer updates) and 3.625 conductances per
//     voxel (every face inside the block and every z face once).
//   * Per plane z: the wait for plane z+1 and the load of its two rows
//     first, then the x and y fluxes from plane z's slot (the load latency
//     overlaps them), the release of plane z's slot, the z fluxes and the
//     update.
//   * Zero flux at the cube's faces costs nothing per plane: a thread whose
//     block touches a face reads its own voxel in place of the missing
//     neighbour, by pointing that neighbour's shared-memory offset at the own
//     voxel once per tile (difference +0, flux +0, the canonical result).
//   * x differences are formed as scalars straight into the packed pairs the
//     flux arithmetic uses, and the x sums are scalars into the pairs of the
//     update; every other step runs on packed f32x2 instructions.
//
// Requirements checked by the host: nx * 2 bytes a multiple of 16 (nx a
// multiple of 8), 16-byte aligned pointers.  Every mbarrier wait is bounded
// (afd_ptx.cuh); tile indices taken from the counter are range-checked.
#include "afd_internal.h"
#include "afd_ptx.cuh"
#include "afd_check.cuh"
#include "afd_store.cuh"
#include "pm_block.cuh"

namespace afd {
namespace {

constexpr int NCWW = kWideConsumerWarps;   // consumer warps
constexpr int NTW = NCWW * 32;              // consumer threads
constexpr int TXW = kWideTX;                // single cube: 128 x TYW tiles
constexpr int TYW = kWideTY;
static_assert(TXW == 16 * 8 && TYW == 2 * (NTW / 16), "single-cube thread mapping");

// Slot ring per storage kind: 2-byte tiles in 8 slots of 6400 bytes, float32
// tiles in 4 slots of 10752 bytes (three CTAs per SM fit either way).  A
// slot holds one TMA box: the tile with a one-row y halo and a 16-byte x
// halo (HX elements) on each side.
template <int S>
struct Ring_ {
    static constexpr int ES = Store<S>::bytes;
    static constexpr int HX = 16 / ES;
    static constexpr int BYTES = wide_slot_bytes(S);
    static constexpr uint32_t N = S == STORE_F32 ? 4 : 8;
    static_assert((N & (N - 1)) == 0 && BYTES % 128 == 0, "ring geometry");
};

// The consumers' view of the slot ring: ring index r -> slot r % N, phase
// (r / N) % 2.
template <int S>
struct Ring {
    typedef Ring_<S> G;
    const unsigned char *slots;
    uint32_t full, empty;  // shared-memory addresses of the barrier arrays
    int *err;
    __device__ __forceinline__ const unsigned char *slot(uint32_t r) const
    {
        return slots + (r & (G::N - 1)) * G::BYTES;
    }
    __device__ __forceinline__ bool wait(uint32_t r) const
    {
        return mbar_wait_sleep(full + (r & (G::N - 1)) * 8, (r / G::N) & 1u, err, kErrWaitFull);
    }
    // every consumer thread arrives (the barrier counts all of them)
    __device__ __forceinline__ void release(uint32_t r) const
    {
        mbar_arrive_u32(empty + (r & (G::N - 1)) * 8);
    }
};

// Where a block's results go: row 0 at po, row 1 at po + px; the cube's
// extent for the bounds checks of checked builds.
template <int S>
struct Dst {
    typename Store<S>::T *po;
    int px;         // row pitch (elements)
    int64_t plane;  // plane pitch (elements)
    const typename Store<S>::T *obase;
    int64_t oext;
    bool act0, act1;
};

// One plane z (ring index r) of the block: plane z+1's rows (ring index r+1;
// own values at the top face) are waited for and read first, so that their
// latency overlaps the x and y arithmetic from plane z's slot; then plane
// z's slot is released, the z fluxes and the update computed and the block's
// results stored.  In: plane z (c0, c1) and its lower z-face flux (fb0, fb1).
// Out: plane z+1 (n0, n1) and the flux between them (fa0, fa1).
template <int S, int SO, int C>
__device__ __forceinline__ bool plane_step(const Ring<S> &ring, const Offs &o, const Kp &k,
                                           uint32_t r, bool has_next, int clamp_m,
                                           const Dst<SO> &d, const f2_t (&c0)[4],
                                           const f2_t (&c1)[4], const f2_t (&fb0)[4],
                                           const f2_t (&fb1)[4], f2_t (&n0)[4], f2_t (&n1)[4],
                                           f2_t (&fa0)[4], f2_t (&fa1)[4])
{
    Raw8<S> w0{}, w1{};
    if (has_next) {
        if (!ring.wait(r + 1))
            return false;
        w0 = ld_raw8<S>(ring.slot(r + 1) + o.r0);
        w1 = ld_raw8<S>(ring.slot(r + 1) + o.r1);
    }
    f2_t s0[4], s1[4];
    xy_sums<S, C>(ring.slot(r), o, k, c0, c1, s0, s1);
    ring.release(r);
    if (has_next) {
        cvt8<S>(w0, n0);
        cvt8<S>(w1, n1);
        if (clamp_m > 0) {  // a block across the cube's x face (batches only)
            clamp8(n0, clamp_m);
            clamp8(n1, clamp_m);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            n0[i] = c0[i];
            n1[i] = c1[i];
        }
    }
    // z fluxes and the update I' = I + ((s_x + s_y) + s_z)
    f2_t o0[4], o1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        fa0[i] = face_flux2<C>(f2_sub(n0[i], c0[i]), k.az, k.bz, k.z);
        fa1[i] = face_flux2<C>(f2_sub(n1[i], c1[i]), k.az, k.bz, k.z);
        o0[i] = f2_add(c0[i], f2_add(s0[i], f2_sub(fa0[i], fb0[i])));
        o1[i] = f2_add(c1[i], f2_add(s1[i], f2_sub(fa1[i], fb1[i])));
    }
    stg8<SO>(d.po, o0,
             d.act0 && check_range(ring.err, d.po - d.obase, 0, d.oext - 7, kChkStreamStore));
    stg8<SO>(d.po + d.px, o1,
            d.act1 &&
                check_range(ring.err, d.po + d.px - d.obase, 0, d.oext - 7, kChkStreamStore));
    return true;
}

// One tile as the kernel sees it.
template <int S>
struct WTile {
    int x0, y0, z0, z1;
    int nx, ny, nz;
    int tx, ty, nq, rp;  // interior; 8-voxel blocks per row pair; row pairs
    int64_t px;          // row pitch of the cube (elements)
    const void *map;     // TMA map of the source, box (tx + 2 HX) x (ty + 2)
    void *out;           // the result, in the kernel's output format
    Coef k;
};

// One dense cube (pitch nx), 128 x TYW tiles; t indexes columns fastest,
// then rows, then the planner's z-chunks.
template <int S>
struct WOne {
    static constexpr bool kRagged = false;  // nx is a multiple of 8
    const void *map;
    void *out;
    int nx, ny, nz, tiles_x, txy;
    const ZLevels *lv;
    unsigned long long *ctr;
    unsigned long long base;
    Coef k;
    __device__ __forceinline__ void tile(int64_t t, WTile<S> &w) const
    {
        const int tz = static_cast<int>(t / txy);
        const int r = static_cast<int>(t - static_cast<int64_t>(tz) * txy);
        const int ty = r / tiles_x;
        w.x0 = (r - ty * tiles_x) * TXW;
        w.y0 = ty * TYW;
        zchunk(*lv, tz, w.z0, w.z1);
        w.nx = nx;
        w.ny = ny;
        w.nz = nz;
        w.tx = TXW;
        w.ty = TYW;
        w.nq = TXW / 8;
        w.rp = TYW / 2;
        w.px = nx;
        w.map = map;
        w.out = out;
        w.k = k;
    }
    __device__ __forceinline__ int64_t next(int64_t) const
    {
        return static_cast<int64_t>(gridDim.x) +
               static_cast<int64_t>(atomicAdd(ctr, 1ull) - base);
    }
};

// Many cubes of a resident batch, each with its own tile shape (from its
// descriptor); the list holds (cube, tile) pairs, tiles of a cube numbered
// columns fastest, then rows, then z-chunks of zc planes.
template <int S>
struct WMany {
    static constexpr bool kRagged = true;
    const BatchDesc *desc;
    const int2 *list;
    const int2 *roles;
    int src, dst;
    unsigned long long *ctr;
    unsigned long long base;
    __device__ __forceinline__ void tile(int64_t t, WTile<S> &w) const
    {
        const int2 ct = list[t];
        const BatchDesc &d = desc[ct.x];
        const int txy = d.wtiles_x * d.wtiles_y;
        const int tz = ct.y / txy;
        const int r = ct.y - tz * txy;
        const int ty = r / d.wtiles_x;
        w.tx = d.wtx;
        w.ty = d.wty;
        w.nq = d.wtx / 8;
        w.rp = d.wty / 2;
        w.x0 = (r - ty * d.wtiles_x) * d.wtx;
        w.y0 = ty * d.wty;
        w.z0 = tz * d.zc;
        w.z1 = min(w.z0 + d.zc, d.nz);
        w.nx = d.nx;
        w.ny = d.ny;
        w.nz = d.nz;
        w.px = d.px;
        int sr = src, dr = dst;
        if (roles) {
            const int2 rr = roles[ct.x];
            sr = rr.x;
            dr = rr.y;
        }
        w.map = &d.mapw[sr];
        w.out = d.buf[dr];
        w.k = d.coef;
    }
    __device__ __forceinline__ int64_t next(int64_t t) const
    {
        if (!ctr)
            return t + gridDim.x;
        return static_cast<int64_t>(gridDim.x) +
               static_cast<int64_t>(atomicAdd(ctr, 1ull) - base);
    }
};

template <int S, int SO, int C, class Src>
__device__ __forceinline__ void wide_body(const Src &src, int64_t ntiles, int *err)
{
    typedef Ring_<S> G;
    typedef typename Store<SO>::T EO;
    typedef typename Store<S>::T E;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t sbase = smem_u32(smem_raw);
    unsigned char *slots = smem_raw + ((128u - (sbase & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(slots + G::N * G::BYTES);
    uint64_t *empty = full + G::N;
    int *tile_of = reinterpret_cast<int *>(empty + G::N);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < G::N; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NTW);  // every consumer thread arrives
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCWW) {
        // ---------------- producer ----------------
        if (lane == 0) {
            grid_dep_wait();  // the previous pass's writes are visible from here on
            uint32_t kk = 0;
            int64_t t = blockIdx.x;
            for (;;) {
                const bool more = t >= 0 && t < ntiles;
                int np = 1, zlo = 0;
                WTile<S> w;
                if (more) {
                    src.tile(t, w);
                    zlo = max(w.z0 - 1, 0);
                    np = min(w.z1, w.nz - 1) - zlo + 1;
                }
                const uint32_t box = more ? static_cast<uint32_t>((w.tx + 2 * G::HX) *
                                                                  (w.ty + 2) * G::ES)
                                          : 0u;
                for (int j = 0; j < np; ++j, ++kk) {
                    const uint32_t slot = kk & (G::N - 1);
                    const uint32_t use = kk / G::N;
                    // a suspending wait: a spinning producer would take issue
                    // slots from the consumer warps on its scheduler
                    if (use > 0 && !mbar_wait_sleep(smem_u32(&empty[slot]), (use - 1) & 1u, err,
                                                    kErrWaitEmpty))
                        return;
                    if (j == 0)
                        tile_of[slot] = more ? static_cast<int>(t) : -1;
                    if (!more) {
                        mbar_arrive(&full[slot]);  // the end mark: no data
                        break;
                    }
                    mbar_arrive_expect_tx(&full[slot], box);
                    tma_load_3d(slots + slot * G::BYTES, w.map, w.x0 - G::HX, w.y0 - 1, zlo + j,
                                &full[slot]);
                }
                if (!more)
                    break;
                t = src.next(t);
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    uint32_t kk = 0;
    for (;;) {
        if (!mbar_wait_sleep(smem_u32(&full[kk & (G::N - 1)]), (kk / G::N) & 1u, err,
                             kErrWaitFull))
            return;
        const int t = tile_of[kk & (G::N - 1)];
        if (t < 0)
            break;
        WTile<S> w;
        src.tile(t, w);
        const int zlo = max(w.z0 - 1, 0);
        const int np = min(w.z1, w.nz - 1) - zlo + 1;
        const int nx = w.nx, ny = w.ny, nz = w.nz;
        const bool tile_ok = check_range(err, w.z1, w.z0 + 1, static_cast<int64_t>(nz) + 1,
                                         kChkStreamTile) &&
                             check_range(err, w.x0, 0, nx, kChkStreamTile) &&
                             check_range(err, w.y0, 0, ny, kChkStreamTile);
        // thread -> (8-voxel column block qx, row pair ry) of the tile; a
        // warp whose first row pair lies past the tile keeps the slot
        // protocol and skips the arithmetic (warp-uniform)
        int qx = threadIdx.x % w.nq, ry = threadIdx.x / w.nq;
        bool idle = false, lane_on = true;
        if constexpr (Src::kRagged) {  // batches: tile shapes that leave threads over
            idle = (warp * 32) / w.nq >= w.rp;
            lane_on = ry < w.rp;
            if (!lane_on)
                qx = ry = 0;
        }
        const int x = w.x0 + 8 * qx;
        const int ya = w.y0 + 2 * ry, yb = ya + 1;
        const int PX = (w.tx + 2 * G::HX) * G::ES;  // slot row, bytes
        Offs o;
        o.r0 = (1 + 2 * ry) * PX + (G::HX + 8 * qx) * G::ES;
        o.r1 = (yb < ny) ? o.r0 + PX : o.r0;  // row 1 outside: zero flux to row 0
        o.dn = (ya == 0) ? o.r0 : o.r0 - PX;
        o.up = (yb + 1 >= ny) ? o.r1 : o.r1 + PX;
        o.xl0 = (x == 0) ? o.r0 : o.r0 - G::ES;
        o.xl1 = (x == 0) ? o.r1 : o.r1 - G::ES;
        o.xr0 = (x + 8 >= nx) ? o.r0 + 7 * G::ES : o.r0 + 8 * G::ES;
        o.xr1 = (x + 8 >= nx) ? o.r1 + 7 * G::ES : o.r1 + 8 * G::ES;
        const int box = PX * (w.ty + 2);
        // checked builds: every slot read of the block inside the tile's box
        // (else a safe block is read and nothing stored)
        const bool slot_ok = check_range(err, box, 1, G::BYTES + 1, kChkStreamSlot) &&
                             check_range(err, o.dn, 0, box - 8 * G::ES + 1, kChkStreamSlot) &&
                             check_range(err, o.up, 0, box - 8 * G::ES + 1, kChkStreamSlot) &&
                             check_range(err, o.r1, 0, box - 8 * G::ES + 1, kChkStreamSlot) &&
                             check_range(err, o.xl0, 0, box, kChkStreamSlot) &&
                             check_range(err, o.xr1, 0, box, kChkStreamSlot);
        if (!slot_ok)
            o = Offs{PX + 16, 2 * PX + 16, 16, 2 * PX + 16, PX + 16 - G::ES, PX + 16,
                     2 * PX + 16 - G::ES, 2 * PX + 16};
        // a block across the cube's x face: m < 8 of its voxels inside
        const int clamp_m = (Src::kRagged && x < nx && x + 8 > nx) ? nx - x : 0;
        const Kp k = make_kp<C>(w.k);
        Dst<SO> d;
        d.px = static_cast<int>(w.px);
        d.plane = w.px * ny;
        d.po = static_cast<EO *>(w.out) + (static_cast<int64_t>(w.z0) * ny + ya) * w.px + x;
        d.obase = static_cast<const EO *>(w.out);
        d.oext = static_cast<int64_t>(nz) * d.plane;
        d.act0 = lane_on && slot_ok && tile_ok && x < nx && ya < ny;
        d.act1 = lane_on && slot_ok && tile_ok && x < nx && yb < ny;
        const uint32_t kbase = kk;
        const Ring<S> ring{slots, smem_u32(full), smem_u32(empty), err};
        uint32_t r = kbase + static_cast<uint32_t>(w.z0 - zlo);  // ring index of plane z0

        if (idle) {
            // every plane of the chunk: wait for it, release it, in the order
            // of the arithmetic path below
            if (w.z0 > 0) {
                if (!ring.wait(r))
                    return;
                ring.release(kbase);
            }
            for (int z = w.z0; z < w.z1; ++z, ++r) {
                if (z + 1 < nz && !ring.wait(r + 1))
                    return;
                ring.release(r);
            }
            if (w.z1 < nz)
                ring.release(r);
            kk = kbase + static_cast<uint32_t>(np);
            continue;
        }

        f2_t c0[4], c1[4], fb0[4], fb1[4];  // plane z (rows 0, 1); flux through its lower z face
        if (w.z0 > 0) {
            f2_t p0[4], p1[4];
            cvt8<S>(ld_raw8<S>(ring.slot(kbase) + o.r0), p0);
            cvt8<S>(ld_raw8<S>(ring.slot(kbase) + o.r1), p1);
            if (!ring.wait(r))
                return;
            cvt8<S>(ld_raw8<S>(ring.slot(r) + o.r0), c0);
            cvt8<S>(ld_raw8<S>(ring.slot(r) + o.r1), c1);
            if (clamp_m > 0) {
                clamp8(p0, clamp_m);
                clamp8(p1, clamp_m);
                clamp8(c0, clamp_m);
                clamp8(c1, clamp_m);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fb0[i] = face_flux2<C>(f2_sub(c0[i], p0[i]), k.az, k.bz, k.z);
                fb1[i] = face_flux2<C>(f2_sub(c1[i], p1[i]), k.az, k.bz, k.z);
            }
            ring.release(kbase);
        } else {
            cvt8<S>(ld_raw8<S>(ring.slot(r) + o.r0), c0);
            cvt8<S>(ld_raw8<S>(ring.slot(r) + o.r1), c1);
            if (clamp_m > 0) {
                clamp8(c0, clamp_m);
                clamp8(c1, clamp_m);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                fb0[i] = fb1[i] = 0ull;  // +0: the zero flux at z = 0
        }
        // two planes per iteration with the register roles swapped: no copies
        f2_t n0[4], n1[4], fa0[4], fa1[4];
        int z = w.z0;
        for (; z + 1 < w.z1; z += 2, r += 2) {
            if (!plane_step<S, SO, C>(ring, o, k, r, z + 1 < nz, clamp_m, d, c0, c1, fb0, fb1, n0,
                                  n1, fa0, fa1))
                return;
            d.po += d.plane;
            if (!plane_step<S, SO, C>(ring, o, k, r + 1, z + 2 < nz, clamp_m, d, n0, n1, fa0, fa1,
                                  c0, c1, fb0, fb1))
                return;
            d.po += d.plane;
        }
        if (z < w.z1) {
            if (!plane_step<S, SO, C>(ring, o, k, r, z + 1 < nz, clamp_m, d, c0, c1, fb0, fb1, n0,
                                  n1, fa0, fa1))
                return;
            ++r;
        }
        if (w.z1 < nz)
            ring.release(r);  // the halo plane above the chunk
        kk = kbase + static_cast<uint32_t>(np);
    }
}

// One cube, input format S, output format SO.
template <int S, int SO, int C>
__global__ void __maxnreg__(kWideMaxRegs)
    pm_step_wide(const __grid_constant__ CUtensorMap tmap,
                 typename Store<SO>::T *__restrict__ out, int nx, int ny, int nz, int tiles_x,
                 int txy, const __grid_constant__ ZLevels lv, int ntiles,
                 unsigned long long *ctr, unsigned long long base, Coef kc, int *err)
{
    grid_dep_launch_dependents();  // the next pass may take SMs as this one frees them
    const WOne<S> src{&tmap, out, nx, ny, nz, tiles_x, txy, &lv, ctr, base, kc};
    wide_body<S, SO, C>(src, ntiles, err);
}

template <int S, int C>
__global__ void __maxnreg__(kWideMaxRegs)
    pm_step_wide_batch(const BatchDesc *__restrict__ desc, const int2 *__restrict__ list,
                       const int2 *__restrict__ roles, int64_t ntiles, int src_role,
                       int dst_role, unsigned long long *ctr, unsigned long long base, int *err)
{
    grid_dep_launch_dependents();
    const WMany<S> src{desc, list, roles, src_role, dst_role, ctr, base};
    wide_body<S, S, C>(src, ntiles, err);
}

template <int S>
size_t smem_of()
{
    typedef Ring_<S> G;
    return static_cast<size_t>(G::N) * G::BYTES + 2 * G::N * sizeof(uint64_t) +
           G::N * sizeof(int) + 128;
}

template <int S, int C>
cudaError_t wide_attr()
{
    cudaError_t e = cudaFuncSetAttribute(pm_step_wide<S, S, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem_of<S>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pm_step_wide_batch<S, C>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem_of<S>()));
    return e;
}

// storage -> float32 and float32 -> storage (the ends of a chain of
// one-iteration passes), for the two conductances
template <int S, int SO>
cudaError_t wide_attr_pair()
{
    const int smem = static_cast<int>(smem_of<S>());
    cudaError_t e = cudaFuncSetAttribute(pm_step_wide<S, SO, COND_EXP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pm_step_wide<S, SO, COND_RAT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <int S>
cudaError_t wide_attr_all()
{
    cudaError_t e = wide_attr<S, COND_EXP>();
    if (e == cudaSuccess)
        e = wide_attr<S, COND_RAT>();
    if (e == cudaSuccess)
        e = wide_attr<S, COND_LIN>();
    if constexpr (S != STORE_F32) {
        if (e == cudaSuccess)
            e = wide_attr_pair<S, STORE_F32>();
        if (e == cudaSuccess)
            e = wide_attr_pair<STORE_F32, S>();
    }
    return e;
}

cudaLaunchConfig_t wide_cfg(int grid, size_t smem, bool pdl, cudaStream_t stream,
                            cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kWideThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cfg;
}

template <int S, int SO, int C>
cudaError_t wide_launch(const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                        const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                        unsigned long long base, int *err, cudaStream_t stream)
{
    if (plan.ntiles > 0x7fffffff)
        return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = wide_cfg(plan.grid, smem_of<S>(), plan.pdl, stream, attr);
    return cudaLaunchKernelEx(&cfg, pm_step_wide<S, SO, C>, tmap,
                              static_cast<typename Store<SO>::T *>(out), nx, ny, nz, plan.tiles_x,
                              plan.tiles_x * plan.tiles_y, plan.lv, static_cast<int>(plan.ntiles),
                              ctr, base, k, err);
}

template <int S>
cudaError_t wide_launch_c(int cond, const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                          const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                          unsigned long long base, int *err, cudaStream_t stream)
{
    switch (cond) {
    case COND_EXP:
        return wide_launch<S, S, COND_EXP>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                           stream);
    case COND_RAT:
        return wide_launch<S, S, COND_RAT>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                           stream);
    default:
        return wide_launch<S, S, COND_LIN>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                           stream);
    }
}

template <int S, int SO>
cudaError_t wide_launch_pair(int cond, const CUtensorMap &tmap, void *out, int nx, int ny,
                             int nz, const Coef &k, const StreamPlan &plan,
                             unsigned long long *ctr, unsigned long long base, int *err,
                             cudaStream_t stream)
{
    switch (cond) {
    case COND_EXP:
        return wide_launch<S, SO, COND_EXP>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                            stream);
    case COND_RAT:
        return wide_launch<S, SO, COND_RAT>(tmap, out, nx, ny, nz, k, plan, ctr, base, err,
                                            stream);
    default:
        return cudaErrorInvalidValue;  // the chain's ends take the two conductances only
    }
}

template <int S>
cudaError_t wide_batch_c(int cond, const BatchDesc *desc, const int2 *list, const int2 *roles,
                         int64_t ntiles, int src, int dst, int grid, unsigned long long *ctr,
                         unsigned long long base, bool pdl, int *err, cudaStream_t stream)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = wide_cfg(grid, smem_of<S>(), pdl, stream, attr);
    switch (cond) {
    case COND_EXP:
        return cudaLaunchKernelEx(&cfg, pm_step_wide_batch<S, COND_EXP>, desc, list, roles, ntiles,
                                  src, dst, ctr, base, err);
    case COND_RAT:
        return cudaLaunchKernelEx(&cfg, pm_step_wide_batch<S, COND_RAT>, desc, list, roles, ntiles,
                                  src, dst, ctr, base, err);
    default:
        return cudaLaunchKernelEx(&cfg, pm_step_wide_batch<S, COND_LIN>, desc, list, roles, ntiles,
                                  src, dst, ctr, base, err);
    }
}

}  // namespace

size_t pm_wide_smem_bytes(int S)
{
    switch (S) {
    case STORE_F32: return smem_of<STORE_F32>();
    case STORE_F16: return smem_of<STORE_F16>();
    case STORE_BF16: return smem_of<STORE_BF16>();
    default: return smem_of<STORE_I16>();
    }
}

void pm_wide_box(int S, int *box_w, int *box_h)
{
    *box_w = TXW + 2 * (16 / store_bytes(S));
    *box_h = TYW + 2;
}

void pm_wide_shape(int S, int nx, int *tx, int *ty, int *tiles_x)
{
    const int es = store_bytes(S), hx = 16 / es;
    const int nt = (nx + TXW - 1) / TXW;               // tile columns of at most 128
    const int w = ((nx + nt - 1) / nt + 7) / 8 * 8;    // equal widths, multiples of 8
    const int nq = w / 8;
    int rp = NTW / nq;                                 // row pairs the threads cover
    const int rp_max = (wide_slot_bytes(S) / (es * (w + 2 * hx)) - 2) / 2;  // box fits a slot
    if (rp > rp_max)
        rp = rp_max;
    if (2 * rp + 2 > 256)                              // TMA box height limit
        rp = 127;
    *tx = w;
    *ty = 2 * rp;
    *tiles_x = nt;
}

cudaError_t pm_wide_prepare()
{
    cudaError_t e = wide_attr_all<STORE_F32>();
    if (e == cudaSuccess)
        e = wide_attr_all<STORE_F16>();
    if (e == cudaSuccess)
        e = wide_attr_all<STORE_BF16>();
    if (e == cudaSuccess)
        e = wide_attr_all<STORE_I16>();
    return e;
}

cudaError_t pm_wide_occupancy(int *blocks_per_sm)
{
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, pm_step_wide<STORE_F16, STORE_F16, COND_RAT>, kWideThreads, smem_of<STORE_F16>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, pm_step_wide_batch<STORE_F32, COND_RAT>, kWideThreads, smem_of<STORE_F32>());
    *blocks_per_sm = min(a, b);
    return e;
}

cudaError_t launch_pm_wide(int S, int cond, const CUtensorMap &tmap_in, void *out, int nx, int ny,
                           int nz, const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                           unsigned long long base, int *err, cudaStream_t stream)
{
    switch (S) {
    case STORE_F16:
        return wide_launch_c<STORE_F16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                        stream);
    case STORE_BF16:
        return wide_launch_c<STORE_BF16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                         stream);
    case STORE_I16:
        return wide_launch_c<STORE_I16>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                        stream);
    default:
        return wide_launch_c<STORE_F32>(cond, tmap_in, out, nx, ny, nz, k, plan, ctr, base, err,
                                        stream);
    }
}

cudaError_t launch_pm_wide_chain_end(int S, int SO, int cond, const CUtensorMap &tmap_in,
                                     void *out, int nx, int ny, int nz, const Coef &k,
                                     const StreamPlan &plan, unsigned long long *ctr,
                                     unsigned long long base, int *err, cudaStream_t stream)
{
    if (S == STORE_F32) {
        switch (SO) {
        case STORE_F16:
            return wide_launch_pair<STORE_F32, STORE_F16>(cond, tmap_in, out, nx, ny, nz, k, plan,
                                                          ctr, base, err, stream);
        case STORE_BF16:
            return wide_launch_pair<STORE_F32, STORE_BF16>(cond, tmap_in, out, nx, ny, nz, k,
                                                           plan, ctr, base, err, stream);
        case STORE_I16:
            return wide_launch_pair<STORE_F32, STORE_I16>(cond, tmap_in, out, nx, ny, nz, k, plan,
                                                          ctr, base, err, stream);
        }
    } else if (SO == STORE_F32) {
        switch (S) {
        case STORE_F16:
            return wide_launch_pair<STORE_F16, STORE_F32>(cond, tmap_in, out, nx, ny, nz, k, plan,
                                                          ctr, base, err, stream);
        case STORE_BF16:
            return wide_launch_pair<STORE_BF16, STORE_F32>(cond, tmap_in, out, nx, ny, nz, k,
                                                           plan, ctr, base, err, stream);
        case STORE_I16:
            return wide_launch_pair<STORE_I16, STORE_F32>(cond, tmap_in, out, nx, ny, nz, k, plan,
                                                          ctr, base, err, stream);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pm_wide_batch(int S, int cond, const BatchDesc *desc, const int2 *list,
                                 const int2 *roles, int64_t ntiles, int src_role, int dst_role,
                                 int grid, unsigned long long *ctr, unsigned long long base,
                                 bool pdl, int *err, cudaStream_t stream)
{
    switch (S) {
    case STORE_F32:
        return wide_batch_c<STORE_F32>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                       ctr, base, pdl, err, stream);
    case STORE_F16:
        return wide_batch_c<STORE_F16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                       ctr, base, pdl, err, stream);
    case STORE_BF16:
        return wide_batch_c<STORE_BF16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                        ctr, base, pdl, err, stream);
    default:
        return wide_batch_c<STORE_I16>(cond, desc, list, roles, ntiles, src_role, dst_role, grid,
                                       ctr, base, pdl, err, stream);
    }
}

}  // namespace afd
