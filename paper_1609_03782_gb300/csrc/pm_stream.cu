// One explicit per-face Perona-Malik iteration over an FP32 cube:
// TMA-staged x-y tiles streamed along z (arXiv:1609.03782 Sec. 3.3, the
// per-face discretisation of eq. "perona" with the gradient conductance).
//
// Design (sm_103a):
//   * Persistent CTAs walk a static list of tiles: a tile is 64 (x) x 16 (y)
//     columns over a chunk of zc planes.  Tiles are numbered x fastest, then
//     y, then z-chunk, so CTAs running at the same time share halo rows and
//     planes through L2.
//   * Warp 8 is the producer: one lane issues a 3-D TMA load
//     (cp.async.bulk.tensor) per plane of the tile's chunk, plus one halo
//     plane below and above, into a ring of shared-memory slots guarded by
//     "full" / "empty" mbarriers.  A slot holds the plane's 64 x 16 interior
//     with a one-row halo in y and a four-float halo in x (the TMA x
//     coordinate must be a multiple of 4 floats); elements outside the cube
//     are zero-filled by the TMA unit and never used.
//   * Warps 0-7 consume: thread (qx, ry) owns the 4 x-consecutive voxels
//     x0+4qx..x0+4qx+3 of row y0+ry.  Its voxels of the planes below and
//     above live in registers (the z neighbours roll through registers), the
//     x and y neighbours come from the plane's slot.  Each x face inside the
//     quad and each z face is evaluated once and used for both voxels that
//     share it (5 x-, 8 y- and 4 z-face conductances per 4 voxels).
//   * Results go straight to global memory with 16-byte stores.
// Requirements checked by the host: nx % 4 == 0, 16-byte aligned pointers.
// Every mbarrier wait is bounded (afd_ptx.cuh).
#include "afd_internal.h"
#include "afd_ptx.cuh"

namespace afd {
namespace {

constexpr int TX = kStreamTX;
constexpr int TY = kStreamTY;
constexpr int PX = TX + 8;                                // floats per slot row
constexpr int PY = TY + 2;                                // rows per slot
constexpr uint32_t BOX_BYTES = PX * PY * sizeof(float);   // one TMA box
constexpr int SLOT_BYTES = (BOX_BYTES + 127) / 128 * 128;  // 128-B aligned slots
constexpr int SLOT_FLOATS = SLOT_BYTES / 4;
constexpr int NSLOT = 6;
constexpr int NCW = kStreamConsumerWarps;
static_assert(TX == 16 * 4 && TY * 16 == NCW * 32, "thread mapping");

struct TileCoord {
    int x0, y0, z0, z1, zlo, np;
};

__device__ __forceinline__ TileCoord decode_tile(int64_t t, int tiles_x, int tiles_y, int zc,
                                                 int nz)
{
    const int64_t txy = static_cast<int64_t>(tiles_x) * tiles_y;
    const int tz = static_cast<int>(t / txy);
    const int r = static_cast<int>(t - static_cast<int64_t>(tz) * txy);
    const int ty = r / tiles_x;
    const int tx = r - ty * tiles_x;
    TileCoord c;
    c.x0 = tx * TX;
    c.y0 = ty * TY;
    c.z0 = tz * zc;
    c.z1 = min(c.z0 + zc, nz);
    c.zlo = max(c.z0 - 1, 0);
    const int zhi = min(c.z1, nz - 1);
    c.np = zhi - c.zlo + 1;
    return c;
}

template <int C>
__device__ __forceinline__ float4 flux4(float4 lo, float4 hi, float kappa)
{
    return make_float4(face_flux<C>(__fsub_rn(hi.x, lo.x), kappa),
                       face_flux<C>(__fsub_rn(hi.y, lo.y), kappa),
                       face_flux<C>(__fsub_rn(hi.z, lo.z), kappa),
                       face_flux<C>(__fsub_rn(hi.w, lo.w), kappa));
}

template <int C>
__global__ void __launch_bounds__(kStreamThreads, 3)
    pm_step_stream(const __grid_constant__ CUtensorMap tmap, float *__restrict__ out, int nx,
                   int ny, int nz, int tiles_x, int tiles_y, int zc, int64_t ntiles, Coef k,
                   int *err)
{
    extern __shared__ unsigned char smem_raw[];
    // 128-byte align the slot array (TMA destination)
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((128u - (base & 127u)) & 127u);
    float *slots = reinterpret_cast<float *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NSLOT * SLOT_BYTES);
    uint64_t *empty = full + NSLOT;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NCW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ---------------- producer ----------------
        if (lane == 0) {
            uint32_t kk = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const TileCoord tc = decode_tile(t, tiles_x, tiles_y, zc, nz);
                for (int j = 0; j < tc.np; ++j, ++kk) {
                    const uint32_t slot = kk % NSLOT;
                    const uint32_t use = kk / NSLOT;
                    if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u, err, kErrWaitEmpty))
                        return;
                    mbar_arrive_expect_tx(&full[slot], BOX_BYTES);
                    tma_load_3d(slots + slot * SLOT_FLOATS, &tmap, tc.x0 - 4, tc.y0 - 1,
                                tc.zlo + j, &full[slot]);
                }
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    const int qx = threadIdx.x & 15;
    const int ry = threadIdx.x >> 4;
    uint32_t kk = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileCoord tc = decode_tile(t, tiles_x, tiles_y, zc, nz);
        const int x = tc.x0 + 4 * qx;
        const int y = tc.y0 + ry;
        const bool active = (x < nx) && (y < ny);
        const uint32_t kbase = kk;
        const int cen = (ry + 1) * PX + 4 + 4 * qx;  // this thread's quad in a slot

#define RING(z) (kbase + static_cast<uint32_t>((z) - tc.zlo))
#define SLOT_PTR(r) (slots + ((r) % NSLOT) * SLOT_FLOATS)
#define WAIT_FULL(r)                                                                     \
    if (!mbar_wait(&full[(r) % NSLOT], ((r) / NSLOT) & 1u, err, kErrWaitFull))           \
        return;
#define RELEASE(r)                                                                       \
    do {                                                                                 \
        __syncwarp();                                                                    \
        if (lane == 0)                                                                   \
            mbar_arrive(&empty[(r) % NSLOT]);                                            \
    } while (0)

        float4 cur, fzprev;
        {
            const uint32_t r0 = RING(tc.z0);
            if (tc.z0 > 0) {
                const uint32_t rb = RING(tc.z0 - 1);
                WAIT_FULL(rb);
                const float4 prev = *reinterpret_cast<const float4 *>(SLOT_PTR(rb) + cen);
                WAIT_FULL(r0);
                cur = *reinterpret_cast<const float4 *>(SLOT_PTR(r0) + cen);
                fzprev = flux4<C>(prev, cur, k.kz);
                RELEASE(rb);
            } else {
                WAIT_FULL(r0);
                cur = *reinterpret_cast<const float4 *>(SLOT_PTR(r0) + cen);
                fzprev = flux4<C>(cur, cur, k.kz);  // zero flux through z = 0
            }
        }

        for (int z = tc.z0; z < tc.z1; ++z) {
            const uint32_t rc = RING(z);
            const float *s = SLOT_PTR(rc);
            float4 nxt, fznext;
            if (z + 1 < nz) {
                const uint32_t rn = RING(z + 1);
                WAIT_FULL(rn);
                nxt = *reinterpret_cast<const float4 *>(SLOT_PTR(rn) + cen);
                fznext = flux4<C>(cur, nxt, k.kz);
            } else {
                nxt = cur;
                fznext = flux4<C>(cur, cur, k.kz);  // zero flux through z = nz-1
            }
            // x neighbours of the quad, y neighbour quads (own value at the faces)
            const float xl = (x > 0) ? s[cen - 1] : cur.x;
            const float xr = (x + 4 < nx) ? s[cen + 4] : cur.w;
            const float4 dn = (y > 0) ? *reinterpret_cast<const float4 *>(s + cen - PX) : cur;
            const float4 up = (y + 1 < ny) ? *reinterpret_cast<const float4 *>(s + cen + PX) : cur;

            const float f0 = face_flux<C>(__fsub_rn(cur.x, xl), k.kx);
            const float f1 = face_flux<C>(__fsub_rn(cur.y, cur.x), k.kx);
            const float f2 = face_flux<C>(__fsub_rn(cur.z, cur.y), k.kx);
            const float f3 = face_flux<C>(__fsub_rn(cur.w, cur.z), k.kx);
            const float f4 = face_flux<C>(__fsub_rn(xr, cur.w), k.kx);
            const float4 fyl = flux4<C>(dn, cur, k.ky);
            const float4 fyu = flux4<C>(cur, up, k.ky);

            float4 o;
            o.x = pm_update(cur.x, -f0, f1, -fyl.x, fyu.x, -fzprev.x, fznext.x, k);
            o.y = pm_update(cur.y, -f1, f2, -fyl.y, fyu.y, -fzprev.y, fznext.y, k);
            o.z = pm_update(cur.z, -f2, f3, -fyl.z, fyu.z, -fzprev.z, fznext.z, k);
            o.w = pm_update(cur.w, -f3, f4, -fyl.w, fyu.w, -fzprev.w, fznext.w, k);
            if (active)
                *reinterpret_cast<float4 *>(
                    out + (static_cast<int64_t>(z) * ny + y) * static_cast<int64_t>(nx) + x) = o;

            RELEASE(rc);
            cur = nxt;
            fzprev = fznext;
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

}  // namespace

size_t pm_stream_smem_bytes()
{
    return static_cast<size_t>(NSLOT) * SLOT_BYTES + 2 * NSLOT * sizeof(uint64_t) + 128;
}

cudaError_t pm_stream_prepare()
{
    const int smem = static_cast<int>(pm_stream_smem_bytes());
    cudaError_t e;
    e = cudaFuncSetAttribute(pm_step_stream<COND_EXP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(pm_step_stream<COND_RAT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(pm_step_stream<COND_LIN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t pm_stream_occupancy(int *blocks_per_sm)
{
    int a = 0, b = 0, c = 0;
    const size_t smem = pm_stream_smem_bytes();
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, pm_step_stream<COND_EXP>,
                                                                  kStreamThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pm_step_stream<COND_RAT>,
                                                          kStreamThreads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, pm_step_stream<COND_LIN>,
                                                          kStreamThreads, smem);
    *blocks_per_sm = min(a, min(b, c));
    return e;
}

StreamPlan pm_stream_plan(int nx, int ny, int nz, int sm_count, int blocks_per_sm, int zc_hint)
{
    StreamPlan p;
    p.tiles_x = (nx + TX - 1) / TX;
    p.tiles_y = (ny + TY - 1) / TY;
    const int64_t txy = static_cast<int64_t>(p.tiles_x) * p.tiles_y;
    const int64_t gmax = static_cast<int64_t>(sm_count) * (blocks_per_sm > 0 ? blocks_per_sm : 1);
    int zc = zc_hint;
    if (zc <= 0) {
        // Largest chunk that keeps the CTA slots busy: score = fraction of CTA
        // slots doing work over the rounds x fraction of loaded planes that
        // are not halo.
        const int cand[4] = {64, 32, 16, 8};
        double best = -1.0;
        zc = 8;
        for (int i = 0; i < 4; ++i) {
            const int c = cand[i];
            const int64_t nt = txy * ((nz + c - 1) / c);
            const int64_t rounds = (nt + gmax - 1) / gmax;
            const double busy = static_cast<double>(nt) / static_cast<double>(rounds * gmax);
            const int planes = c < nz ? c : nz;
            const double halo = static_cast<double>(planes) / (planes + (nz > planes ? 2 : 0));
            const double score = busy * halo;
            if (score > best + 1e-9) {
                best = score;
                zc = c;
            }
        }
    }
    if (zc > nz)
        zc = nz;
    p.zc = zc;
    p.tiles_z = (nz + zc - 1) / zc;
    p.ntiles = txy * p.tiles_z;
    const int64_t rounds = (p.ntiles + gmax - 1) / gmax;
    p.grid = static_cast<int>((p.ntiles + rounds - 1) / rounds);
    return p;
}

cudaError_t launch_pm_stream(int cond, const CUtensorMap &tmap_in, float *out, int nx, int ny,
                             int nz, const Coef &k, const StreamPlan &plan, int *err,
                             cudaStream_t stream)
{
    const size_t smem = pm_stream_smem_bytes();
    switch (cond) {
    case COND_EXP:
        pm_step_stream<COND_EXP><<<plan.grid, kStreamThreads, smem, stream>>>(
            tmap_in, out, nx, ny, nz, plan.tiles_x, plan.tiles_y, plan.zc, plan.ntiles, k, err);
        break;
    case COND_RAT:
        pm_step_stream<COND_RAT><<<plan.grid, kStreamThreads, smem, stream>>>(
            tmap_in, out, nx, ny, nz, plan.tiles_x, plan.tiles_y, plan.zc, plan.ntiles, k, err);
        break;
    default:
        pm_step_stream<COND_LIN><<<plan.grid, kStreamThreads, smem, stream>>>(
            tmap_in, out, nx, ny, nz, plan.tiles_x, plan.tiles_y, plan.zc, plan.ntiles, k, err);
        break;
    }
    return cudaGetLastError();
}

}  // namespace afd
