// T fused iterations of the per-face Perona-Malik step per pass over the cube
// (temporal blocking), for float32 or 2-byte storage (arXiv:1609.03782
// Sec. 3.3: the explicit iteration of eq. "perona" with the gradient
// conductance; the paper's float-precision argument of Sec. 6 motivates the
// 2-byte storage, the arithmetic stays float32).
//
// One pass reads the cube once and writes it once for T iterations, so HBM
// traffic per voxel-iteration is 2 * bytes / T.  Design (sm_103a):
//   * Persistent CTAs walk tiles of TX x TY columns over z-chunks of zc
//     planes.  Warp NCW (the last) is the producer: one lane issues a 3-D TMA
//     load per input plane (storage format, TX + 2 HX by TY + 2T elements:
//     the tile with a halo of T, widened in x to the TMA's 16-byte
//     alignment) into a small ring guarded by full/empty mbarriers.
//   * Consumer thread i owns a 4 (x) x 2 (y) block of the tile's computed
//     region, x in [x0 - HC, x0 + TX + HC) and y in [y0 - T, y0 + TY + T),
//     HC = T rounded up to whole 4-voxel blocks.  The pass is a pipeline of
//     stages along z: at step s, stage 0 converts input plane s to float32
//     and stage t (1..T) computes iteration t of plane s - t.  Each stage
//     keeps, per thread, its input plane and the flux through its lower z
//     face in registers (register-rolled z) and publishes its output plane
//     in a double-buffered float32 shared-memory plane that stage t+1 reads
//     for x and y neighbours at the next step.  One named barrier per step.
//   * Stage t only computes the blocks its successors need (the region
//     shrinks by one voxel per stage); stage T stores the tile's interior,
//     rounded to the storage format.
//   * The per-voxel arithmetic is the canonical form of afd_math.cuh on
//     packed f32x2 instructions, so with float32 storage a pass equals T
//     launches of the one-iteration kernels bit for bit, and with 2-byte
//     storage it equals dequantise -> T float32 iterations -> quantise.
// Requirements checked by the host: nx * element size a multiple of 16
// bytes, 16-byte aligned pointers.  Every mbarrier wait is bounded; after an
// expired wait the CTA keeps stepping (no thread leaves the named barrier)
// without waiting again, and the host reads the error word.
#pragma once

#include "afd_internal.h"
#include "afd_ptx.cuh"
#include "afd_store.cuh"
#include "afd_check.cuh"

namespace afd {
namespace tb {

template <int T>
struct Geom {
    static constexpr int TX = 64;
    static constexpr int TY = (T >= 8) ? 16 : 32;
    static constexpr int HC = ((T + 3) / 4) * 4;  // computed-region halo in x
    static constexpr int QX = TX / 4 + HC / 2;    // 4-voxel blocks per computed row
    static constexpr int RP = TY / 2 + T;         // row pairs: rows y0-T .. y0+TY+T-1
    static constexpr int ITEMS = QX * RP;
    static constexpr int NCONS = (ITEMS + 31) / 32 * 32;
    static constexpr int NCW = NCONS / 32;
    static constexpr int THREADS = NCONS + 32;
    static constexpr int BW = TX + 2 * HC + 8;  // stage plane row: x0-HC-4 .. x0+TX+HC+3
    static constexpr int BH = TY + 2 * T + 2;   // stage plane rows: y0-T-1 .. y0+TY+T
    static constexpr int BFLOATS = BW * BH;
    static constexpr int MIN_BLOCKS = (T <= 2) ? 2 : 1;  // CTAs per SM to fit
    static_assert(BW % 4 == 0, "16-byte rows");
};

template <int S, int T>
struct Ring {
    static constexpr int ES = Store<S>::bytes;
    static constexpr int AL = 16 / ES;  // TMA x alignment in elements
    static constexpr int HX = ((Geom<T>::HC + AL - 1) / AL) * AL;
    static constexpr int W = Geom<T>::TX + 2 * HX;  // box width (elements)
    static constexpr int H = Geom<T>::TY + 2 * T;   // box height: y0-T .. y0+TY+T-1
    static constexpr uint32_t BOX_BYTES = W * H * ES;
    static constexpr int SLOT_BYTES = (BOX_BYTES + 127) / 128 * 128;
    static constexpr uint32_t NSLOT = (T >= 8) ? 2 : 4;
    static_assert(W <= 256 && H <= 256, "TMA box limits");
};

template <int S, int T>
constexpr size_t smem_bytes()
{
    return static_cast<size_t>(Ring<S, T>::NSLOT) * Ring<S, T>::SLOT_BYTES +
           static_cast<size_t>(2 * T) * Geom<T>::BFLOATS * sizeof(float) +
           2 * Ring<S, T>::NSLOT * sizeof(uint64_t) + 128;
}

struct Q {
    f2_t a, b;
};

struct Packed {
    f2_t ax, ay, az, bx, by, bz, z;
};

__device__ __forceinline__ Q lds_q(const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {f2_pack(v.x, v.y), f2_pack(v.z, v.w)};
}

__device__ __forceinline__ void sts_q(float *p, Q v)
{
    float4 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(v.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.z), "=f"(o.w) : "l"(v.b));
    *reinterpret_cast<float4 *>(p) = o;
}

__device__ __forceinline__ Q q_sub(Q u, Q v) { return {f2_sub(u.a, v.a), f2_sub(u.b, v.b)}; }

template <int C>
__device__ __forceinline__ Q q_flux(Q d, f2_t A2, f2_t B2, f2_t Z2)
{
    return {face_flux2<C>(d.a, A2, B2, Z2), face_flux2<C>(d.b, A2, B2, Z2)};
}

// Four storage elements -> four floats (storage units).
template <int S>
__device__ __forceinline__ Q load_block(const unsigned char *p)
{
    typedef typename Store<S>::T E;
    if constexpr (S == STORE_F32) {
        return lds_q(reinterpret_cast<const float *>(p));
    } else {
        const uint2 w = *reinterpret_cast<const uint2 *>(p);
        const E e0 = static_cast<E>(w.x & 0xffffu), e1 = static_cast<E>(w.x >> 16);
        const E e2 = static_cast<E>(w.y & 0xffffu), e3 = static_cast<E>(w.y >> 16);
        return {f2_pack(Store<S>::load(e0), Store<S>::load(e1)),
                f2_pack(Store<S>::load(e2), Store<S>::load(e3))};
    }
}

// Four floats -> four storage elements at global address p.
template <int S>
__device__ __forceinline__ void store_block(typename Store<S>::T *p, Q v)
{
    float f0, f1, f2, f3;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f0), "=f"(f1) : "l"(v.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f2), "=f"(f3) : "l"(v.b));
    if constexpr (S == STORE_F32) {
        *reinterpret_cast<float4 *>(p) = make_float4(f0, f1, f2, f3);
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2(store2<S>(f0, f1), store2<S>(f2, f3));
    }
}

// s_x = G_x+ - G_x- for the 4 voxels of one row; F0 (xl|c0) .. F4 (c3|xr),
// f4 = F4 computed by the caller.
template <int C>
__device__ __forceinline__ Q x_sums(Q c, float xl, float f4, const Packed &k)
{
    float c0, c1, c2, c3;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(c.a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c2), "=f"(c3) : "l"(c.b));
    const f2_t f01 = face_flux2<C>(f2_sub(c.a, f2_pack(xl, c0)), k.ax, k.bx, k.z);
    const f2_t f23 = face_flux2<C>(f2_sub(c.b, f2_pack(c1, c2)), k.ax, k.bx, k.z);
    const f2_t f12 = f2_pack(f2_hi(f01), f2_lo(f23));
    const f2_t f34 = f2_pack(f2_hi(f23), f4);
    return {f2_sub(f12, f01), f2_sub(f34, f23)};
}

template <int S, int T, int C>
__global__ void __launch_bounds__(Geom<T>::THREADS, Geom<T>::MIN_BLOCKS)
    pm_tb_kernel(const __grid_constant__ CUtensorMap tmap, typename Store<S>::T *__restrict__ out,
                 int nx, int ny, int nz, int tiles_x, int tiles_y, int zc, int64_t ntiles, Coef kc,
                 int *err)
{
    typedef Geom<T> G;
    typedef Ring<S, T> R;
    typedef typename Store<S>::T E;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((128u - (base & 127u)) & 127u);
    unsigned char *ring = smem;
    float *bufs = reinterpret_cast<float *>(smem + R::NSLOT * R::SLOT_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(bufs + 2 * T * G::BFLOATS);
    uint64_t *empty = full + R::NSLOT;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < R::NSLOT; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], G::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == G::NCW) {
        // ---------------- producer ----------------
        if (lane == 0) {
            uint32_t kk = 0;
            const int64_t txy = static_cast<int64_t>(tiles_x) * tiles_y;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const int tz = static_cast<int>(t / txy);
                const int r = static_cast<int>(t - static_cast<int64_t>(tz) * txy);
                const int x0 = (r % tiles_x) * G::TX, y0 = (r / tiles_x) * G::TY;
                const int z0 = tz * zc, z1 = min(z0 + zc, nz);
                const int sbeg = max(z0 - T, 0), iend = min(z1 + T, nz);
                for (int s = sbeg; s < iend; ++s, ++kk) {
                    const uint32_t slot = kk & (R::NSLOT - 1);
                    const uint32_t use = kk / R::NSLOT;
                    if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u, err, kErrWaitEmpty)) {
                        atomicExch(&abort_flag, 1);
                        return;
                    }
                    mbar_arrive_expect_tx(&full[slot], R::BOX_BYTES);
                    tma_load_3d(ring + slot * R::SLOT_BYTES, &tmap, x0 - R::HX, y0 - T, s,
                                &full[slot]);
                }
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    Packed k;
    k.ax = f2_pack(kc.ax, kc.ax);
    k.ay = f2_pack(kc.ay, kc.ay);
    k.az = f2_pack(kc.az, kc.az);
    k.bx = f2_pack(kc.bx, kc.bx);
    k.by = f2_pack(kc.by, kc.by);
    k.bz = f2_pack(kc.bz, kc.bz);
    k.z = f2_pack(kc.nz, kc.nz);

    const bool item_ok = threadIdx.x < G::ITEMS;
    const int item = item_ok ? threadIdx.x : 0;
    const int qx = item % G::QX;
    const int rp = item / G::QX;
    const int col = 4 + 4 * qx;              // block column in a stage plane
    const int rowa = 1 + 2 * rp;             // block's first row in a stage plane
    int ra = rowa * G::BW + col;       // offsets of the block's rows
    int rb = ra + G::BW;
    const int rcol = (R::HX - G::HC + 4 * qx) * R::ES;  // byte column in a ring slot
    const int rrow = 2 * rp;                           // first row in a ring slot
    int ring_a = rrow * R::W * R::ES + rcol;
    int ring_b = ring_a + R::W * R::ES;
    // the block reads stage-plane floats [ra - BW, rb + BW + 4) and ring-slot
    // bytes [ring_a, ring_b + 4 ES); a thread that would leave them (checked
    // builds) works on a safe block and stores nothing
    const bool blk_ok = check_range(err, ra - G::BW, 0, G::BFLOATS, kChkTbSmem) &&
                        check_range(err, rb + G::BW + 3, 0, G::BFLOATS, kChkTbSmem) &&
                        check_range(err, ring_a, 0, R::SLOT_BYTES, kChkTbSmem) &&
                        check_range(err, ring_b + 4 * R::ES - 1, 0, R::SLOT_BYTES, kChkTbSmem);
    if (!blk_ok) {
        ra = G::BW + 4;
        rb = ra + G::BW;
        ring_a = 0;
        ring_b = R::W * R::ES;
    }

    uint32_t kk = 0, g = 0;
    const int64_t txy = static_cast<int64_t>(tiles_x) * tiles_y;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tz = static_cast<int>(t / txy);
        const int r = static_cast<int>(t - static_cast<int64_t>(tz) * txy);
        const int x0 = (r % tiles_x) * G::TX, y0 = (r / tiles_x) * G::TY;
        const int z0 = tz * zc, z1 = min(z0 + zc, nz);
        const int sbeg = max(z0 - T, 0), iend = min(z1 + T, nz);
        const int slast = z1 - 1 + T;
        const int xb = x0 - G::HC + 4 * qx;  // first voxel of the block
        const int ya = y0 - T + 2 * rp;      // rows of the block
        const int yb = ya + 1;
        const bool edge = (x0 - G::HC <= 0) || (x0 + G::TX + G::HC >= nx) || (y0 - T <= 0) ||
                          (y0 + G::TY + T >= ny);
        // stage t needs this block if it meets [x0-(T-t), x0+TX+T-t) x [y0-(T-t), y0+TY+T-t)
        unsigned need = 0;
#pragma unroll
        for (int st = 1; st <= T; ++st) {
            const int h = T - st;
            const bool nx_ok = (xb + 4 > x0 - h) && (xb < x0 + G::TX + h);
            const bool ny_ok = (yb >= y0 - h) && (ya < y0 + G::TY + h);
            if (item_ok && nx_ok && ny_ok)
                need |= 1u << st;
        }
        const bool out_x = (xb >= x0) && (xb < x0 + G::TX) && (xb < nx);
        const bool out_a = out_x && (ya >= y0) && (ya < y0 + G::TY) && (ya < ny);
        const bool out_b = out_x && (yb >= y0) && (yb < y0 + G::TY) && (yb < ny);

        // per stage: the flux through the lower z face of its current plane
        // (the current plane itself is re-read from the stage's input buffer)
        Q fb[T + 1][2];
#pragma unroll
        for (int st = 0; st <= T; ++st)
            fb[st][0] = fb[st][1] = Q{0ull, 0ull};

        for (int s = sbeg; s <= slast; ++s) {
            const int par = static_cast<int>(g & 1u);
            // ---- stage 0: input plane s, converted to float32
            Q nxt[2];
            nxt[0] = nxt[1] = Q{0ull, 0ull};
            if (s < iend) {
                const uint32_t slot = kk & (R::NSLOT - 1);
                if (!*reinterpret_cast<volatile int *>(&abort_flag)) {
                    if (!mbar_wait(&full[slot], (kk / R::NSLOT) & 1u, err, kErrWaitFull))
                        atomicExch(&abort_flag, 1);
                }
                const unsigned char *sp = ring + slot * R::SLOT_BYTES;
                nxt[0] = load_block<S>(sp + ring_a);
                nxt[1] = load_block<S>(sp + ring_b);
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&empty[slot]);
                ++kk;
                float *b0 = bufs + par * G::BFLOATS;
                sts_q(b0 + ra, nxt[0]);
                sts_q(b0 + rb, nxt[1]);
            }
            // ---- stages 1..T
#pragma unroll
            for (int st = 1; st <= T; ++st) {
                const int p = s - st;
                // this stage's input plane p (stage st-1's output of the
                // previous step) and its x/y neighbours
                const float *B = bufs + ((st - 1) * 2 + (par ^ 1)) * G::BFLOATS;
                const Q c0 = lds_q(B + ra), c1 = lds_q(B + rb);
                Q nx2[2];
                if (p + 1 < nz) {
                    nx2[0] = nxt[0];
                    nx2[1] = nxt[1];
                } else {
                    nx2[0] = c0;  // zero flux at z = nz-1
                    nx2[1] = c1;
                }
                const Q fa0 = q_flux<C>(q_sub(nx2[0], c0), k.az, k.bz, k.z);
                const Q fa1 = q_flux<C>(q_sub(nx2[1], c1), k.az, k.bz, k.z);
                const int pbeg = max(z0 - (T - st), 0);
                const int pend = min(z1 + (T - st), nz);
                Q o0 = nx2[0], o1 = nx2[1];
                if (p >= pbeg && p < pend && ((need >> st) & 1u)) {
                    Q fb0 = fb[st][0], fb1 = fb[st][1];
                    if (p == 0) {  // zero flux at z = 0
                        fb0 = q_flux<C>(q_sub(c0, c0), k.az, k.bz, k.z);
                        fb1 = q_flux<C>(q_sub(c1, c1), k.az, k.bz, k.z);
                    }
                    Q dn = lds_q(B + ra - G::BW);
                    Q up = lds_q(B + rb + G::BW);
                    Q mid = c1;
                    float xl0 = B[ra - 1], xr0 = B[ra + 4];
                    float xl1 = B[rb - 1], xr1 = B[rb + 4];
                    if (edge) {
                        if (ya == 0)
                            dn = c0;
                        if (!(ya >= 0 && yb < ny))
                            mid = c0;
                        if (yb + 1 >= ny)
                            up = c1;
                        if (xb == 0) {
                            xl0 = f2_lo(c0.a);
                            xl1 = f2_lo(c1.a);
                        }
                        if (xb + 4 >= nx) {
                            xr0 = f2_hi(c0.b);
                            xr1 = f2_hi(c1.b);
                        }
                    }
                    const Q fdn = q_flux<C>(q_sub(c0, dn), k.ay, k.by, k.z);
                    const Q fmid = q_flux<C>(q_sub(mid, c0), k.ay, k.by, k.z);
                    const Q fup = q_flux<C>(q_sub(up, c1), k.ay, k.by, k.z);
                    const f2_t c3p = f2_pack(f2_hi(c0.b), f2_hi(c1.b));
                    const f2_t f4 = face_flux2<C>(f2_sub(f2_pack(xr0, xr1), c3p), k.ax, k.bx, k.z);
                    const Q sx0 = x_sums<C>(c0, xl0, f2_lo(f4), k);
                    const Q sx1 = x_sums<C>(c1, xl1, f2_hi(f4), k);
                    o0 = {pm_update2(c0.a, sx0.a, f2_sub(fmid.a, fdn.a), f2_sub(fa0.a, fb0.a)),
                          pm_update2(c0.b, sx0.b, f2_sub(fmid.b, fdn.b), f2_sub(fa0.b, fb0.b))};
                    o1 = {pm_update2(c1.a, sx1.a, f2_sub(fup.a, fmid.a), f2_sub(fa1.a, fb1.a)),
                          pm_update2(c1.b, sx1.b, f2_sub(fup.b, fmid.b), f2_sub(fa1.b, fb1.b))};
                    if (st < T) {
                        float *Bo = bufs + (st * 2 + par) * G::BFLOATS;
                        sts_q(Bo + ra, o0);
                        sts_q(Bo + rb, o1);
                    } else if (p >= z0 && p < z1) {
                        E *po = out + (static_cast<int64_t>(p) * ny + ya) * static_cast<int64_t>(nx) +
                                xb;
                        const int64_t oext = static_cast<int64_t>(nz) * ny * nx - 3;
                        if (out_a && blk_ok &&
                            check_range(err, po - out, 0, oext, kChkTbStore))
                            store_block<S>(po, o0);
                        if (out_b && blk_ok &&
                            check_range(err, po + nx - out, 0, oext, kChkTbStore))
                            store_block<S>(po + nx, o1);
                    }
                }
                nxt[0] = o0;
                nxt[1] = o1;
                fb[st][0] = fa0;
                fb[st][1] = fa1;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(G::NCONS) : "memory");
            ++g;
        }
    }
}

}  // namespace tb
}  // namespace afd
