// Per-thread block arithmetic of the 8 x 2-voxel streaming kernels
// (pm_wide.cu, pm_wide2.cu): a thread owns 8 (x) x 2 (y) voxels of a plane
// and computes the canonical per-face update (afd_math.cuh; arXiv:1609.03782
// Sec. 3.3) from a shared-memory tile of the plane (the slot, with its x and
// y halo), its block's values of the plane in registers and the plane above.
//   * Raw8 / ld_raw8 / cvt8: one block row (8 stored elements) from shared
//     memory and its conversion to packed float32 pairs in storage units.
//   * stg8: one block row to global memory (predicated), rounded back to the
//     storage format.
//   * clamp8: outside-the-cube voxels of a row that straddles an x face take
//     the nearest inside value (zero flux across the face).
//   * Offs: the block's rows and neighbours in a slot; a missing neighbour
//     across a cube face points at the own voxel (zero flux).
//   * xy_sums: s = s_x + s_y of the block's 16 voxels.
#pragma once

#include "afd_math.cuh"
#include "afd_store.cuh"

namespace afd {

// 8 stored elements (one block row) as read from a slot: one 16-byte load
// for 2-byte formats, two for float32.  A8: the row starts only 8-byte
// aligned (2-byte formats), so it takes two 8-byte loads.
template <int S>
struct Raw8 {
    uint4 w[S == STORE_F32 ? 2 : 1];
};

template <int S, bool A8 = false>
__device__ __forceinline__ Raw8<S> ld_raw8(const unsigned char *p)
{
    Raw8<S> r;
    if constexpr (A8 && S != STORE_F32) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        const uint2 b = *reinterpret_cast<const uint2 *>(p + 8);
        r.w[0] = make_uint4(a.x, a.y, b.x, b.y);
    } else {
        r.w[0] = *reinterpret_cast<const uint4 *>(p);
        if constexpr (S == STORE_F32)
            r.w[1] = *reinterpret_cast<const uint4 *>(p + 16);
    }
    return r;
}

// -> 4 packed float32 pairs (x, x+1), (x+2, x+3), ... in storage units, with
// Store<S>::load's arithmetic for every element.
template <int S>
__device__ __forceinline__ void cvt8(const Raw8<S> &raw, f2_t (&p)[4])
{
    if constexpr (S == STORE_F32) {
        p[0] = f2_pack(__uint_as_float(raw.w[0].x), __uint_as_float(raw.w[0].y));
        p[1] = f2_pack(__uint_as_float(raw.w[0].z), __uint_as_float(raw.w[0].w));
        p[2] = f2_pack(__uint_as_float(raw.w[1].x), __uint_as_float(raw.w[1].y));
        p[3] = f2_pack(__uint_as_float(raw.w[1].z), __uint_as_float(raw.w[1].w));
    } else {
        const unsigned ws[4] = {raw.w[0].x, raw.w[0].y, raw.w[0].z, raw.w[0].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if constexpr (S == STORE_F16) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&ws[i]));
                p[i] = f2_pack(f.x, f.y);
            } else if constexpr (S == STORE_BF16) {
                p[i] = f2_pack(__uint_as_float(ws[i] << 16),
                               __uint_as_float(ws[i] & 0xffff0000u));
            } else {
                const int lo = static_cast<int>(static_cast<short>(ws[i] & 0xffffu));
                const int hi = static_cast<int>(ws[i]) >> 16;
                // bits(1.5*2^23) + q, minus 1.5*2^23: exactly q (Store<I16>::load)
                p[i] = f2_sub(f2_pack(__int_as_float(0x4B400000 + lo),
                                      __int_as_float(0x4B400000 + hi)),
                              f2_pack(12582912.0f, 12582912.0f));
            }
        }
    }
}

template <int S>
__device__ __forceinline__ float lds_elem(const unsigned char *slot, int byte_off)
{
    typedef typename Store<S>::T E;
    return Store<S>::load(*reinterpret_cast<const E *>(slot + byte_off));
}

// 4 packed pairs -> 8 stored elements at p if `on` (predicated stores: no
// branch around them).
template <int S>
__device__ __forceinline__ void stg8(typename Store<S>::T *p, const f2_t (&v)[4], bool on)
{
    if constexpr (S == STORE_F32) {
        unsigned w[8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm("mov.b64 {%0, %1}, %2;" : "=r"(w[2 * i]), "=r"(w[2 * i + 1]) : "l"(v[i]));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %9, 0;\n\t"
            "@p st.global.v4.b32 [%0], {%1, %2, %3, %4};\n\t"
            "@p st.global.v4.b32 [%0+16], {%5, %6, %7, %8};\n\t}" ::"l"(p),
            "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]),
            "r"(w[7]), "r"(static_cast<unsigned>(on))
            : "memory");
    } else {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v[i]));
            w[i] = store2<S>(lo, hi);
        }
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
            "@p st.global.v4.b32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
            "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(static_cast<unsigned>(on))
            : "memory");
    }
}

// A block row that straddles the cube's x face (only its first m < 8 voxels
// inside, possible when nx is not a multiple of 8): the outside voxels take
// the last inside value, so the face at the cube boundary has difference +0
// (zero flux); the outside voxels' own results land in the row padding.
__device__ __forceinline__ void clamp8(f2_t (&p)[4], int m)
{
    float v[8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v[2 * i]), "=f"(v[2 * i + 1]) : "l"(p[i]));
#pragma unroll
    for (int i = 1; i < 8; ++i)
        v[i] = (i >= m) ? v[i - 1] : v[i];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        p[i] = f2_pack(v[2 * i], v[2 * i + 1]);
}

// Two-sided form: voxels before position a (outside the cube's lower x face)
// take the value at a, voxels from position b on (outside the upper face)
// the value at b - 1 (0 <= a < b <= 8).
__device__ __forceinline__ void clamp8_ab(f2_t (&p)[4], int a, int b)
{
    float v[8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v[2 * i]), "=f"(v[2 * i + 1]) : "l"(p[i]));
#pragma unroll
    for (int i = 1; i < 8; ++i)
        v[i] = (i >= b) ? v[i - 1] : v[i];
#pragma unroll
    for (int i = 6; i >= 0; --i)
        v[i] = (i < a) ? v[i + 1] : v[i];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        p[i] = f2_pack(v[2 * i], v[2 * i + 1]);
}

struct Kp {
    f2_t ax, ay, az, bx, by, bz, z;
    f2_t ai, one;  // the intensity form's 1/(K rms)^2 and 1 (COND_INT only)
};

template <int C>
__device__ __forceinline__ Kp make_kp(const Coef &kc)
{
    // the rational conductance has one A for every axis (A = 1/(K^2 dt); only
    // B depends on the spacing): one register pair instead of three
    const float ay = (C == COND_RAT) ? kc.ax : kc.ay, az = (C == COND_RAT) ? kc.ax : kc.az;
    return Kp{f2_pack(kc.ax, kc.ax), f2_pack(ay, ay), f2_pack(az, az), f2_pack(kc.bx, kc.bx),
              f2_pack(kc.by, kc.by), f2_pack(kc.bz, kc.bz), f2_pack(kc.nz, kc.nz),
              f2_pack(kc.ai, kc.ai), f2_pack(1.0f, 1.0f)};
}

// Per-thread shared-memory byte offsets (within a slot) of the block's rows
// and neighbours; a missing neighbour across a cube face points at the own
// voxel (zero flux).
struct Offs {
    int r0, r1, dn, up, xl0, xr0, xl1, xr1;
};

// The x and y parts of the update of one plane: s = s_x + s_y for the
// block's 16 voxels, from the plane's slot and the plane's values in
// registers (c0: row 0, c1: row 1).  A8 as for ld_raw8.
template <int S, int C, bool A8 = false>
__device__ __forceinline__ void xy_sums(const unsigned char *slot, const Offs &o, const Kp &k,
                                        const f2_t (&c0)[4], const f2_t (&c1)[4],
                                        f2_t (&s0)[4], f2_t (&s1)[4])
{
    f2_t dn[4], up[4];
    cvt8<S>(ld_raw8<S, A8>(slot + o.dn), dn);
    cvt8<S>(ld_raw8<S, A8>(slot + o.up), up);
    const float xl0 = lds_elem<S>(slot, o.xl0), xr0 = lds_elem<S>(slot, o.xr0);
    const float xl1 = lds_elem<S>(slot, o.xl1), xr1 = lds_elem<S>(slot, o.xr1);

    // ---- y: faces (dn|r0), (r0|r1), (r1|up); s_y = G(upper) - G(lower)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const f2_t gd = face_flux2<C>(f2_sub(c0[i], dn[i]), k.ay, k.by, k.z);
        const f2_t gm = face_flux2<C>(f2_sub(c1[i], c0[i]), k.ay, k.by, k.z);
        const f2_t gu = face_flux2<C>(f2_sub(up[i], c1[i]), k.ay, k.by, k.z);
        s0[i] = f2_sub(gm, gd);
        s1[i] = f2_sub(gu, gm);
    }

    // ---- x: faces F0 (xl|v0) .. F8 (v7|xr) of each row; the differences
    // are scalar subtractions written into the pairs (F0,F1), (F2,F3), ...,
    // F8 of both rows in one pair; s_x(v_i) = F_{i+1} - F_i as scalars into
    // the update's pairs.
    float v0[8], v1[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v0[2 * i]), "=f"(v0[2 * i + 1]) : "l"(c0[i]));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(v1[2 * i]), "=f"(v1[2 * i + 1]) : "l"(c1[i]));
    }
    const f2_t f8 = face_flux2<C>(f2_pack(__fsub_rn(xr0, v0[7]), __fsub_rn(xr1, v1[7])), k.ax,
                                  k.bx, k.z);
    float F0[9], F1[9];
    F0[8] = f2_lo(f8);
    F1[8] = f2_hi(f8);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float l0 = i == 0 ? xl0 : v0[2 * i - 1];
        const float l1 = i == 0 ? xl1 : v1[2 * i - 1];
        const f2_t g0 = face_flux2<C>(
            f2_pack(__fsub_rn(v0[2 * i], l0), __fsub_rn(v0[2 * i + 1], v0[2 * i])), k.ax, k.bx,
            k.z);
        const f2_t g1 = face_flux2<C>(
            f2_pack(__fsub_rn(v1[2 * i], l1), __fsub_rn(v1[2 * i + 1], v1[2 * i])), k.ax, k.bx,
            k.z);
        asm("mov.b64 {%0, %1}, %2;" : "=f"(F0[2 * i]), "=f"(F0[2 * i + 1]) : "l"(g0));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(F1[2 * i]), "=f"(F1[2 * i + 1]) : "l"(g1));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const f2_t sx0 = f2_pack(__fsub_rn(F0[2 * i + 1], F0[2 * i]),
                                 __fsub_rn(F0[2 * i + 2], F0[2 * i + 1]));
        const f2_t sx1 = f2_pack(__fsub_rn(F1[2 * i + 1], F1[2 * i]),
                                 __fsub_rn(F1[2 * i + 2], F1[2 * i + 1]));
        // canonical order: (s_x + s_y), then + s_z in the caller
        s0[i] = f2_add(sx0, s0[i]);
        s1[i] = f2_add(sx1, s1[i]);
    }
}


}  // namespace afd
