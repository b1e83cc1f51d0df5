// Canonical per-face arithmetic of the anisotropic-diffusion step.
//
// One explicit iteration of the per-face Perona-Malik scheme (arXiv:1609.03782,
// Sec. 3.3, eq. "perona" discretised face by face, gradient conductance as
// printed after it): through the face between a lower voxel and an upper voxel
// along axis a (spacing h_a) with raw difference delta = I(upper) - I(lower),
// the weighted flux is
//     G = w_a g(delta/(K h_a)) delta,        w_a = dt / h_a^2,
// the lower voxel gains G and the upper voxel loses it.  The weight w_a is
// folded into the conductance so that one face costs one FMA-class op more
// than its difference:
//     rational     G = delta / (A_a delta^2 + B_a),  A_a = 1/(K^2 dt),
//                                                    B_a = h_a^2 / dt
//     exponential  G = delta 2^(A_a delta^2 + B_a),  A_a = -log2(e)/(K h_a)^2,
//                                                    B_a = log2(dt / h_a^2)
//     linear (K = +inf, the heat equation)  G = A_a delta,  A_a = w_a.
// Per voxel, with G_a- the flux through its lower face and G_a+ through its
// upper face along axis a:
//     I' = I + ((s_x + s_y) + s_z),   s_a = G_a+ - G_a-.
//
// Every kernel of the library computes G and I' with exactly these
// operations, each rounded to nearest (explicit intrinsics or packed f32x2
// instructions, which round every lane like the scalar instruction; nothing
// is left to the compiler's contraction).  So all kernel variants — any tile
// shape, packed or scalar, any temporal depth, any batch placement — give
// bit-identical float32 results.
//
// The final product of a flux, delta * g, is formed as fma(delta, g, Z) with
// Z = -0 taken from a kernel argument: delta*g + (-0) is delta*g exactly, so
// this is the correctly rounded product, but the code generator can neither
// see through it nor fuse it into the subtraction that consumes it (a packed
// mul.rn.f32x2 feeding a packed sub was found fused into one FFMA2 with a
// single rounding, which made the streaming kernel differ from the
// one-voxel-per-thread kernel in the last bit).
//
// Face sharing: G depends on delta through delta^2 and a final product with
// delta, and float subtraction is exactly antisymmetric (RN(a-b) = -RN(b-a)),
// so a face's flux is one number for both voxels: kernels compute it once.
//
// A face on the cube boundary is handled by substituting the voxel's own value
// for the missing neighbour: delta = +0 and G = +0 exactly (zero flux).
#pragma once

#include <cmath>
#include <cstdint>
#include <limits>
#include <cuda_runtime.h>

namespace afd {

// Conductance kinds as the kernels see them.  LIN (g = 1) is what both
// conductances become for K = +inf.  INT is the paper's intensity-driven form
// (Sec. 3.3, the update after eq. "conductivepara"): linear face fluxes
// G = tau C_a delta and one conductance per voxel,
//     I' = I + S ((s_x + s_y) + s_z),  S = 1 / (1 + I^2 / (K rms)^2),
// evaluated as I' = fma((s_x + s_y) + s_z, rcp(fma(ai, I*I, 1)), I) with
// ai = 1/(K rms)^2.
enum CondKind : int { COND_EXP = 0, COND_RAT = 1, COND_LIN = 2, COND_INT = 3 };

// Per-call, per-axis coefficients (see above), computed on the host in double
// and rounded once.
struct Coef {
    float ax, ay, az;
    float bx, by, bz;
    float nz;  // -0.0f (see above)
    float ai;  // intensity form: 1/(K rms)^2 (unused otherwise)
};

// Host: coefficients for spacing h (NULL = unit), K > 0 (may be +inf), dt > 0.
// cond_exponential selects the exponential conductance.  *kind receives the
// kernel kind.  A is clamped to the float range so that a tiny K cannot give
// inf * 0 = NaN (for such K every flux is 0 to within float precision).
inline Coef make_coef(const float *spacing, float K, float dt, bool cond_exponential, int *kind)
{
    const double h[3] = {spacing ? spacing[0] : 1.0, spacing ? spacing[1] : 1.0,
                         spacing ? spacing[2] : 1.0};
    const double fmax = static_cast<double>(std::numeric_limits<float>::max());
    const bool lin = std::isinf(K);
    *kind = lin ? COND_LIN : (cond_exponential ? COND_EXP : COND_RAT);
    const double log2e = 1.4426950408889634074;  // exp(-u) = 2^(-u log2 e)
    const double Kd = static_cast<double>(K), dtd = static_cast<double>(dt);
    double A[3], B[3];
    for (int a = 0; a < 3; ++a) {
        const double w = dtd / (h[a] * h[a]);
        if (lin) {
            A[a] = w;
            B[a] = 0.0;
        } else if (cond_exponential) {
            const double kh = Kd * h[a];
            A[a] = -log2e / (kh * kh);
            if (!(A[a] >= -fmax))
                A[a] = -fmax;
            B[a] = std::log2(w);
        } else {
            A[a] = 1.0 / (Kd * Kd * dtd);
            if (!(A[a] <= fmax))
                A[a] = fmax;
            B[a] = (h[a] * h[a]) / dtd;
        }
    }
    Coef c;
    c.ax = static_cast<float>(A[0]);
    c.ay = static_cast<float>(A[1]);
    c.az = static_cast<float>(A[2]);
    c.bx = static_cast<float>(B[0]);
    c.by = static_cast<float>(B[1]);
    c.bz = static_cast<float>(B[2]);
    c.nz = -0.0f;
    c.ai = 0.0f;
    return c;
}

// Host: coefficients of the paper's intensity-driven form: face weights
// tau C_a and ai = 1/(K rms)^2 (clamped to the float range; K rms = +inf gives
// S = 1, the heat equation with weights tau C_a).
inline Coef make_coef_intensity(const float *C, float K, float rms, float tau)
{
    Coef c;
    const double t = static_cast<double>(tau);
    c.ax = static_cast<float>(t * static_cast<double>(C[0]));
    c.ay = static_cast<float>(t * static_cast<double>(C[1]));
    c.az = static_cast<float>(t * static_cast<double>(C[2]));
    c.bx = c.by = c.bz = 0.0f;
    c.nz = -0.0f;
    const double kr = static_cast<double>(K) * static_cast<double>(rms);
    double ai = std::isinf(kr) ? 0.0 : 1.0 / (kr * kr);
    if (!(ai <= static_cast<double>(std::numeric_limits<float>::max())))
        ai = std::numeric_limits<float>::max();
    c.ai = static_cast<float>(ai);
    return c;
}

// Device: the A coefficient of one axis, with make_coef's operations (double
// precision, rounded once to float by the caller), for K given on the device
// (noise-relative K).  The spacing-only B terms involve log2 and come from
// the host's make_coef, so both sides produce the same floats.
__device__ inline double coef_a_device(double Kd, int kind, double dt, double h)
{
    const double fmax = 3.4028234663852886e38;
    if (kind == COND_LIN)
        return dt / (h * h);
    if (kind == COND_EXP) {
        const double kh = Kd * h;
        const double v = -1.4426950408889634074 / (kh * kh);
        return (v >= -fmax) ? v : -fmax;
    }
    const double v = 1.0 / (Kd * Kd * dt);
    return (v <= fmax) ? v : fmax;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- scalar ---
template <int C>
__device__ __forceinline__ float face_flux(float delta, float A, float B, float Z)
{
    if (C == COND_LIN || C == COND_INT)
        return __fmaf_rn(A, delta, Z);
    const float t = __fmul_rn(delta, delta);
    const float u = __fmaf_rn(A, t, B);
    const float g = (C == COND_EXP) ? ex2_approx(u) : rcp_approx(u);
    return __fmaf_rn(delta, g, Z);
}

// I' = I + ((s_x + s_y) + s_z), s_a = G_a+ - G_a-.
__device__ __forceinline__ float pm_update(float c, float gxm, float gxp, float gym, float gyp,
                                           float gzm, float gzp)
{
    const float sx = __fsub_rn(gxp, gxm);
    const float sy = __fsub_rn(gyp, gym);
    const float sz = __fsub_rn(gzp, gzm);
    return __fadd_rn(c, __fadd_rn(__fadd_rn(sx, sy), sz));
}

// The intensity-driven update (COND_INT).
__device__ __forceinline__ float pm_update_int(float c, float gxm, float gxp, float gym,
                                               float gyp, float gzm, float gzp, float ai)
{
    const float sx = __fsub_rn(gxp, gxm);
    const float sy = __fsub_rn(gyp, gym);
    const float sz = __fsub_rn(gzp, gzm);
    const float acc = __fadd_rn(__fadd_rn(sx, sy), sz);
    const float S = rcp_approx(__fmaf_rn(ai, __fmul_rn(c, c), 1.0f));
    return __fmaf_rn(acc, S, c);
}

// ---------------------------------------------------------------- packed ---
// Two float32 lanes in one 64-bit register pair (lo = first voxel).  The
// f32x2 instructions round each lane exactly as the scalar instruction does.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float f2_lo(f2_t v)
{
    float lo;
    asm("{\n\t.reg .f32 h;\n\tmov.b64 {%0, h}, %1;\n\t}" : "=f"(lo) : "l"(v));
    return lo;
}

__device__ __forceinline__ float f2_hi(f2_t v)
{
    float hi;
    asm("{\n\t.reg .f32 l;\n\tmov.b64 {l, %0}, %1;\n\t}" : "=f"(hi) : "l"(v));
    return hi;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Packed face flux: the scalar face_flux on each lane.  A2, B2 and Z2 hold
// the axis coefficients and -0 in both lanes.
template <int C>
__device__ __forceinline__ f2_t face_flux2(f2_t delta, f2_t A2, f2_t B2, f2_t Z2)
{
    if (C == COND_LIN || C == COND_INT)
        return f2_fma(A2, delta, Z2);
    const f2_t t = f2_mul(delta, delta);
    const f2_t u = f2_fma(A2, t, B2);
    float ul, uh;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(ul), "=f"(uh) : "l"(u));
    const f2_t g = (C == COND_EXP) ? f2_pack(ex2_approx(ul), ex2_approx(uh))
                                   : f2_pack(rcp_approx(ul), rcp_approx(uh));
    return f2_fma(delta, g, Z2);
}

// Packed canonical update of two voxels.
__device__ __forceinline__ f2_t pm_update2(f2_t c, f2_t sx, f2_t sy, f2_t sz)
{
    return f2_add(c, f2_add(f2_add(sx, sy), sz));
}

// Packed intensity-driven update of two voxels (pm_update_int on each lane);
// ai2 and one2 hold ai and 1.0f in both lanes.
__device__ __forceinline__ f2_t pm_update2_int(f2_t c, f2_t sx, f2_t sy, f2_t sz, f2_t ai2,
                                               f2_t one2)
{
    const f2_t acc = f2_add(f2_add(sx, sy), sz);
    const f2_t u = f2_fma(ai2, f2_mul(c, c), one2);
    float ul, uh;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(ul), "=f"(uh) : "l"(u));
    return f2_fma(acc, f2_pack(rcp_approx(ul), rcp_approx(uh)), c);
}

// The voxel update of conductance kind C.
template <int C>
__device__ __forceinline__ f2_t update2(f2_t c, f2_t sx, f2_t sy, f2_t sz, f2_t ai2, f2_t one2)
{
    if constexpr (C == COND_INT)
        return pm_update2_int(c, sx, sy, sz, ai2, one2);
    else
        return pm_update2(c, sx, sy, sz);
}

}  // namespace afd
