// Canonical per-face arithmetic of the anisotropic-diffusion step.
//
// One explicit iteration of the per-face Perona-Malik scheme (arXiv:1609.03782,
// Sec. 3.3, eq. "perona" discretised face by face, gradient conductance as
// printed after it): for the face between a lower voxel a and an upper voxel b
// along axis a with spacing h,
//     delta = I(b) - I(a)                 raw difference
//     F     = g(delta^2 * kappa) * delta  flux, kappa = 1/(K h)^2
// voxel a gains w*F and voxel b loses w*F, w = dt / h^2.  Every kernel in the
// library computes F and the per-voxel sum with exactly the operations below
// (explicit round-to-nearest intrinsics, no contraction left to the
// compiler), so all kernel variants — any tile shape, any temporal depth, any
// batch placement — give bit-identical float32 results.
//
// Face sharing: F depends on delta only through delta^2 and a final product
// with delta, and float subtraction is exactly antisymmetric
// (RN(a-b) = -RN(b-a)), so the flux a voxel receives through its lower face is
// bit-for-bit the negation of the flux its lower neighbour sends through its
// upper face.  Kernels may therefore compute each face once and use it for
// both voxels.
//
// A face on the cube boundary is handled by substituting the voxel's own value
// for the missing neighbour: delta = 0 and F = +0 exactly (zero flux).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace afd {

// Conductance kinds as the kernels see them.  LIN (g = 1) is what both
// conductances become for K = +inf: the discrete heat equation.
enum CondKind : int { COND_EXP = 0, COND_RAT = 1, COND_LIN = 2 };

// Per-call coefficients, computed on the host in double and rounded once.
struct Coef {
    float kx, ky, kz;  // kappa_a: 1/(K h_a)^2 (RAT) or log2(e)/(K h_a)^2 (EXP)
    float wx, wy, wz;  // w_a = dt / h_a^2
};

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

// F = g(delta) * delta for the face whose raw difference is delta.
//   EXP: g = 2^(-kappa delta^2) = exp(-(delta/(K h))^2)   (one MUFU.EX2)
//   RAT: g = 1 / (1 + kappa delta^2)                      (one MUFU.RCP)
//   LIN: g = 1
template <int C>
__device__ __forceinline__ float face_flux(float delta, float kappa)
{
    if (C == COND_LIN)
        return delta;
    const float t = __fmul_rn(delta, delta);
    if (C == COND_EXP) {
        const float g = ex2_approx(__fmul_rn(-kappa, t));
        return __fmul_rn(delta, g);
    }
    const float s = __fmaf_rn(kappa, t, 1.0f);
    return __fmul_rn(delta, rcp_approx(s));
}

// Canonical update of one voxel from its six face fluxes (the flux into the
// voxel through its lower (m) and upper (p) face on each axis):
//   s_a = F_am + F_ap;  acc = w_z s_z + (w_y s_y + w_x s_x);  I' = I + acc.
__device__ __forceinline__ float pm_update(float c, float fxm, float fxp,
                                           float fym, float fyp, float fzm,
                                           float fzp, const Coef &k)
{
    const float sx = __fadd_rn(fxm, fxp);
    const float sy = __fadd_rn(fym, fyp);
    const float sz = __fadd_rn(fzm, fzp);
    const float acc = __fmaf_rn(k.wz, sz, __fmaf_rn(k.wy, sy, __fmul_rn(k.wx, sx)));
    return __fadd_rn(c, acc);
}

}  // namespace afd
