// Host-side plan and dispatch of the temporally blocked kernels (pm_tb.cuh).
#include "afd_internal.h"
#include "afd_store.cuh"

namespace afd {

bool tb_depth_ok(int T) { return T == 1 || T == 2 || T == 4 || T == 8; }

cudaError_t tb_prepare(int S, int T)
{
    switch (S) {
    case STORE_F32: return tb_prepare_f32(T);
    case STORE_F16: return tb_prepare_f16(T);
    case STORE_BF16: return tb_prepare_bf16(T);
    default: return tb_prepare_i16(T);
    }
}

TbShape tb_shape(int S, int T)
{
    switch (S) {
    case STORE_F32: return tb_shape_f32(T);
    case STORE_F16: return tb_shape_f16(T);
    case STORE_BF16: return tb_shape_bf16(T);
    default: return tb_shape_i16(T);
    }
}

cudaError_t tb_launch(int S, int T, int cond, const CUtensorMap &tmap, void *out, int nx, int ny,
                      int nz, const Coef &k, const TbPlan &plan, int *err, cudaStream_t stream)
{
    switch (S) {
    case STORE_F32: return tb_launch_f32(T, cond, tmap, out, nx, ny, nz, k, plan, err, stream);
    case STORE_F16: return tb_launch_f16(T, cond, tmap, out, nx, ny, nz, k, plan, err, stream);
    case STORE_BF16: return tb_launch_bf16(T, cond, tmap, out, nx, ny, nz, k, plan, err, stream);
    default: return tb_launch_i16(T, cond, tmap, out, nx, ny, nz, k, plan, err, stream);
    }
}

// CTAs per SM as the kernels are built (one or two).  The z-chunk trades the
// pipeline's fill and drain (about T extra planes of work per chunk) against
// keeping every CTA slot busy over whole rounds of tiles.
TbPlan tb_plan(int S, int T, int nx, int ny, int nz, int sm_count, int zc_hint)
{
    const TbShape sh = tb_shape(S, T);
    TbPlan p;
    p.tiles_x = (nx + sh.tx - 1) / sh.tx;
    p.tiles_y = (ny + sh.ty - 1) / sh.ty;
    const int64_t txy = static_cast<int64_t>(p.tiles_x) * p.tiles_y;
    const int64_t gmax = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * (T <= 2 ? 2 : 1);
    int zc = zc_hint;
    if (zc <= 0) {
        const int cand[5] = {256, 128, 64, 32, 16};
        double best = -1.0;
        zc = 16;
        for (int i = 0; i < 5; ++i) {
            const int c = cand[i] < nz ? cand[i] : nz;
            const int64_t nt = txy * ((nz + c - 1) / c);
            const int64_t rounds = (nt + gmax - 1) / gmax;
            const double busy = static_cast<double>(nt) / static_cast<double>(rounds * gmax);
            const double fill = static_cast<double>(c) / (c + static_cast<double>(T));
            const double score = busy * fill;
            if (score > best + 1e-9) {
                best = score;
                zc = c;
            }
        }
    }
    if (zc > nz)
        zc = nz;
    p.zc = zc;
    p.ntiles = txy * ((nz + zc - 1) / zc);
    const int64_t rounds = (p.ntiles + gmax - 1) / gmax;
    p.grid = static_cast<int>((p.ntiles + rounds - 1) / rounds);
    return p;
}

}  // namespace afd
