// Instantiations and launcher of the temporally blocked kernel for one
// storage format (AFD_TB_STORE), included by pm_tb_<format>.cu so that the
// formats compile in parallel.
#pragma once

#include "pm_tb.cuh"

namespace afd {
namespace {

template <int T, int C>
cudaError_t tb_launch_one(const CUtensorMap &tmap, void *out, int nx, int ny, int nz,
                          const Coef &k, const TbPlan &plan, int *err, cudaStream_t stream)
{
    constexpr int S = AFD_TB_STORE;
    typedef typename Store<S>::T E;
    const size_t smem = tb::smem_bytes<S, T>();
    tb::pm_tb_kernel<S, T, C><<<plan.grid, tb::Geom<T>::THREADS, smem, stream>>>(
        tmap, static_cast<E *>(out), nx, ny, nz, plan.tiles_x, plan.tiles_y, plan.zc, plan.ntiles,
        k, err);
    return cudaGetLastError();
}

template <int T>
cudaError_t tb_prepare_one()
{
    constexpr int S = AFD_TB_STORE;
    const int smem = static_cast<int>(tb::smem_bytes<S, T>());
    cudaError_t e = cudaFuncSetAttribute(tb::pm_tb_kernel<S, T, COND_EXP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tb::pm_tb_kernel<S, T, COND_RAT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <int T>
TbShape tb_shape_one()
{
    constexpr int S = AFD_TB_STORE;
    TbShape sh;
    sh.tx = tb::Geom<T>::TX;
    sh.ty = tb::Geom<T>::TY;
    sh.box_w = tb::Ring<S, T>::W;
    sh.box_h = tb::Ring<S, T>::H;
    sh.hx = tb::Ring<S, T>::HX;
    sh.threads = tb::Geom<T>::THREADS;
    sh.smem = tb::smem_bytes<S, T>();
    return sh;
}

}  // namespace

cudaError_t AFD_TB_FN(prepare)(int T)
{
    switch (T) {
    case 1: return tb_prepare_one<1>();
    case 2: return tb_prepare_one<2>();
    case 4: return tb_prepare_one<4>();
    case 8: return tb_prepare_one<8>();
    }
    return cudaErrorInvalidValue;
}

TbShape AFD_TB_FN(shape)(int T)
{
    switch (T) {
    case 1: return tb_shape_one<1>();
    case 2: return tb_shape_one<2>();
    case 4: return tb_shape_one<4>();
    default: return tb_shape_one<8>();
    }
}

cudaError_t AFD_TB_FN(launch)(int T, int cond, const CUtensorMap &tmap, void *out, int nx, int ny,
                              int nz, const Coef &k, const TbPlan &plan, int *err,
                              cudaStream_t stream)
{
#define AFD_TB_CASE(TT)                                                                           \
    case TT:                                                                                      \
        return cond == COND_EXP                                                                   \
                   ? tb_launch_one<TT, COND_EXP>(tmap, out, nx, ny, nz, k, plan, err, stream)     \
                   : tb_launch_one<TT, COND_RAT>(tmap, out, nx, ny, nz, k, plan, err, stream);
    switch (T) {
        AFD_TB_CASE(1)
        AFD_TB_CASE(2)
        AFD_TB_CASE(4)
        AFD_TB_CASE(8)
    }
#undef AFD_TB_CASE
    return cudaErrorInvalidValue;
}

}  // namespace afd
