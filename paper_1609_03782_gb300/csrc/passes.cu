// The float32 iteration driver's pass sequence (Sec. 3.3: n evaluations of
// the explicit update, each reading only the previous iterate; two buffers,
// Sec. 6), shared by the context entry points (afd_filter, afd_filter_out,
// afd_filter_rel, afd_filter_intensity, afd_filter_host) and by
// afd_filter_noalloc, so that both run exactly the same launches.
#include "afd_internal.h"
#include "afd_trace.h"

namespace afd {

float *pass_dst(const float *in, float *out, float *scratch, int n_iter, int i)
{
    if (in == out)
        return (i & 1) ? out : scratch;
    return ((n_iter - 1 - i) & 1) ? scratch : out;
}

const float *pass_src(const float *in, float *out, float *scratch, int n_iter, int i)
{
    return i == 0 ? in : pass_dst(in, out, scratch, n_iter, i - 1);
}

cudaError_t stream_passes(const PassSeq &q, const CUtensorMap maps[3], const StreamPlan &plan,
                          unsigned long long *ctr, unsigned long long *base, int *err)
{
    cudaError_t e = cudaSuccess;
    const int np = q.n_iter;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
        const float *src = pass_src(q.in, q.out, q.scratch, np, i);
        const int m = (src == q.in) ? 0 : (src == q.out ? 1 : 2);
        const afd_host::TraceRange pass_trace("pass");
        StreamPlan pl = plan;
        pl.pdl = i > 0;
        e = launch_pm_stream(q.kind, maps[m], pass_dst(q.in, q.out, q.scratch, np, i),
                             q.nx, q.ny, q.nz, q.k, pl, ctr, *base, err, q.stream);
        *base += static_cast<unsigned long long>(plan.ntiles);
        if (q.launches)
            ++*q.launches;
    }
    return e;
}

cudaError_t simple_passes(const PassSeq &q)
{
    cudaError_t e = cudaSuccess;
    const int np = q.n_iter;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
        e = launch_pm_simple(q.kind, pass_src(q.in, q.out, q.scratch, np, i),
                             pass_dst(q.in, q.out, q.scratch, np, i), q.nx, q.ny, q.nz,
                             q.k, q.stream);
        if (q.launches)
            ++*q.launches;
    }
    return e;
}

cudaError_t passes_finish(const PassSeq &q)
{
    float *last = pass_dst(q.in, q.out, q.scratch, q.n_iter, q.n_iter - 1);
    if (last == q.out)
        return cudaSuccess;
    const size_t bytes = static_cast<size_t>(q.nx) * q.ny * q.nz * sizeof(float);
    return cudaMemcpyAsync(q.out, last, bytes, cudaMemcpyDeviceToDevice, q.stream);
}

}  // namespace afd
