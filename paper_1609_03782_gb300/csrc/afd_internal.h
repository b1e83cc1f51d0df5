// Internal launcher interface between the C ABI (afd_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "afd_math.cuh"

namespace afd {

// ---- one voxel per thread (any nx, any alignment) -------------------------
cudaError_t launch_pm_simple(int cond, const float *in, float *out, int nx, int ny, int nz,
                             const Coef &k, cudaStream_t stream);

// ---- TMA-staged x-y tiles streamed along z (nx % 4 == 0, 16-B aligned) ----
constexpr int kStreamTX = 64;   // interior tile width  (16 threads x 4 voxels)
constexpr int kStreamTY = 32;   // interior tile height (16 threads x 2 rows)
#ifndef AFD_STREAM_SLOTS
#define AFD_STREAM_SLOTS 8
#endif
#ifndef AFD_STREAM_MIN_BLOCKS
#define AFD_STREAM_MIN_BLOCKS 2
#endif
constexpr int kStreamSlots = AFD_STREAM_SLOTS;          // planes in the smem ring
constexpr int kStreamMinBlocks = AFD_STREAM_MIN_BLOCKS; // CTAs per SM to fit
constexpr int kStreamConsumerWarps = 8;
constexpr int kStreamThreads = kStreamConsumerWarps * 32 + 32;  // + 1 producer warp

struct StreamPlan {
    int tiles_x, tiles_y, tiles_z;  // tile grid
    int zc;                          // planes per z-chunk
    int64_t ntiles;
    int grid;                        // persistent CTAs
};

size_t pm_stream_smem_bytes();
cudaError_t pm_stream_prepare();  // one-time kernel attributes
cudaError_t pm_stream_occupancy(int *blocks_per_sm);
StreamPlan pm_stream_plan(int nx, int ny, int nz, int sm_count, int blocks_per_sm, int zc_hint);
cudaError_t launch_pm_stream(int cond, const CUtensorMap &tmap_in, float *out, int nx, int ny,
                             int nz, const Coef &k, const StreamPlan &plan, int *err,
                             cudaStream_t stream);

// ---- FP64 statistics -------------------------------------------------------
constexpr int kStatsThreads = 256;
// partials: 4 doubles per block; out4: sum, sum sq, negative sum sq, count
cudaError_t launch_stats(const float *x, int64_t n, double *partials, int nblocks, double *out4,
                         cudaStream_t stream);

// ---- diagnostics -----------------------------------------------------------
cudaError_t launch_selftest_wait(uint64_t limit_ns, int *err, cudaStream_t stream);

}  // namespace afd
