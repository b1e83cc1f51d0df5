// The library context (opaque to callers) and the host helpers shared by the
// translation units that implement the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/afd.h"
#include "afd_math.cuh"

struct afd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int stream_bps = 0;          // streaming kernel CTAs per SM (occupancy)
    int wide_bps = 0;            // 2-byte 8 x 2-voxel kernel CTAs per SM (occupancy)
    int wide2_bps = 0;           // two-iteration kernel CTAs per SM (occupancy)
    int zc_hint = 0;             // streaming kernel z-chunk override (0 = auto)
    afd_kernel kernel = AFD_KERNEL_AUTO;
    int *d_err = nullptr;        // device error word (bounded-wait expiries)
    unsigned long long *d_tiles = nullptr;  // streaming kernel tile counter (in d_err's block)
    unsigned long long tiles_base = 0;      // counter value at the next launch's start
    float *scratch = nullptr;    // ping-pong partner buffer
    size_t scratch_bytes = 0;
    // afd_filter_host(_async): two staging slots (device copies of the input
    // and of the result) so that one call's copies overlap another's passes
    struct HostSlot {
        float *buf = nullptr;  // input, then result (2 x the cube)
        size_t bytes = 0;
        cudaEvent_t copied_in = nullptr;   // the H2D copy of the input is done
        cudaEvent_t filtered = nullptr;    // the passes are done
        cudaEvent_t copied_out = nullptr;  // the D2H copy of the result is done
    } host_slot[2];
    unsigned long long host_calls = 0;
    cudaStream_t h2d_stream = nullptr;  // host -> device copies
    cudaStream_t d2h_stream = nullptr;  // device -> host copies
    float *lp_scratch = nullptr; // ping-pong partner of afd_filter_ex (any storage)
    size_t lp_scratch_bytes = 0;
    float *chain_f32 = nullptr;  // two float32 cubes: the links of afd_filter_ex's deep passes
    size_t chain_f32_bytes = 0;
    float *fb_scratch = nullptr; // float32 pair for the afd_filter_ex fallback
    size_t fb_scratch_bytes = 0;
    bool tb_ready[4][9] = {};    // tb_prepare done, per storage kind and depth
    double *d_part = nullptr;    // stats partials
    int part_blocks = 0;
    double *d_out4 = nullptr;    // stats result (device)
    afd::Coef *d_coef = nullptr; // coefficients computed on the device (afd_filter_rel)
    float *fd_buf = nullptr;     // F diagnostic: block partials + result (doubles)
    size_t fd_bytes = 0;
    double *h_out4 = nullptr;    // stats result (pinned host)
    uint64_t launches = 0;
    // pass timing (afd_pass_timing): event pairs around each pass sequence
    bool timing = false;
    std::vector<cudaEvent_t> tev;  // begin, end, begin, end, ...
    int64_t timed_passes = 0;
    char errstr[256] = {0};
};


namespace afd_host {

afd_status cuda_fail(afd_ctx *ctx, cudaError_t e);
afd_status device_alloc(afd_ctx *ctx, void **p, size_t bytes);
afd_status set_device(afd_ctx *ctx);
bool dims_ok(int64_t nx, int64_t ny, int64_t nz);
bool params_ok(const float *spacing, float K, float dt, int n_iter, afd_conductance cond);
bool pow2_scale_ok(float scale);
bool storage_ok(int s);
afd_status encode_box_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int box_w,
                          int box_h, int nx, int ny, int nz);
// As encode_box_map, with an explicit row pitch in elements (>= nx).
afd_status encode_pitched_map(afd_ctx *ctx, CUtensorMap *map, const void *ptr, int S, int box_w,
                              int box_h, int nx, int ny, int nz, int64_t pitch);

}  // namespace afd_host
