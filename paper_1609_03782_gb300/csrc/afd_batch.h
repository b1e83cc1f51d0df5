// The resident batch (opaque to callers), shared with the serving engine.
#pragma once

#include <cstdint>
#include <vector>

#include "afd_ctx.h"
#include "afd_internal.h"

struct afd_batch {
    afd_ctx *ctx = nullptr;
    int count = 0;
    int S = 0;
    float scale = 1.0f;
    double units = 1.0;  // storage units per value unit
    std::vector<int64_t> nx, ny, nz, px, off;  // off: element offset of each cube
    int64_t total = 0;                          // elements per role
    void *arena[3] = {nullptr, nullptr, nullptr};
    std::vector<afd::BatchDesc> h_desc;
    afd::BatchDesc *d_desc = nullptr;
    int2 *d_list = nullptr;
    int64_t ntiles = 0;
    int zc = 0;  // 0 = automatic
    int grid = 0;
    int bpc = 8;                 // stats blocks per cube
    double *d_part = nullptr;    // stats partials: count * bpc * 4
    float *d_kin = nullptr;      // K requests (device), count
    float *h_kin = nullptr;      // pinned staging of the K requests
    float *d_kout = nullptr;     // K used, count
    cudaStream_t cap = nullptr;  // private capture stream
    cudaGraphExec_t exec = nullptr;
    // parameters the captured graph was built for
    int g_n = -1, g_cond = -1, g_kind = -1;
    float g_dt = 0.0f, g_h[3] = {0, 0, 0};
    int g_zc = -1;
};

