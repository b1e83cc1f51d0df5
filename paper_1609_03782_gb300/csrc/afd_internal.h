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
// Registers per thread for kStreamMinBlocks CTAs per SM: the warps are spread
// over the SM's four 16K-register quarters, so the quarter with the most
// warps sets the limit (allocated in multiples of 8).
constexpr int kStreamWarpsPerQuarter = (kStreamMinBlocks * (kStreamThreads / 32) + 3) / 4;
constexpr int kStreamMaxRegs = 16384 / (32 * kStreamWarpsPerQuarter) / 8 * 8 > 248
                                   ? 248
                                   : 16384 / (32 * kStreamWarpsPerQuarter) / 8 * 8;

// z-chunks of the streaming kernel: nuni chunks of zlen (+1 for the first
// zrem) planes from z = 0, then nlev chunks starting at off[0..nlev-1] (and
// off[nlev] = nz).
constexpr int kStreamMaxLevels = 64;
struct ZLevels {
    int nuni, zlen, zrem;
    int nlev;
    int off[kStreamMaxLevels + 1];
};

struct StreamPlan {
    int tiles_x, tiles_y, tiles_z;  // tile grid (tiles_z = number of z-chunks)
    int zc;                          // planes of the longest z-chunk
    int64_t ntiles;
    int grid;                        // persistent CTAs
    ZLevels lv;
    // launch as a programmatic dependent of the previous kernel in the stream
    // (only when that kernel is a streaming pass: its CTAs then overlap that
    // pass's last tiles)
    bool pdl;
    // coefficients in device memory (null: the Coef argument of the launch)
    const Coef *kdev;
};

// Tiles are handed out through a 64-bit counter in device memory: zero it
// (cudaMemsetAsync) before a sequence of launches, pass base = the sum of
// ntiles of the launches before this one in the sequence.

size_t pm_stream_smem_bytes();
cudaError_t pm_stream_prepare();  // one-time kernel attributes
cudaError_t pm_stream_occupancy(int *blocks_per_sm);
StreamPlan pm_stream_plan(int nx, int ny, int nz, int sm_count, int blocks_per_sm, int zc_hint,
                          int tile_x = kStreamTX, int tile_y = kStreamTY, int zmax = 32);

// The planes [z0, z1) of z-chunk tz of a plan's ZLevels.
__host__ __device__ inline void zchunk(const ZLevels &lv, int tz, int &z0, int &z1)
{
    if (tz < lv.nuni) {
        z0 = tz * lv.zlen + (tz < lv.zrem ? tz : lv.zrem);
        z1 = z0 + lv.zlen + (tz < lv.zrem ? 1 : 0);
    } else {
        z0 = lv.off[tz - lv.nuni];
        z1 = lv.off[tz - lv.nuni + 1];
    }
}
cudaError_t launch_pm_stream(int cond, const CUtensorMap &tmap_in, float *out, int nx, int ny,
                             int nz, const Coef &k, const StreamPlan &plan,
                             unsigned long long *ctr, unsigned long long base, int *err,
                             cudaStream_t stream);
// Any storage kind (StoreKind); the map's box is pm_stream_box(S, ...).
cudaError_t launch_pm_stream_s(int S, int cond, const CUtensorMap &tmap_in, void *out, int nx,
                               int ny, int nz, const Coef &k, const StreamPlan &plan,
                               unsigned long long *ctr, unsigned long long base, int *err,
                               cudaStream_t stream);
void pm_stream_box(int S, int *box_w, int *box_h, int *hx);

// ---- the float32 pass sequence (passes.cu) ---------------------------------
// n_iter >= 1 passes in -> ... -> out.  Pass i reads pass_src(i) and writes
// pass_dst(i).  Out of place (in != out) the destinations alternate between
// out and scratch so that the last pass lands in out; in place they
// alternate starting with scratch, and an odd count ends in scratch
// (passes_finish then copies the result to out).
struct PassSeq {
    int kind;              // conductance kind (CondKind)
    const float *in;
    float *out;
    float *scratch;        // a cube-sized buffer other than in and out
    int nx, ny, nz;
    Coef k;                // coefficients (ignored where plan.kdev is set)
    int n_iter;
    cudaStream_t stream;
    uint64_t *launches;    // incremented per launch (may be null)
};
float *pass_dst(const float *in, float *out, float *scratch, int n_iter, int i);
const float *pass_src(const float *in, float *out, float *scratch, int n_iter, int i);
// Streaming passes; maps[0..2]: the TMA maps of in, out and scratch.  The
// tile counter ctr must be zero before the first call of a sequence; *base is
// advanced by plan.ntiles per launch.  Pass 0 is an ordinary launch, the
// others are programmatic dependents of the pass before.
cudaError_t stream_passes(const PassSeq &q, const CUtensorMap maps[3], const StreamPlan &plan,
                          unsigned long long *ctr, unsigned long long *base, int *err);
// One-voxel-per-thread passes (any nx, any alignment).
cudaError_t simple_passes(const PassSeq &q);
// Copy the last pass's result to out if it is not there already.
cudaError_t passes_finish(const PassSeq &q);

// ---- 2-byte depth-1 pass with 8 x 2 voxels per thread (pm_wide.cu) --------
// 128 x (4 x consumer warps) column tiles, the same persistent-CTA / tile-counter / z-chunk
// scheme as the streaming kernel (plan: pm_stream_plan with these tiles);
// nx a multiple of 8, 16-byte aligned pointers.
#ifndef AFD_WIDE_WARPS
#define AFD_WIDE_WARPS 4  // consumer warps per CTA (each covers 4 rows)
#endif
#ifndef AFD_WIDE_SLOTS
#define AFD_WIDE_SLOTS 8
#endif
#ifndef AFD_WIDE_CTAS
#define AFD_WIDE_CTAS 3  // CTAs per SM the register cap is sized for
#endif
constexpr int kWideConsumerWarps = AFD_WIDE_WARPS;
constexpr int kWideTX = 128;
constexpr int kWideTY = 4 * kWideConsumerWarps;
constexpr int kWideSlots = AFD_WIDE_SLOTS;
constexpr int kWideThreads = kWideConsumerWarps * 32 + 32;
// registers per thread for AFD_WIDE_CTAS CTAs per SM (the SM's four 16K
// register quarters each hold a quarter of the warps, rounded up)
constexpr int kWideWarpsPerQuarter = (AFD_WIDE_CTAS * (kWideThreads / 32) + 3) / 4;
constexpr int kWideMaxRegs = 16384 / (32 * kWideWarpsPerQuarter) / 8 * 8 > 248
                                 ? 248
                                 : 16384 / (32 * kWideWarpsPerQuarter) / 8 * 8;
// Shared-memory slot of the kernel per storage kind: one TMA box of the
// largest tile shape the kernel is given.
constexpr int wide_slot_round(int b) { return (b + 127) / 128 * 128; }
constexpr int wide_slot_bytes(int S)
{
    // at least the single-cube box (the tile, a one-row y halo, a 16-byte x
    // halo); no less than 10752 / 6400 bytes, so narrow batch cubes get tall
    // tiles
    return S == 0 ? (wide_slot_round((kWideTX + 8) * (kWideTY + 2) * 4) > 10752
                         ? wide_slot_round((kWideTX + 8) * (kWideTY + 2) * 4)
                         : 10752)
                  : (wide_slot_round((kWideTX + 16) * (kWideTY + 2) * 2) > 6400
                         ? wide_slot_round((kWideTX + 16) * (kWideTY + 2) * 2)
                         : 6400);
}
size_t pm_wide_smem_bytes(int S);
// TMA box (elements, rows) of the single-cube tiles; x starts at x0 - 16/es
void pm_wide_box(int S, int *box_w, int *box_h);
// A batch cube's tile shape: tile columns of at most 128 voxels and equal
// width (a multiple of 8), as many rows as the CTA's threads cover at that
// width (within one slot): narrow cubes get one tall tile column.
void pm_wide_shape(int S, int nx, int *tx, int *ty, int *tiles_x);
cudaError_t pm_wide_prepare();
cudaError_t pm_wide_occupancy(int *blocks_per_sm);
cudaError_t launch_pm_wide(int S, int cond, const CUtensorMap &tmap_in, void *out, int nx, int ny,
                           int nz, const Coef &k, const StreamPlan &plan, unsigned long long *ctr,
                           unsigned long long base, int *err, cudaStream_t stream);
// The ends of a chain of one-iteration passes: a 2-byte cube in, float32
// out (S 2-byte, SO = STORE_F32), or float32 in, 2-byte out (S = STORE_F32);
// exponential or rational conductance.  The TMA map is over the input, with
// pm_wide_box(S, ...).
cudaError_t launch_pm_wide_chain_end(int S, int SO, int cond, const CUtensorMap &tmap_in,
                                     void *out, int nx, int ny, int nz, const Coef &k,
                                     const StreamPlan &plan, unsigned long long *ctr,
                                     unsigned long long base, int *err, cudaStream_t stream);

// ---- two iterations per pass, 8 x 2 voxels per thread (pm_wide2.cu) ---------
// afd_filter_ex's passes of depth 2 and more under AFD_KERNEL_TWO_STAGE:
// input format S, output format SO, either equal or one of them float32 (a
// chain 2-byte -> float32 -> ... -> 2-byte is one pass of depth 2 x links).
// 128 x kWide2TY output tiles; a TMA box of 144 x (kWide2TY + 4) input
// elements around the tile (x starts at x0 - 8, y at y0 - 2); nx a multiple
// of 8, 16-byte aligned pointers.  Plan: pm_stream_plan with these tiles.
#ifndef AFD_WIDE2_TY
#define AFD_WIDE2_TY 28  // 8 stage-1 + 7 stage-2 + 1 producer warps: 16 x 32 x 128 registers
#endif
#ifndef AFD_WIDE2_SLOTS
#define AFD_WIDE2_SLOTS 4
#endif
#ifndef AFD_WIDE2_CTAS
#define AFD_WIDE2_CTAS 1
#endif
#ifndef AFD_WIDE2_P1
#define AFD_WIDE2_P1 4
#endif
constexpr int kWide2TX = 128;
constexpr int kWide2TY = AFD_WIDE2_TY;
// stage 2: one 8 x 2 block per thread over the tile; stage 1: one block per
// thread over the tile grown by one voxel (17 x (TY/2 + 1) blocks)
constexpr int kWide2S2Warps = (kWide2TX / 8) * (kWide2TY / 2) / 32;
constexpr int kWide2S1Warps = ((kWide2TX / 8 + 1) * (kWide2TY / 2 + 1) + 31) / 32;
constexpr int kWide2Slots = AFD_WIDE2_SLOTS;
constexpr int kWide2P1 = AFD_WIDE2_P1;  // stage-1 plane ring
constexpr int kWide2Threads = (kWide2S1Warps + kWide2S2Warps + 1) * 32;  // + 1 producer warp
constexpr int kWide2WarpsPerQuarter = (AFD_WIDE2_CTAS * (kWide2Threads / 32) + 3) / 4;
constexpr int kWide2MaxRegs = 16384 / (32 * kWide2WarpsPerQuarter) / 8 * 8 > 248
                                  ? 248
                                  : 16384 / (32 * kWide2WarpsPerQuarter) / 8 * 8;
void pm_wide2_box(int *box_w, int *box_h);
cudaError_t pm_wide2_prepare();
cudaError_t pm_wide2_occupancy(int *blocks_per_sm);
cudaError_t launch_pm_wide2(int S, int SO, int cond, const CUtensorMap &tmap_in, void *out,
                            int nx, int ny, int nz, const Coef &k, const StreamPlan &plan,
                            unsigned long long *ctr, unsigned long long base, int *err,
                            cudaStream_t stream);

// ---- a resident batch of cubes (streaming kernel over many cubes) ---------
// Per-cube descriptor in device memory.  Roles: 0 input (resident), 1 result,
// 2 scratch.  Rows are padded to `px` elements (a multiple of 16 bytes), which
// is all the TMA needs, so any nx is streamed.
struct BatchDesc {
    CUtensorMap map[3];   // TMA descriptors of the three role buffers (64 x 32 tiles)
    CUtensorMap mapw[3];  // the same buffers with this cube's wide-kernel box
    void *buf[3];         // role buffers of this cube (storage format)
    int64_t px;           // row pitch in elements
    int nx, ny, nz;
    int tiles_x, tiles_y, zc;
    int wtx, wty, wtiles_x, wtiles_y;  // wide-kernel tile shape and grid (pm_wide_shape)
    Coef coef;  // per-call coefficients, written on the device
    float K;    // K of the last call, value units
};

// roles: null (all descriptors use src_role/dst_role) or per-descriptor
// (src, dst) pairs in device memory.  ctr: null (the list is dealt
// round-robin) or a tile counter, as for launch_pm_stream.  pdl: launch as a
// programmatic dependent (only after another pm_step_batch launch).
cudaError_t launch_pm_batch(int S, int cond, const BatchDesc *desc, const int2 *list,
                            const int2 *roles, int64_t ntiles, int src_role, int dst_role, int grid,
                            unsigned long long *ctr, unsigned long long base, bool pdl, int *err,
                            cudaStream_t stream);

// The same over the batch's per-cube wide tiles (pm_wide.cu): the list holds
// (cube, tile) pairs numbered over each cube's wtiles_x x wtiles_y x z-chunks.
cudaError_t launch_pm_wide_batch(int S, int cond, const BatchDesc *desc, const int2 *list,
                                 const int2 *roles, int64_t ntiles, int src_role, int dst_role,
                                 int grid, unsigned long long *ctr, unsigned long long base,
                                 bool pdl, int *err, cudaStream_t stream);

// ---- temporally blocked kernel (T iterations per pass, any storage) --------
struct TbShape {
    int tx, ty;          // interior tile
    int box_w, box_h;    // TMA box (elements, rows)
    int hx;              // TMA box starts at x0 - hx, y0 - T
    int threads;         // threads per CTA
    size_t smem;         // dynamic shared memory per CTA
};

struct TbPlan {
    int tiles_x, tiles_y, zc;
    int64_t ntiles;
    int grid;
};

// Dispatch on storage kind S (StoreKind) and depth T in {1, 2, 4, 8}.
bool tb_depth_ok(int T);
cudaError_t tb_prepare(int S, int T);
TbShape tb_shape(int S, int T);
TbPlan tb_plan(int S, int T, int nx, int ny, int nz, int sm_count, int zc_hint);
cudaError_t tb_launch(int S, int T, int cond, const CUtensorMap &tmap, void *out, int nx, int ny,
                      int nz, const Coef &k, const TbPlan &plan, int *err, cudaStream_t stream);

#define AFD_TB_DECL(n)                                                                           \
    cudaError_t tb_prepare_##n(int T);                                                           \
    TbShape tb_shape_##n(int T);                                                                 \
    cudaError_t tb_launch_##n(int T, int cond, const CUtensorMap &tmap, void *out, int nx,       \
                              int ny, int nz, const Coef &k, const TbPlan &plan, int *err,       \
                              cudaStream_t stream);
AFD_TB_DECL(f32)
AFD_TB_DECL(f16)
AFD_TB_DECL(bf16)
AFD_TB_DECL(i16)
#undef AFD_TB_DECL

// ---- storage conversion (a2 quantise, a7 dequantise) -----------------------
// units = storage units per value unit (a power of two); quantise computes
// store(v * units), dequantise load(q) / units, elementwise over n values.
cudaError_t launch_quantize(int S, const float *in, void *out, int64_t n, float units,
                            cudaStream_t stream);
cudaError_t launch_dequantize(int S, const void *in, float *out, int64_t n, float units,
                              cudaStream_t stream);

// ---- FP64 statistics -------------------------------------------------------
constexpr int kStatsThreads = 256;
// partials: 4 doubles per block; out4: sum, sum sq, negative sum sq, count
// Box / Gaussian smoothing (normalised correlation).  Separable weights:
// wx[0..2rx], wy[0..2ry], wz[0..2rz] (offset k - r).
constexpr int kSepMaxR = 24;   // x and y radius of the separable kernel
constexpr int kSepMaxRz = 12;  // z radius (a template parameter)
struct SepWeights {
    float wx[2 * kSepMaxR + 1], wy[2 * kSepMaxR + 1], wz[2 * kSepMaxRz + 1];
    int rx, ry, rz;
};
cudaError_t launch_smooth_sep(const float *in, float *out, int nx, int ny, int nz,
                              const SepWeights &w, int *err, cudaStream_t stream);
// Direct correlation with W (device, x fastest) of (2rx+1)(2ry+1)(2rz+1).
// wsum: the total weight (the divisor of voxels whose window is inside).
// W: the (2rz+1)(2ry+1)(2rx+1) weights, x fastest; S: their FP64 prefix
// sums, (2rz+2)(2ry+2)(2rx+2) with S[k][j][i] = sum over dz < k, dy < j,
// dx < i (the in-cube weight of a voxel near a face, by inclusion-exclusion)
cudaError_t launch_smooth_direct(const float *in, float *out, int nx, int ny, int nz,
                                 const float *W, const double *S, int rx, int ry, int rz,
                                 float wsum, int *err, cudaStream_t stream);
size_t smooth_direct_smem(int rx, int ry, int rz);  // bytes of shared memory it needs
// The separable pass with TMA-streamed planes: nx % 4 == 0, 16-byte aligned
// cubes.  tmap: 3-D float32 map over the input with the box of
// smooth_tma_box (x halo hx, a multiple of 4 >= rx).
void smooth_tma_box(int rx, int ry, int *box_w, int *box_h, int *hx);
size_t smooth_tma_smem(int ry, int hx, int rz);
cudaError_t launch_smooth_sep_tma(const CUtensorMap &tmap, float *out, int nx, int ny, int nz,
                                  const SepWeights &w, int hx, int *err, cudaStream_t stream);
// F diagnostic sums over the ROI box roi = {x0, x1, y0, y1, z0, z1} of cubes
// with row pitch nx and ny rows per plane: out6 = {S_of, S_oo, S_mf, S_m, N_o,
// N_f} (device doubles; im may be null).  t_o, t_f: float thresholds already
// rounded up from nsig x rms.  part: nblocks x 6 doubles of scratch.
cudaError_t launch_fdiag(const float *io, const float *iff, const float *im, int64_t nx,
                         int64_t ny, const int roi[6], float t_o, float t_f, double *part,
                         int nblocks, double *out6, cudaStream_t stream);
// Noise-relative coefficients: from launch_stats' out4, K = k_rms x rms
// (rms of the negative voxels) and the coefficients of conductance `kind`
// into *coef (device); A on the device, the B terms taken from b (host
// make_coef).  K_out (device, may be null) receives K.
cudaError_t launch_rel_coef(const double *out4, double k_rms, int kind, double dt, const double h[3],
                            const Coef &b, Coef *coef, float *K_out, cudaStream_t stream);
cudaError_t launch_stats(const float *x, int64_t n, double *partials, int nblocks, double *out4,
                         cudaStream_t stream);

// ---- diagnostics -----------------------------------------------------------
cudaError_t launch_selftest_wait(uint64_t limit_ns, int *err, cudaStream_t stream);

}  // namespace afd
