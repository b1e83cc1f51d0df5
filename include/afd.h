/*
 * afd.h — C ABI of the GB300 (sm_103a) anisotropic-diffusion library.
 *
 * The library filters 3-D H I spectral-line cubes with the gradient
 * anisotropic-diffusion (Perona-Malik) filter of Punzo, van der Hulst &
 * Roerdink, arXiv:1609.03782, Sec. 3.3 (eq. "perona", the gradient
 * conductance printed after it, and the explicit n-step iteration that
 * follows).  All arithmetic runs in hand-written CUDA kernels; the signatures
 * below carry only plain pointers and sizes.
 *
 * Cube layout (every entry point): x fastest, element (x, y, z) at index
 * x + nx*(y + ny*z), z the velocity axis.  "Device pointer" means memory the
 * current CUDA context can address from the GPU (cudaMalloc, a torch CUDA
 * tensor); "host pointer" means ordinary or pinned host memory.
 *
 * One filter iteration, per voxel p and each of its six face neighbours q
 * along axis a with spacing h_a:
 *     d  = (I[q] - I[p]) / h_a
 *     I'[p] = I[p] + dt * sum_q g(d; K) * d / h_a
 * with g(d; K) = exp(-(d/K)^2) (AFD_COND_EXPONENTIAL) or 1/(1+(d/K)^2)
 * (AFD_COND_RATIONAL, the form printed in Sec. 3.3).  A face on the cube
 * boundary carries no flux; the update is synchronous (every voxel of step
 * i+1 reads step i only, the two-buffer memory model of Sec. 6); exactly
 * n_iter steps are taken.  K = 0 is the identity; K = +inf is the discrete
 * heat equation.
 *
 * Conventions shared by every entry point
 *   - Ordering: work is enqueued on the context's stream and runs
 *     asynchronously unless the entry point says it synchronises.  Argument
 *     errors are reported synchronously and enqueue nothing.
 *   - Errors: AFD_EINVAL for bad arguments (null pointers, sizes < 1, sizes
 *     whose byte count overflows int64, non-finite or non-positive spacing or
 *     dt, negative or NaN K, negative n_iter); AFD_ENOMEM when the library
 *     cannot allocate its scratch; AFD_ECUDA when a CUDA call fails (the
 *     CUDA error string is kept, see afd_last_error_string); AFD_ETIMEOUT
 *     when a kernel's bounded wait expired (reported by afd_sync).
 *   - Ownership: the caller owns every cube and output buffer it passes; the
 *     context owns its scratch memory and frees it in afd_destroy.
 *   - Threading: a context is not thread-safe; use one context per host
 *     thread.
 */
#ifndef AFD_H
#define AFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afd_ctx afd_ctx; /* opaque, owned by the library */

typedef enum {
    AFD_OK = 0,
    AFD_EINVAL = 1,
    AFD_ENOMEM = 2,
    AFD_ECUDA = 3,
    AFD_ETIMEOUT = 4,
    AFD_EBUSY = 5
} afd_status;

/* Edge-stopping conductance g(d; K) (Sec. 3.3). */
typedef enum {
    AFD_COND_EXPONENTIAL = 0, /* exp(-(d/K)^2)                              */
    AFD_COND_RATIONAL = 1     /* 1/(1+(d/K)^2), the paper's printed form    */
} afd_conductance;

/* Storage format of a cube (precision line).  The 2-byte formats hold
 * value/scale with a power-of-two per-cube scale, rounded to nearest even. */
typedef enum {
    AFD_F32 = 0,    /* float32                                              */
    AFD_F16 = 1,    /* IEEE binary16 of value/scale                        */
    AFD_BF16 = 2,   /* bfloat16 of value/scale                             */
    AFD_I16FIX = 3  /* int16 count of scale/1024 steps, clamped to +-32767 */
} afd_storage;

/* Kernel selection (tests and tuning; AUTO is the production choice). */
typedef enum {
    AFD_KERNEL_AUTO = 0,   /* streaming kernel when the layout allows it   */
    AFD_KERNEL_SIMPLE = 1, /* one voxel per thread, any layout             */
    AFD_KERNEL_STREAM = 2, /* TMA-staged x-y tiles streamed along z;
                              needs nx % 4 == 0 and a 16-byte aligned cube */
    AFD_KERNEL_TWO_STAGE = 3 /* as AUTO, but afd_filter_ex's deep passes run
                                on the two-iteration kernel */
} afd_kernel;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * the context enqueues on (NULL: the legacy default stream of the device).
 * *out receives the context.  Allocates a few bytes of device memory (the
 * context's error word).  AFD_EINVAL if out is NULL or the device does not
 * exist; AFD_ECUDA if the device cannot be initialised. */
afd_status afd_create(afd_ctx **out, int device, void *cuda_stream);

/* Free the context's scratch and the context itself after waiting for its
 * stream.  NULL is accepted and returns AFD_OK. */
afd_status afd_destroy(afd_ctx *ctx);

/* Change the stream later calls enqueue on. */
afd_status afd_set_stream(afd_ctx *ctx, void *cuda_stream);

/* Choose the kernel family used by afd_filter (default AFD_KERNEL_AUTO).
 * AFD_KERNEL_STREAM on a cube it cannot handle makes afd_filter return
 * AFD_EINVAL.  For afd_filter_ex's depth-1 passes on 2-byte storage, AUTO
 * runs the 8 x 2-voxel-per-thread streaming kernel and STREAM the 4 x 2 one;
 * for its passes of depth 2, 4 and 8 (nx a multiple of 8), AUTO runs chains
 * of one-iteration launches (storage -> float32 -> ... -> storage),
 * TWO_STAGE chains of the two-iteration 8 x 2 kernel, and STREAM the general
 * temporally blocked kernel.  All kernels give bit-identical results. */
afd_status afd_set_kernel(afd_ctx *ctx, afd_kernel kernel);

/* Tuning knob of the streaming kernel: the largest number of z planes one
 * CTA streams per tile; the cube is cut into chunks of equal length (+-1)
 * no longer than zc.  0 = automatic: a guided sequence from the cube shape
 * and the device's SM count, long chunks first and short ones last (tiles
 * are handed to the CTAs dynamically).  Results do not depend on it.
 * AFD_EINVAL if zc < 0. */
afd_status afd_set_stream_zchunk(afd_ctx *ctx, int zc);

/* Filter a float32 cube in place (Sec. 3.3: n_iter explicit iterations of
 * the per-face scheme above).
 *   cube     DEVICE pointer, nx*ny*nz floats, caller-owned, overwritten with
 *            the result.
 *   spacing  HOST pointer to (hx, hy, hz) > 0, or NULL for unit spacing.
 *   K        conductance scale in the cube's intensity units (K = k*sigma for
 *            a noise level sigma); 0 gives the identity, +inf the heat
 *            equation.
 *   dt       step (the paper's tau) > 0.  Steps beyond the stability bound
 *            dt * sum_a 2/h_a^2 <= 1 are allowed (the paper's range reaches
 *            tau = 0.0625 for its own weights) but lose the maximum
 *            principle.
 *   n_iter   number of iterations >= 0; 0 is a no-op.
 * Uses 4*nx*ny*nz bytes of context scratch (allocated on first need, grown
 * when needed, kept until afd_destroy) for the second buffer of the
 * ping-pong; an odd n_iter ends with one device-to-device copy.
 * Asynchronous. */
afd_status afd_filter(afd_ctx *ctx, float *cube, int64_t nx, int64_t ny,
                      int64_t nz, const float *spacing, float K, float dt,
                      int n_iter, afd_conductance cond);

/* Out-of-place afd_filter: reads `in`, writes the result to `out` (both
 * DEVICE pointers to nx*ny*nz floats, caller-owned; `in` is not modified
 * unless in == out, which is the in-place afd_filter).  Iterations alternate
 * between `out` and context scratch so that the last one lands in `out`:
 * no extra copy for any n_iter.  n_iter = 0 or K = 0 copies in to out.
 * Asynchronous. */
afd_status afd_filter_out(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const float *spacing, float K, float dt, int n_iter,
                          afd_conductance cond);

/* afd_filter_out with K given in units of the input's noise level (Sec. 3.3
 * states K relative to the rms of the noise): K = k_rms x rms, rms the rms
 * of the negative voxels of `in` (as afd_noise_rms computes it), rounded to
 * float.  On the streaming kernel (nx % 4 == 0, 16-byte aligned cubes, kernel
 * not forced to SIMPLE) the statistics, K and the coefficients are computed
 * on the device and the call returns without waiting; otherwise the rms
 * takes a round trip through the host.  Either way the result is bit for bit
 * afd_filter_out's with that K.  K_out: DEVICE float receiving K (may be
 * NULL).  An input without negative voxels has rms 0: K = 0 and the result
 * equals the input.  AFD_EINVAL if k_rms is not finite and > 0, or as
 * afd_filter_out. */
afd_status afd_filter_rel(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const float *spacing, float k_rms, float dt, int n_iter,
                          afd_conductance cond, float *K_out);

/* The paper's own intensity-driven gradient filter (Sec. 3.3, the explicit
 * update after eq. "conductivepara"), out of place:
 *     I' = I + tau (C_x D_x + C_y D_y + C_z D_z) / (1 + I^2 / (K^2 rms^2))
 * with D_a = [I(a+1) - I] + [I(a-1) - I] the nearest-neighbour second
 * difference (a neighbour outside the cube adds nothing) and the conductance
 * taken once per voxel from its own intensity.  It does not conserve the
 * voxel sum (the paper notes the flux scale is not kept).
 *   in, out  DEVICE pointers to nx*ny*nz floats (in == out allowed).
 *   C        HOST pointer to (C_x, C_y, C_z), each >= 0 (paper range [0, 10]).
 *   K        >= 0, in units of rms (paper range [0.5, 10], default 1.5);
 *            K = 0 or rms = 0 is the identity, K * rms = +inf gives S = 1.
 *   rms      the cube's noise level (e.g. afd_noise_rms).
 *   tau      > 0 (paper range [0.0025, 0.0625], default 0.0325).
 *   n_iter   >= 0 (paper default 20).
 * Stable (no new extrema) for tau * 2 (C_x + C_y + C_z) <= 1.  Uses the
 * kernels of afd_filter; asynchronous. */
afd_status afd_filter_intensity(afd_ctx *ctx, const float *in, float *out, int64_t nx,
                                int64_t ny, int64_t nz, const float *C, float K, float rms,
                                float tau, int n_iter);

/* afd_filter with the cube in pageable or pinned HOST memory: copies host_in
 * to context-owned device memory, filters, and copies the result to
 * host_out (host_in == host_out is allowed).  Synchronous: returns after the
 * result is in host memory, so the timing of this call includes the
 * host<->device transfers, as the paper's GPU timings do (Sec. 6).  Uses
 * 8*nx*ny*nz bytes of context device memory (staging slot 0) besides the
 * filter's scratch. */
afd_status afd_filter_host(afd_ctx *ctx, const float *host_in, float *host_out, int64_t nx,
                           int64_t ny, int64_t nz, const float *spacing, float K, float dt,
                           int n_iter, afd_conductance cond);

/* afd_filter_host without waiting: enqueues the copy of host_in to the
 * device (on a context-owned copy stream), the n_iter passes (on the
 * context's stream) and the copy of the result to host_out (on a second
 * copy stream), and returns.  Consecutive calls alternate between two
 * staging slots of 8*nx*ny*nz device bytes each, so one call's copies run
 * while the previous call's passes do: a sequence of cubes then costs about
 * max(copies, passes) per cube instead of their sum.  host_in must stay
 * unchanged and host_out untouched until afd_sync(ctx) returns; page-locked
 * (pinned) buffers are needed for the overlap (pageable ones work, without
 * it).  Errors of the asynchronous work are reported by afd_sync. */
afd_status afd_filter_host_async(afd_ctx *ctx, const float *host_in, float *host_out, int64_t nx,
                                 int64_t ny, int64_t nz, const float *spacing, float K, float dt,
                                 int n_iter, afd_conductance cond);

/* afd_filter for a cube larger than the device memory it may use: the cube
 * stays in HOST memory and passes through the device in z-slabs of slab_nz
 * planes, in rounds of up to `halo` iterations.  An explicit nearest-
 * neighbour iteration (Sec. 3.3) moves information one plane per iteration,
 * so a slab loaded with `halo` extra planes on each side (fewer at the
 * cube's z faces, which are the true zero-flux faces) and filtered for
 * `halo` iterations holds the whole cube's result on its own planes: the
 * result is bit-identical to afd_filter on the whole cube.  Extends the
 * paper's memory model (Sec. 6: the cube in RAM, two cube-sized buffers in
 * DRAM) to device memory of 2 x 2 x (slab_nz + 2 halo) planes.
 *   host_in   the cube (x fastest); unchanged.  Pinned memory lets the copies
 *             overlap the passes (two staging slots on two copy streams).
 *   host_out  the result; must not be host_in.
 *   host_tmp  a cube-sized host buffer, used when n_iter > halo (the rounds
 *             alternate between it and host_out); may be NULL otherwise.
 *   slab_nz   >= 1 planes per slab; halo >= 1 iterations per round.
 * Host traffic per round: the cube in (plus 2 halo planes per slab) and
 * out.  Synchronous: returns when host_out holds the result.  Returns
 * AFD_EINVAL for bad arguments (nothing is done), else as afd_sync. */
afd_status afd_filter_slabs(afd_ctx *ctx, const float *host_in, float *host_out, float *host_tmp,
                            int64_t nx, int64_t ny, int64_t nz, const float *spacing, float K,
                            float dt, int n_iter, afd_conductance cond, int64_t slab_nz,
                            int halo);

/* afd_filter_intensity for a cube in HOST memory, through the device in
 * z-slabs as afd_filter_slabs: the paper's intensity-driven update (Sec.
 * 3.3, after eq. "conductivepara") also reaches one plane per iteration, so
 * the same ghost planes make the result bit-identical to
 * afd_filter_intensity on the whole cube.  It is also the paper's own GPU
 * protocol, the cube in from and out to RAM (Sec. 6), with the copies of one
 * slab overlapping the passes of another.
 *   host_in, host_out, host_tmp, slab_nz, halo   as afd_filter_slabs.
 *   C, K, rms, tau, n_iter                        as afd_filter_intensity.
 * Synchronous.  AFD_EINVAL for bad arguments (nothing is done), else as
 * afd_sync. */
afd_status afd_filter_intensity_slabs(afd_ctx *ctx, const float *host_in, float *host_out,
                                      float *host_tmp, int64_t nx, int64_t ny, int64_t nz,
                                      const float *C, float K, float rms, float tau, int n_iter,
                                      int64_t slab_nz, int halo);

/* Round a float32 cube into a 2-byte storage format (precision line): out[i]
 * = RN(in[i] / scale) in float16 or bfloat16, or RN(in[i] * 1024 / scale)
 * as int16 clamped to +-32767; nearest, ties to even.
 *   in       DEVICE pointer to n floats.
 *   out      DEVICE pointer to n 2-byte elements.
 *   storage  AFD_F16, AFD_BF16 or AFD_I16FIX (AFD_F32 is rejected).
 *   scale    the cube's power-of-two scale (> 0, finite; e.g. the power of
 *            two nearest the noise level), so the division is exact.
 * The paper argues float precision suffices for H I data (Sec. 6); the
 * 2-byte formats halve the bytes again.  Asynchronous; AFD_EINVAL for a
 * non-power-of-two scale or n < 1. */
afd_status afd_quantize(afd_ctx *ctx, const float *in, void *out, int64_t n,
                        afd_storage storage, float scale);

/* Inverse of afd_quantize: out[i] = stored value * scale (exact).  in: DEVICE
 * pointer to n 2-byte elements; out: DEVICE pointer to n floats.
 * Asynchronous. */
afd_status afd_dequantize(afd_ctx *ctx, const void *in, float *out, int64_t n,
                          afd_storage storage, float scale);

/* The filter on a cube in any storage format, with T = t_block iterations
 * between roundings to the storage format (temporal blocking).
 *   in, out   DEVICE pointers to nx*ny*nz elements of `storage` (in == out
 *             filters in place; other overlaps are rejected).
 *   storage   AFD_F32, AFD_F16, AFD_BF16 or AFD_I16FIX.
 *   scale     the cube's power-of-two scale (ignored for AFD_F32).
 *   K         in the cube's value units (value = stored value * scale).
 *   spacing, dt, n_iter, cond   as for afd_filter.
 *   t_block   1, 2, 4 or 8 (0 = 1: one iteration per pass on the
 *             streaming kernel, which on GB300 outruns every blocked depth;
 *             tune.Tuner.tune_filter_ex picks a depth by timing).
 * Each pass reads the stored cube, runs its iterations in float32 with the
 * arithmetic of afd_filter, and rounds the result once into the storage
 * format; n_iter = (n_iter / T) passes of depth T, the remainder as passes
 * of depth 4, 2, 1 (at most T).  A pass is bit-identical to dequantise ->
 * that many afd_filter iterations -> quantise; with AFD_F32 the whole call
 * is bit-identical to afd_filter_out.  How a pass runs (afd_set_kernel):
 * under AUTO, with nx a multiple of 8, a pass of depth T >= 2 is T
 * one-iteration launches whose intermediate cubes are float32 (storage ->
 * float32 -> ... -> storage: (2 b + 8 (T - 1)) / T bytes per voxel-iteration
 * for b-byte elements, e.g. 6 at depth 2 in 2 bytes; on GB300 these bytes
 * cost less than the instructions of a fused pass); under
 * AFD_KERNEL_TWO_STAGE, T/2 two-iteration launches ((2 b + 8 (T/2 - 1)) / T
 * bytes); under AFD_KERNEL_STREAM, or otherwise, one launch of the general
 * blocked kernel (2 b / T bytes).  Uses one cube of context scratch in the
 * storage format, plus two float32 cubes for passes of depth 2 or more under
 * AUTO and TWO_STAGE, or when nx * element size is not a multiple of 16
 * bytes or K = +inf (passes through float32 scratch).  Asynchronous. */
afd_status afd_filter_ex(afd_ctx *ctx, const void *in, void *out, afd_storage storage,
                         float scale, int64_t nx, int64_t ny, int64_t nz,
                         const float *spacing, float K, float dt, int n_iter,
                         afd_conductance cond, int t_block);

/* FP64 statistics of a float32 cube (noise level and conservation check).
 *   cube     DEVICE pointer to n floats.
 *   out4     DEVICE pointer to 4 doubles receiving, in this order:
 *            sum I, sum I^2, sum over I<0 of I^2, number of I<0.
 * Partial sums of 16 consecutive values are formed in float32 and every
 * partial is accumulated in double in a fixed order, so repeated calls give
 * bit-identical results.  Uses a few KB of context scratch.  Asynchronous. */
afd_status afd_stats(afd_ctx *ctx, const float *cube, int64_t n,
                     double *out4);

/* Noise level of a float32 cube, sqrt(sum_{I<0} I^2 / #{I<0}) in FP64: the
 * rms of the negative voxels (emission is positive, noise symmetric).  The
 * paper sets K in units of this noise level "rms" (Sec. 3.3).  0 when no
 * voxel is negative.  cube: DEVICE pointer; out: HOST pointer.
 * Synchronises the context's stream. */
afd_status afd_noise_rms(afd_ctx *ctx, const float *cube, int64_t n,
                         double *out);

/* FP64 sum of a float32 cube (conservation check: the per-face scheme moves
 * intensity between voxels and never creates it).  cube: DEVICE pointer;
 * out: HOST pointer.  Synchronises the context's stream. */
afd_status afd_sum(afd_ctx *ctx, const float *cube, int64_t n, double *out);

/* Wait for the context's stream and report the first asynchronous error:
 * AFD_ECUDA for a CUDA error, AFD_ETIMEOUT when a kernel's bounded wait
 * expired (the error word is then cleared). */
afd_status afd_sync(afd_ctx *ctx);

/* The box (mean) filter of Sec. 3.1: out(p) = the mean of the voxels of the
 * N[0] x N[1] x N[2] window centred on p that lie inside the cube (the
 * boundary rule is this library's reading: the paper states none; constants
 * stay constant).  N odd, N[0], N[1] <= 49, N[2] <= 25.  in, out: DEVICE
 * float32 cubes, distinct and not overlapping.  One fused pass on the
 * context's stream; asynchronous. */
afd_status afd_smooth_box(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                          int64_t nz, const int *N);

/* The Gaussian filter of Sec. 3.2: a normalised correlation (as
 * afd_smooth_box) with G = exp(-sum_i x_i^2 / (2 sigma_i^2)),
 * sigma_i = fwhm[i] / (2 sqrt(2 ln 2)), rotated by R = Rz Ry Rx (angles_deg
 * = {theta_x, theta_y, theta_z} in degrees; K(p) = G(R^T p)), truncated
 * where the kernel's ellipsoid passes `truncate` sigma along each axis
 * (radius ceil(truncate sqrt(Sigma_aa)), Sigma = R diag(sigma^2) R^T;
 * truncate 0 = 3).  angles_deg NULL or all zero: the separable fused pass
 * (radius <= 24 in x and y, <= 12 in z); otherwise a direct 3-D correlation
 * whose weights and plane ring must fit in shared memory (AFD_EINVAL if
 * not), preceded by a synchronous upload of the weights. */
afd_status afd_smooth_gauss(afd_ctx *ctx, const float *in, float *out, int64_t nx, int64_t ny,
                            int64_t nz, const float *fwhm, const float *angles_deg,
                            float truncate);

/* The paper's smoothing-quality diagnostic F (Sec. 4, eqs. "F_equa",
 * "Sequa", "Mfequa") and recovered-signal fraction F_M (Sec. 5, eq.
 * "sums_equa") of a filtered cube against its original, over a ROI box.
 *   masks:  M_o = [I_o >= nsig rms_o],  M_f = [I_f >= nsig rms_f]  (nsig = 3
 *           in the paper)
 *   sums (always of the ORIGINAL intensities, or of the model's):
 *           S_of = sum I_o M_f, S_oo = sum I_o M_o, S_mf = sum I_m M_f,
 *           S_m = sum I_m
 *   F = |S_of| / |S_oo|;  F_M = |S_mf| / |S_m| (NaN without a model);
 *   sigma_F = sqrt(s_of^2 / S_oo^2 + S_of^2 s_oo^2 / S_oo^4) with
 *           s_oi = sqrt(N_i / beam) rms_i, N_i the voxels in mask i and beam
 *           the voxels per independent element (1: uncorrelated noise). */
typedef struct {
    double S_of, S_oo, S_mf, S_m;
    int64_t N_o, N_f;
    double rms_o, rms_f; /* the noise levels used */
    double F, sigma_F, F_M;
} afd_fdiag;

/* orig, filt, model: DEVICE float32 cubes of one shape (model may be NULL).
 * roi: HOST array {x0, x1, y0, y1, z0, z1} (half-open, inside the cube; NULL
 * = the whole cube).  rms_o / rms_f <= 0: estimated as afd_noise_rms of the
 * full cube (Sec. 4 takes the rms constant over the cube).  The mask
 * decisions are exact (thresholds rounded up to the next float); the sums
 * are accurate to a few float32 ulps of the summed magnitudes.  Synchronous:
 * *out (HOST) is filled on return.  AFD_EINVAL for an empty or out-of-range
 * box, nsig not finite and > 0, beam < 1 or not finite, or a NaN/inf rms. */
afd_status afd_f_diagnostic(afd_ctx *ctx, const float *orig, const float *filt,
                            const float *model, int64_t nx, int64_t ny, int64_t nz,
                            const int64_t *roi, double rms_o, double rms_f, double nsig,
                            double beam, afd_fdiag *out);

/* Bounds checks (a debug build of the library compiled with -DAFD_CHECK):
 * the kernels check their hand-computed shared-memory and global indices,
 * skip an access that would fall outside its buffer and record the number
 * of such violations, the first one's code and its index.  This call
 * synchronises the context's stream, returns the record (HOST ints) and
 * clears it.  In the release build nothing is recorded: *count is 0.
 * afd_checked_build() is 1 in the checked build, else 0. */
afd_status afd_check_violations(afd_ctx *ctx, int *count, int *code, int *index);
int afd_checked_build(void);

/* Pass timing, for profiling: while on, every float32 filter call that runs
 * on the streaming kernel records a pair of CUDA events on the context's
 * stream around its sequence of passes (after the statistics of
 * afd_filter_rel, before any copy).  afd_pass_timing_read waits for the
 * last recorded event, returns the summed device time of the recorded
 * sequences (ms) and their number of passes, and clears the record. */
afd_status afd_pass_timing(afd_ctx *ctx, int on);
afd_status afd_pass_timing_read(afd_ctx *ctx, double *ms, int64_t *passes);

/* Diagnostic of the bounded-wait machinery: launches one kernel whose
 * mbarrier wait can never complete and gives up after limit_ns nanoseconds
 * (clamped to [1 us, 5 s]), recording the expiry in the context's error
 * word.  The following afd_sync returns AFD_ETIMEOUT and the context stays
 * usable.  The paper has no counterpart; it exists to test error reporting
 * without hanging a GPU. */
afd_status afd_selftest_wait(afd_ctx *ctx, int64_t limit_ns);

/* ---- resident batches (hundreds of uneven cutouts filtered together) ----
 *
 * A batch keeps `count` cubes resident in library-owned device memory (an
 * input, a result and a scratch copy of each, rows padded to 16 bytes so the
 * streaming kernel's TMA loads work for any nx).  afd_batch_filter filters all
 * of them with one CUDA-graph launch: FP64 noise statistics of every cube,
 * per-cube K and conductance coefficients computed on the device, then the
 * n_iter passes, each one persistent launch over the tiles of all cubes.
 * Each cube's result is bit-identical to afd_filter_out (float32) or
 * afd_filter_ex with t_block 1 (2-byte storage) on that cube alone with the
 * same K.  The paper motivates batches by the hundreds of galaxies a survey
 * cube holds (Sec. 1). */
typedef struct afd_batch afd_batch;

/* dims: HOST array of 3*count int64 (nx, ny, nz of each cube).  storage and
 * scale as for afd_filter_ex.  Allocates 3 x the padded cubes' bytes (plus
 * small tables) and zeroes them.  AFD_EINVAL for bad sizes or scale,
 * AFD_ENOMEM when the arena does not fit. */
afd_status afd_batch_create(afd_ctx *ctx, afd_batch **out, int count, const int64_t *dims,
                            afd_storage storage, float scale);

/* Copy cube i (a DEVICE or HOST pointer to a dense nx*ny*nz array in the
 * batch's storage format) into the batch's resident input.  Asynchronous on
 * the context's stream. */
afd_status afd_batch_set(afd_batch *b, int i, const void *cube);

/* Copy the result of cube i out to a dense DEVICE or HOST array.
 * Asynchronous on the context's stream (synchronise before reading host
 * memory). */
afd_status afd_batch_get(afd_batch *b, int i, void *cube);

/* Filter every cube: n_iter >= 1 iterations from its resident input into its
 * result.
 *   K        HOST array of count floats: K[i] > 0 is cube i's K in value
 *            units; K[i] < 0 asks for K = -K[i] * (noise rms of cube i),
 *            the rms of its negative voxels in FP64 on the GPU (so -1.5 is
 *            K = 1.5 sigma).  +inf (all cubes) gives the heat equation; 0,
 *            NaN and a mix of finite and infinite values are AFD_EINVAL.
 *   spacing, dt, cond  as for afd_filter (shared by the batch).
 * The first call (and any call whose n_iter, dt, spacing, conductance or
 * z-chunk differ from the previous one) captures a CUDA graph; later calls
 * only copy K and launch it.  Asynchronous; waits for earlier work on the
 * context's stream before reusing its K staging buffer. */
afd_status afd_batch_filter(afd_batch *b, const float *K, const float *spacing, float dt,
                            int n_iter, afd_conductance cond);

/* The K each cube was filtered with in the last afd_batch_filter (value
 * units), into a HOST array of count floats.  Synchronises the stream. */
afd_status afd_batch_k(afd_batch *b, float *K_out);

/* Tuning: z planes per tile of the batched streaming kernel (0 = 64).
 * Results do not depend on it. */
afd_status afd_batch_set_zchunk(afd_batch *b, int zc);

/* Tile kinds of the batched pass (afd_batch_set_tiles). */
#define AFD_TILES_64X32 0 /* 64 x 32 tiles, 4 x 2 voxels per thread            */
#define AFD_TILES_WIDE 1  /* per-cube tiles of 8 x 2 voxels per thread: tile
                             columns of at most 128 voxels and equal width,
                             as tall as the CTA's threads cover (narrow cubes
                             get one tall tile column, no halo columns
                             between tiles); the default                   */

/* Tuning: the tile kind of the batch's passes (and of a service over it).
 * Results do not depend on it (every kind computes the same per-face
 * arithmetic, bit for bit).  AFD_EINVAL for another value. */
afd_status afd_batch_set_tiles(afd_batch *b, int kind);

/* Free the batch's device memory after the context's stream is idle.  NULL
 * is accepted. */
afd_status afd_batch_destroy(afd_batch *b);

/* ---- interactive re-filter service (continuous batching) ----
 *
 * A service runs re-filter requests (cube of a resident batch, K, dt,
 * n_iter, conductance) against the batch's resident inputs.  Requests are
 * admitted while a descriptor slot and slot memory for their result and
 * scratch cubes fit the service's HBM budget; each round is one launch of
 * the batched streaming kernel per conductance kind over the tiles of every
 * admitted request, each advancing one iteration.  Requests submitted while
 * others run join at the next round.  A request's result is bit-identical
 * to afd_filter_ex (t_block 1) on that cube alone.  The paper's aim is
 * interactive filtering of faint structure (Sec. 1, Sec. 6). */
typedef struct afd_serve afd_serve;

/* mem_bytes: HBM budget for request results and scratch (allocated once).
 * max_active: most requests admitted at once.  The batch must belong to
 * ctx and outlive the service. */
afd_status afd_serve_create(afd_ctx *ctx, afd_batch *cubes, size_t mem_bytes, int max_active,
                            afd_serve **out);

/* Queue a request; *ticket identifies it.  K in value units (> 0; +inf is
 * the heat equation), dt and cond as for afd_filter, unit spacing.
 * AFD_ENOMEM if the request could never fit the budget.  Host-side only. */
afd_status afd_serve_submit(afd_serve *s, int cube, float K, float dt, int n_iter,
                            afd_conductance cond, uint64_t *ticket);

/* Advance the service: retire finished rounds, admit queued requests that
 * fit, launch the next round if fewer than two are in flight.  wait != 0
 * blocks for the oldest round when nothing new could be launched.  *active
 * and *queued (may be NULL) receive the counts afterwards. */
afd_status afd_serve_step(afd_serve *s, int wait, int *active, int *queued);

/* *state: 0 queued, 1 running, 2 done; *latency_s (may be NULL): seconds
 * from submit to the completion of its last round as seen by a step (-1 if
 * not done).  AFD_EINVAL for an unknown ticket. */
afd_status afd_serve_poll(afd_serve *s, uint64_t ticket, int *state, double *latency_s);

/* Copy a done request's result (dense, the batch's storage format) to a
 * DEVICE or HOST pointer; asynchronous on the context's stream.  AFD_EBUSY
 * if not done. */
afd_status afd_serve_result(afd_serve *s, uint64_t ticket, void *dst);

/* Host timestamps of a request (seconds on the library's steady clock):
 * out4[0] submitted, out4[1] admitted (slot memory granted; -1 while
 * queued), out4[2] its first iteration's round launched (-1 before),
 * out4[3] its last round seen complete (-1 before).  They split a latency
 * into waiting for memory, waiting for a round and running.  AFD_EINVAL for
 * an unknown (or released) ticket. */
afd_status afd_serve_times(afd_serve *s, uint64_t ticket, double *out4);

/* Free a done request's slot memory (after its result has been copied).
 * AFD_EBUSY if not done. */
afd_status afd_serve_release(afd_serve *s, uint64_t ticket);

/* Bytes of the budget not held by admitted requests. */
afd_status afd_serve_free_bytes(afd_serve *s, size_t *out);

/* Free the service after the context's stream is idle.  NULL is accepted. */
afd_status afd_serve_destroy(afd_serve *s);

/* Largest cube afd_filter_noalloc accepts: 8,388,608 voxels, i.e. 32 MiB of
 * float32 scratch (for example 256 x 256 x 128). */
#define AFD_NOALLOC_MAX_VOXELS 8388608

/* afd_filter_out for callers that cannot allocate GPU memory.
 *
 * The paper has no counterpart; this entry point exists for callers that may
 * not call cudaMalloc: a host application that has already pooled every
 * device byte for itself, a real-time loop where an allocation (and the
 * device synchronisation it can cause) is not allowed, or a plug-in that is
 * given no allocator.  Such callers cannot create an afd_ctx, which owns
 * device memory, so this call takes no context.  It allocates nothing: three
 * fixed-size arrays inside the library's device image hold its state (the
 * ping-pong scratch of AFD_NOALLOC_MAX_VOXELS floats, 32 MiB; a 256-byte
 * error word; the streaming kernel's 8-byte tile counter), which a GPU holds
 * from the first call on it until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 *   in, out      DEVICE pointers to nx*ny*nz floats, caller-owned (in == out
 *                filters in place; other overlaps are rejected).
 *   spacing, K, dt, n_iter, cond   as for afd_filter.
 *   cuda_stream  cudaStream_t to run on, on the current device (NULL: the
 *                legacy default stream).
 * Results are bit-identical to afd_filter_out's.
 * Sizes: nx*ny*nz > AFD_NOALLOC_MAX_VOXELS returns AFD_EINVAL before any GPU
 * work, as do the argument errors of afd_filter_out.
 * Set-up: the first call on each device (with that device current) looks up
 * the arrays' device addresses; make that first call before any stream
 * capture.
 * Sharing: every call on a device uses the same three arrays, which keep
 * the last call's contents (the call zeroes its error word and tile counter
 * itself).  Calls whose work overlaps on the GPU (from several host threads
 * or streams at once) race on all three (scratch, error word, tile counter)
 * and corrupt each other's results: serialise them.
 * Synchronous: returns after the result is in `out`; AFD_ETIMEOUT if a
 * kernel's bounded wait expired, AFD_ECUDA on a CUDA error. */
afd_status afd_filter_noalloc(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz,
                              const float *spacing, float K, float dt, int n_iter,
                              afd_conductance cond, void *cuda_stream);

/* Number of kernels this context has launched since it was created. */
afd_status afd_launch_count(afd_ctx *ctx, uint64_t *out);

/* Static description of a status code. */
const char *afd_status_str(afd_status s);

/* Text of the last CUDA error seen by this context ("" if none). */
const char *afd_last_error_string(afd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* AFD_H */
