/* Multithreaded FP32 CPU build of the per-face anisotropic-diffusion filter
 * (arXiv:1609.03782, Sec. 3.3: the explicit update of eq. "perona" with the
 * gradient conductance, evaluated face by face; zero flux across the cube's
 * faces; n Jacobi iterations with two buffers, the memory model of Sec. 6).
 *
 * This is the host-side baseline the GPU library is measured against, in the
 * role of the paper's own OpenMP implementation (Sec. 6 times its filters on
 * 8 CPU cores).  It is portable C with OpenMP: no ISA intrinsics, no
 * target-specific flags; the compiler vectorises the x loops.  It shares no
 * code with the CUDA library or with the FP64 checker.
 *
 * Arithmetic (float32).  Through the face between a lower voxel a and an
 * upper voxel b along axis x, y or z (spacing h), with d = b - a:
 *     rational     G = d / (A d^2 + B),        A = 1/(K^2 dt), B = h^2/dt
 *     exponential  G = (dt/h^2) d exp(-(d/(K h))^2)
 * (the weight dt/h^2 folded into the flux), the lower voxel gains G and the
 * upper voxel loses it.  Each face is evaluated once per iteration and used
 * by both of its voxels.  Per voxel, I' = I + ((s_x + s_y) + s_z), with
 * s = G(upper face) - G(lower face).  K = 0 is the identity (no flux);
 * K = +inf gives g = 1 (the heat equation).
 *
 * Parallel layout: each thread owns a contiguous range of z planes for the
 * whole call (one parallel region, a barrier between iterations).  It walks
 * its planes upwards keeping the fluxes through the current plane's lower z
 * faces (one plane) and the current row's lower y faces (one row); the z
 * faces at the edge of a thread's range are evaluated by both neighbouring
 * threads from the same inputs with the same operations, so the result does
 * not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

enum { OMP_COND_EXPONENTIAL = 0, OMP_COND_RATIONAL = 1 };

typedef struct {
    int kind;         /* 0 exponential, 1 rational, 2 linear (K = inf) */
    float a[3], b[3]; /* per axis: rational A, B; exponential -1/(K h)^2, dt/h^2;
                         linear dt/h^2 */
} coefs;

static inline float flux(float d, float a, float b, int kind)
{
    if (kind == OMP_COND_RATIONAL) {
        const float t = d * d;
        const float u = a * t + b;
        return d / u;
    }
    if (kind == OMP_COND_EXPONENTIAL) {
        const float t = d * d;
        return b * d * expf(a * t);
    }
    return b * d;
}

/* Fluxes through the faces between rows lo and hi (n voxels, hi = lo's
 * neighbour along one axis): out[i] = G(hi[i] - lo[i]). */
static void face_row(float *restrict out, const float *restrict lo, const float *restrict hi,
                     int64_t n, float a, float b, int kind)
{
    if (kind == OMP_COND_RATIONAL) {
        for (int64_t i = 0; i < n; ++i) {
            const float d = hi[i] - lo[i];
            out[i] = d / (a * (d * d) + b);
        }
    } else if (kind == OMP_COND_EXPONENTIAL) {
        for (int64_t i = 0; i < n; ++i) {
            const float d = hi[i] - lo[i];
            out[i] = b * d * expf(a * (d * d));
        }
    } else {
        for (int64_t i = 0; i < n; ++i)
            out[i] = b * (hi[i] - lo[i]);
    }
}

/* One iteration over the planes [z0, z1) of the thread: in -> out. */
static void iterate(const float *restrict in, float *restrict out, int64_t nx, int64_t ny,
                    int64_t nz, int64_t z0, int64_t z1, const coefs *c, float *restrict gz,
                    float *restrict gzu, float *restrict gy, float *restrict gyu,
                    float *restrict gx)
{
    const int64_t nxy = nx * ny;
    const int kind = c->kind;
    /* fluxes through the lower z faces of plane z0 */
    if (z0 == 0)
        memset(gz, 0, (size_t)nxy * sizeof(float));
    else
        face_row(gz, in + (z0 - 1) * nxy, in + z0 * nxy, nxy, c->a[2], c->b[2], kind);
    for (int64_t z = z0; z < z1; ++z) {
        const float *p = in + z * nxy;
        /* fluxes through the upper z faces of plane z */
        if (z + 1 < nz)
            face_row(gzu, p, p + nxy, nxy, c->a[2], c->b[2], kind);
        else
            memset(gzu, 0, (size_t)nxy * sizeof(float));
        memset(gy, 0, (size_t)nx * sizeof(float));
        for (int64_t y = 0; y < ny; ++y) {
            const float *r = p + y * nx;
            float *o = out + z * nxy + y * nx;
            const float *gzl = gz + y * nx, *gzh = gzu + y * nx;
            if (y + 1 < ny)
                face_row(gyu, r, r + nx, nx, c->a[1], c->b[1], kind);
            else
                memset(gyu, 0, (size_t)nx * sizeof(float));
            /* x faces: gx[i] between voxels i-1 and i; gx[0] = gx[nx] = 0 */
            gx[0] = 0.0f;
            face_row(gx + 1, r, r + 1, nx - 1, c->a[0], c->b[0], kind);
            gx[nx] = 0.0f;
            for (int64_t i = 0; i < nx; ++i) {
                const float sx = gx[i + 1] - gx[i];
                const float sy = gyu[i] - gy[i];
                const float sz = gzh[i] - gzl[i];
                o[i] = r[i] + ((sx + sy) + sz);
            }
            float *t = gy;
            gy = gyu;
            gyu = t;
        }
        float *t = gz;
        gz = gzu;
        gzu = t;
    }
}

/* n_iter iterations of the filter on the float32 cube (x fastest, index
 * x + nx (y + ny z)), in place.  spacing: hx, hy, hz (NULL: unit).  cond:
 * 0 exponential, 1 rational.  threads <= 0: OpenMP's default.  Returns 0, or
 * -1 on an argument error, -2 if memory could not be allocated. */
int afd_omp_filter(float *cube, int64_t nx, int64_t ny, int64_t nz, const float *spacing,
                   float K, float dt, int n_iter, int cond, int threads)
{
    if (!cube || nx < 1 || ny < 1 || nz < 1 || n_iter < 0 || !(dt > 0.0f) || isnan(K) ||
        K < 0.0f || (cond != OMP_COND_EXPONENTIAL && cond != OMP_COND_RATIONAL))
        return -1;
    if (n_iter == 0 || K == 0.0f)
        return 0;
    coefs c;
    c.kind = isinf(K) ? 2 : cond;
    for (int a = 0; a < 3; ++a) {
        const double h = spacing ? spacing[a] : 1.0;
        if (!(h > 0.0))
            return -1;
        const double w = (double)dt / (h * h), kd = (double)K;
        if (c.kind == OMP_COND_RATIONAL) {
            c.a[a] = (float)(1.0 / (kd * kd * (double)dt));
            c.b[a] = (float)(h * h / (double)dt);
        } else if (c.kind == OMP_COND_EXPONENTIAL) {
            c.a[a] = (float)(-1.0 / (kd * h * kd * h));
            c.b[a] = (float)w;
        } else {
            c.a[a] = 0.0f;
            c.b[a] = (float)w;
        }
    }
    const int64_t nxy = nx * ny, n = nxy * nz;
    float *other = (float *)malloc((size_t)n * sizeof(float));
    if (!other)
        return -2;
    int nt = threads > 0 ? threads : omp_get_max_threads();
    if (nt > nz)
        nt = (int)nz;
    int fail = 0;
#pragma omp parallel num_threads(nt) shared(fail)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int64_t z0 = nz * t / T, z1 = nz * (t + 1) / T;
        float *buf = (float *)malloc((size_t)(2 * nxy + 3 * nx + 1) * sizeof(float));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp barrier
        if (!fail) {
            float *gz = buf, *gzu = buf + nxy, *gy = buf + 2 * nxy, *gyu = gy + nx,
                  *gx = gyu + nx;
            const float *src = cube;
            float *dst = other;
            for (int it = 0; it < n_iter; ++it) {
                iterate(src, dst, nx, ny, nz, z0, z1, &c, gz, gzu, gy, gyu, gx);
#pragma omp barrier
                const float *s2 = dst;
                dst = (float *)src;
                src = s2;
            }
            /* the result is in src: an odd count ends in `other` */
            if (src != cube && z1 > z0)
                memcpy(cube + z0 * nxy, src + z0 * nxy, (size_t)((z1 - z0) * nxy) * sizeof(float));
        }
        free(buf);
    }
    free(other);
    return fail ? -2 : 0;
}

/* Threads OpenMP would use by default. */
int afd_omp_max_threads(void) { return omp_get_max_threads(); }

/* Host memory bandwidth, STREAM-copy style: `reps` copies of `bytes` bytes
 * between two buffers, every thread copying its own contiguous part (first
 * touched by that thread).  Returns the best (read + write) GB/s, or -1. */
double afd_omp_stream_copy(int64_t bytes, int reps, int threads)
{
    const int64_t n = bytes / (int64_t)sizeof(float);
    float *a = (float *)malloc((size_t)n * sizeof(float));
    float *b = (float *)malloc((size_t)n * sizeof(float));
    if (!a || !b) {
        free(a);
        free(b);
        return -1.0;
    }
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int64_t i0 = n * t / T, i1 = n * (t + 1) / T;
        for (int64_t i = i0; i < i1; ++i) {
            a[i] = (float)(i & 1023);
            b[i] = 0.0f;
        }
    }
    double best = 0.0;
    for (int r = 0; r < reps; ++r) {
        const double t0 = omp_get_wtime();
#pragma omp parallel num_threads(nt)
        {
            const int t = omp_get_thread_num(), T = omp_get_num_threads();
            const int64_t i0 = n * t / T, i1 = n * (t + 1) / T;
            memcpy(b + i0, a + i0, (size_t)(i1 - i0) * sizeof(float));
        }
        const double el = omp_get_wtime() - t0;
        const double gbs = 2.0 * (double)n * sizeof(float) / el / 1e9;
        if (gbs > best)
            best = gbs;
    }
    volatile float sink = b[n / 2];
    (void)sink;
    free(a);
    free(b);
    return best;
}
