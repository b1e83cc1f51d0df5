/*
 * Plain FP64 CPU oracle for the gradient anisotropic-diffusion filter of
 * Punzo, van der Hulst & Roerdink, "Finding faint H I structure in and around
 * galaxies: scraping the barrel" (arXiv:1609.03782), Sec. 3.3.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header or constant with the CUDA library; the product path never
 * calls it.
 *
 * Everything is single-threaded plain loops in double precision, compiled
 * with -O2 -ffp-contract=off so that every operation is the one written.
 *
 * Layout of every cube: x fastest, index = x + nx*(y + ny*z), z = velocity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Conductance choices (this file's own numbering). */
#define ORC_EXPONENTIAL 0 /* g = exp(-(d/K)^2), Perona-Malik's first choice   */
#define ORC_RATIONAL 1    /* g = 1/(1+(d/K)^2), Sec. 3.3 eq. after "perona"   */

/*
 * Edge-stopping conductance g(d; K) for a directional face difference d.
 * Sec. 3.3 prints the rational form 1/(1+|grad I|^2/K^2); the exponential form
 * is Perona and Malik's other standard choice, the paper cites their work for
 * the discretisation.  Limits: K = 0 stops every flux (g = 0, the identity
 * filter); K = +inf gives g = 1 (the plain heat equation).
 */
static double orc_conductance(double d, double K, int cond)
{
    if (K == 0.0)
        return 0.0;
    double r = d / K;
    if (cond == ORC_EXPONENTIAL)
        return exp(-(r * r));
    return 1.0 / (1.0 + r * r);
}

/*
 * n_iter explicit iterations of div(g(|grad I|) grad I) (Sec. 3.3, eq.
 * "perona": dI/dt = S lap I + grad S . grad I, which is div(S grad I)),
 * discretised per face as Perona and Malik do: for every voxel p and each of
 * its six face neighbours q,
 *     d   = (I[q] - I[p]) / h_a          (directional face difference)
 *     acc += g(d; K) * d / h_a           (flux through that face)
 * and then I'[p] = I[p] + dt * acc.  A face on the cube's boundary carries no
 * flux (zero-flux boundary).  The update is synchronous (Jacobi): iteration
 * i+1 reads only iteration i, which is what the two-buffer memory model of
 * Sec. 6 (2 eta) implies.  Exactly n_iter updates are made.
 *
 * I is overwritten with the result.  Returns 0, or -1 on bad arguments or if
 * the scratch buffer cannot be allocated.
 */
int orc_pm_filter(double *I, int64_t nx, int64_t ny, int64_t nz,
                  double hx, double hy, double hz,
                  double K, double dt, int n_iter, int cond)
{
    if (!I || nx < 1 || ny < 1 || nz < 1 || n_iter < 0)
        return -1;
    if (cond != ORC_EXPONENTIAL && cond != ORC_RATIONAL)
        return -1;
    int64_t n = nx * ny * nz;
    double *J = (double *)malloc((size_t)n * sizeof(double));
    if (!J)
        return -1;
    const double h[3] = {hx, hy, hz};
    const int64_t dim[3] = {nx, ny, nz};
    const int64_t stride[3] = {1, nx, nx * ny};
    double *cur = I, *nxt = J;

    for (int it = 0; it < n_iter; ++it) {
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c[3] = {x, y, z};
                    const int64_t p = x + nx * (y + ny * z);
                    double acc = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        for (int s = -1; s <= 1; s += 2) {
                            int64_t cq = c[a] + s;
                            if (cq < 0 || cq >= dim[a])
                                continue; /* zero flux through the boundary */
                            int64_t q = p + s * stride[a];
                            double d = (cur[q] - cur[p]) / h[a];
                            acc += orc_conductance(d, K, cond) * d / h[a];
                        }
                    }
                    nxt[p] = cur[p] + dt * acc;
                }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != I)
        memcpy(I, cur, (size_t)n * sizeof(double));
    free(J);
    return 0;
}

/*
 * The paper's own intensity-driven form (Sec. 3.3, the discretised equation
 * after "conductivepara"):
 *     I' = I + tau * (Cx Dx + Cy Dy + Cz Dz) / (1 + I^2 / (K^2 rms^2))
 * with Dx = [I(x+1) - I] + [I(x-1) - I], the nearest-neighbour second
 * difference, and the conductance taken once per voxel from the voxel's own
 * intensity.  A neighbour outside the cube contributes no difference (the
 * same zero-flux boundary as above).  n_iter synchronous updates.
 */
int orc_intensity_filter(double *I, int64_t nx, int64_t ny, int64_t nz,
                         double cx, double cy, double cz,
                         double K, double rms, double tau, int n_iter)
{
    if (!I || nx < 1 || ny < 1 || nz < 1 || n_iter < 0)
        return -1;
    int64_t n = nx * ny * nz;
    double *J = (double *)malloc((size_t)n * sizeof(double));
    if (!J)
        return -1;
    const double C[3] = {cx, cy, cz};
    const int64_t dim[3] = {nx, ny, nz};
    const int64_t stride[3] = {1, nx, nx * ny};
    const double krms2 = K * K * rms * rms;
    double *cur = I, *nxt = J;

    for (int it = 0; it < n_iter; ++it) {
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t c[3] = {x, y, z};
                    const int64_t p = x + nx * (y + ny * z);
                    double lap = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double D = 0.0;
                        for (int s = -1; s <= 1; s += 2) {
                            int64_t cq = c[a] + s;
                            if (cq < 0 || cq >= dim[a])
                                continue;
                            D += cur[p + s * stride[a]] - cur[p];
                        }
                        lap += C[a] * D;
                    }
                    double S = (krms2 == 0.0)
                                   ? 0.0
                                   : 1.0 / (1.0 + cur[p] * cur[p] / krms2);
                    nxt[p] = cur[p] + tau * lap * S;
                }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != I)
        memcpy(I, cur, (size_t)n * sizeof(double));
    free(J);
    return 0;
}

/*
 * Whole-cube statistics of an FP32 cube, accumulated in double in index
 * order:
 *   out[0] = sum I                      (conservation check)
 *   out[1] = sum I^2                    (plain rms = sqrt(out[1]/n))
 *   out[2] = sum over I<0 of I^2        (negative-half noise estimate)
 *   out[3] = number of voxels with I<0
 * The paper sets K in units of the noise level "rms" (Sec. 3.3) and assumes
 * it constant over the cube (Sec. 4) without saying how it is measured; the
 * noise estimate used here is sqrt(out[2]/out[3]), the rms of the negative
 * voxels, because H I emission is positive and the noise is symmetric.
 */
void orc_stats(const float *I, int64_t n, double out[4])
{
    double s = 0.0, s2 = 0.0, ns2 = 0.0, nneg = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v = (double)I[i];
        s += v;
        s2 += v * v;
        if (v < 0.0) {
            ns2 += v * v;
            nneg += 1.0;
        }
    }
    out[0] = s;
    out[1] = s2;
    out[2] = ns2;
    out[3] = nneg;
}

/*
 * Smoothing-quality sums of Sec. 4 (eqs. "F_equa", "Sequa", "Mfequa") and of
 * the recovered-signal fraction of Sec. 5 (eq. "sums_equa"), over the ROI
 * box [roi[0], roi[1]) x [roi[2], roi[3]) x [roi[4], roi[5]) (x, y, z).
 *
 * The masks are M_o = [I_o >= t_o] and M_f = [I_f >= t_f], where t_i is a
 * multiple (3 in the paper) of cube i's rms.  The sums always take the
 * ORIGINAL cube's intensities, as Sec. 4 stresses.  Im, the noiseless model,
 * may be NULL.
 *   out[0] = S_of = sum I_o M_f       out[1] = S_oo = sum I_o M_o
 *   out[2] = S_mf = sum I_m M_f       out[3] = S_m  = sum I_m
 *   out[4] = N_o  = sum M_o           out[5] = N_f  = sum M_f
 * Returns -1 for an empty or out-of-range box.
 */
int orc_fdiag(const float *Io, const float *If, const float *Im, int64_t nx, int64_t ny,
              int64_t nz, const int64_t roi[6], double t_o, double t_f, double out[6])
{
    if (roi[0] < 0 || roi[1] > nx || roi[0] >= roi[1] || roi[2] < 0 || roi[3] > ny ||
        roi[2] >= roi[3] || roi[4] < 0 || roi[5] > nz || roi[4] >= roi[5])
        return -1;
    double s_of = 0.0, s_oo = 0.0, s_mf = 0.0, s_m = 0.0, n_o = 0.0, n_f = 0.0;
    for (int64_t z = roi[4]; z < roi[5]; ++z)
        for (int64_t y = roi[2]; y < roi[3]; ++y)
            for (int64_t x = roi[0]; x < roi[1]; ++x) {
                const int64_t p = x + nx * (y + ny * z);
                const double io = (double)Io[p];
                const double iff = (double)If[p];
                const int mo = io >= t_o;
                const int mf = iff >= t_f;
                if (mo) {
                    s_oo += io;
                    n_o += 1.0;
                }
                if (mf) {
                    s_of += io;
                    n_f += 1.0;
                }
                if (Im) {
                    const double im = (double)Im[p];
                    s_m += im;
                    if (mf)
                        s_mf += im;
                }
            }
    out[0] = s_of;
    out[1] = s_oo;
    out[2] = s_mf;
    out[3] = s_m;
    out[4] = n_o;
    out[5] = n_f;
    return 0;
}

/*
 * Smoothing by a normalised correlation (the box and Gaussian filters of
 * Sec. 3.1 and 3.2):
 *   out(p) = sum_q W(q - p) I(q) / sum_q W(q - p),
 * q over the (2rx+1) x (2ry+1) x (2rz+1) window around p that lies inside
 * the cube.  W is given explicitly (x fastest, index dx+rx + (2rx+1) *
 * (dy+ry + (2ry+1) * (dz+rz))).  The paper states no boundary rule; dividing
 * by the in-cube weight makes the box filter the mean of the existing
 * neighbours ("the mean value of its neighbors, including itself") and keeps
 * a constant cube constant.  Returns -1 for a bad radius, or when the
 * in-cube weight of some voxel is not positive.
 */
int orc_smooth(double *out, const float *I, int64_t nx, int64_t ny, int64_t nz, const double *W,
               int rx, int ry, int rz)
{
    if (rx < 0 || ry < 0 || rz < 0)
        return -1;
    const int64_t wx = 2 * rx + 1, wy = 2 * ry + 1;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double num = 0.0, den = 0.0;
                for (int dz = -rz; dz <= rz; ++dz) {
                    const int64_t qz = z + dz;
                    if (qz < 0 || qz >= nz)
                        continue;
                    for (int dy = -ry; dy <= ry; ++dy) {
                        const int64_t qy = y + dy;
                        if (qy < 0 || qy >= ny)
                            continue;
                        for (int dx = -rx; dx <= rx; ++dx) {
                            const int64_t qx = x + dx;
                            if (qx < 0 || qx >= nx)
                                continue;
                            const double w = W[(dx + rx) + wx * ((dy + ry) + wy * (dz + rz))];
                            num += w * (double)I[qx + nx * (qy + ny * qz)];
                            den += w;
                        }
                    }
                }
                if (!(den > 0.0))
                    return -1;
                out[x + nx * (y + ny * z)] = num / den;
            }
    return 0;
}
