/*
 * Plain CPU oracle of SceneFlowFields' own matching cost (Sec. 3.1,
 * "Matching Cost", Eq. 1): per pixel the first three principal components
 * phi of a dense SIFT descriptor, the principal axes computed over the
 * descriptors of all four images, and the cost of a scene flow vector as the
 * sum over a 7 x 7 window of the Euclidean distances between phi of the
 * reference view and phi of the three other views.
 *
 * TEST INFRASTRUCTURE ONLY: the slow statement of what the CUDA path
 * computes, loaded by the tests and the benchmark's CPU leg.  It shares no
 * source with the CUDA path.
 *
 * The paper gives the cost, the window and "first three principal
 * components of a SIFT feature vector"; the descriptor itself is SIFTFlow's
 * dense SIFT, whose details it does not restate.  Readings (implemented
 * identically by the CUDA path, in the same floating-point order, without
 * fused multiply-adds):
 *   - at scale s (pixel stride n = 2^s) the descriptor is taken on the grey
 *     value (R + 2G + B + 2) >> 2 of the scale's box-smoothed image;
 *   - gradient at q: dx = g(q + (n, 0)) - g(q - (n, 0)), dy = g(q + (0, n)) -
 *     g(q - (0, n)), positions clamped; magnitude sqrtf(dx^2 + dy^2) in
 *     single precision; orientation bin k in 0..7 when the direction lies in
 *     [k 45, (k + 1) 45) degrees, found exactly by integer cross products;
 *   - 4 x 4 cells of 3 x 3 samples at stride n: sample (i, j), i, j in
 *     0..11, at offset ((i - 6) n, (j - 6) n) from the pixel, clamped; cell
 *     (i / 3, j / 3); each cell sums its samples' magnitudes per bin in
 *     row-major sample order;
 *   - descriptor: the 128 sums (cell-major, bin-minor), divided by their L2
 *     norm, clipped at 0.2, divided by the new norm (norms as sequential sums
 *     of squares, sqrtf), quantised to min(255, (int)(v 512 + 0.5));
 *   - principal axes: the covariance of the full-resolution descriptors of
 *     the four images from exact integer sums, in double precision; its top
 *     three eigenvectors by 200 power iterations from the all-ones vector,
 *     each deflated by the previous ones, normalised, sign such that the
 *     largest component is positive; every dot product of the iteration
 *     (matrix rows, deflation, norm) as four partial sums over the indices
 *     mod 4, each in index order by fused multiply-adds, combined as
 *     (s0 + s1) + (s2 + s3); the same axes at every scale;
 *   - phi_c = sum_k fl(a_ck) fl(q_k) (sequential, single precision) minus
 *     fl(sum_k a_ck mu_k) (double precision); stored as 4 floats per pixel;
 *   - cost: the window's 49 pixels p + n (i, j), i, j in -3..3, row-major,
 *     each adding |phi_ref - phi_tmp|, |phi_ref - phi_ste|, |phi_ref -
 *     phi_crs| in that order (single precision, positions clamped), with
 *     |a - b| = sqrtf((dx dx + dy dy) + dz dz); the non-negative float is
 *     kept as its bit pattern in an int32, which orders like the float.
 * Pins: tests/test_oracle_sift.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

void sffo_smooth(const uint8_t* img, int w, int h, int s, uint8_t* out);

static int g_fthreads = 1;
void sfft_set_threads(int n) { g_fthreads = n < 1 ? 1 : n; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* the 8 sector boundaries, 45 degrees apart, as integer directions */
static const int kRay[9][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}, {-1, 0}, {-1, -1}, {0, -1}, {1, -1}, {1, 0}};

int sfft_orientation_bin(int dx, int dy) {
    for (int k = 0; k < 8; k++) {
        const long a = (long)kRay[k][0] * dy - (long)kRay[k][1] * dx;          /* >= 0: not before ray k */
        const long b = (long)kRay[k + 1][0] * dy - (long)kRay[k + 1][1] * dx;  /* < 0: before ray k + 1 */
        if (a >= 0 && b < 0) return k;
    }
    return 0; /* zero gradient */
}

/* Descriptors of one image at scale s: rgb_s is the scale's smoothed image
 * (H x W x 3), desc out [H][W][128]. */
void sfft_descriptors(const uint8_t* rgb_s, int w, int h, int s, uint8_t* desc) {
    const int n = 1 << s;
    const size_t np = (size_t)w * h;
    uint8_t* g = (uint8_t*)malloc(np);
    float* mag = (float*)malloc(np * sizeof(float));
    uint8_t* bin = (uint8_t*)malloc(np);
    for (size_t i = 0; i < np; i++) {
        const uint8_t* p = rgb_s + 3 * i;
        g[i] = (uint8_t)((p[0] + 2 * p[1] + p[2] + 2) >> 2);
    }
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            const int dx = g[(size_t)y * w + clampi(x + n, 0, w - 1)] - g[(size_t)y * w + clampi(x - n, 0, w - 1)];
            const int dy = g[(size_t)clampi(y + n, 0, h - 1) * w + x] - g[(size_t)clampi(y - n, 0, h - 1) * w + x];
            mag[(size_t)y * w + x] = sqrtf((float)(dx * dx + dy * dy));
            bin[(size_t)y * w + x] = (uint8_t)sfft_orientation_bin(dx, dy);
        }
    #pragma omp parallel for num_threads(g_fthreads) schedule(static)
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            float v[128];
            memset(v, 0, sizeof v);
            for (int j = 0; j < 12; j++)
                for (int i = 0; i < 12; i++) {
                    const int qx = clampi(x + (i - 6) * n, 0, w - 1), qy = clampi(y + (j - 6) * n, 0, h - 1);
                    const size_t q = (size_t)qy * w + qx;
                    const int cell = (j / 3) * 4 + i / 3;
                    v[cell * 8 + bin[q]] = v[cell * 8 + bin[q]] + mag[q];
                }
            float ss = 0.0f;
            for (int k = 0; k < 128; k++) ss = ss + v[k] * v[k];
            float nr = sqrtf(ss);
            if (nr > 0.0f)
                for (int k = 0; k < 128; k++) {
                    v[k] = v[k] / nr;
                    if (v[k] > 0.2f) v[k] = 0.2f;
                }
            ss = 0.0f;
            for (int k = 0; k < 128; k++) ss = ss + v[k] * v[k];
            nr = sqrtf(ss);
            uint8_t* out = desc + ((size_t)y * w + x) * 128;
            for (int k = 0; k < 128; k++) {
                const float u = nr > 0.0f ? v[k] / nr : 0.0f;
                const int qv = (int)(u * 512.0f + 0.5f);
                out[k] = (uint8_t)(qv > 255 ? 255 : qv);
            }
        }
    free(g);
    free(mag);
    free(bin);
}

/* Dot product of two 128-vectors as in the power iteration: four partial
 * sums over the indices k = 0, 1, 2, 3 mod 4, each accumulated in index
 * order by fused multiply-adds (one rounding each), combined as
 * (s0 + s1) + (s2 + s3). */
static double dot128(const double* a, const double* b) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < 128; k++) s[k & 3] = fma(a[k], b[k], s[k & 3]);
    return (s[0] + s[1]) + (s[2] + s[3]);
}

/* Principal axes of n_desc descriptors [n_desc][128]: mean[128] and
 * axes[3][128] (double precision). */
void sfft_pca(const uint8_t* desc, int64_t n_desc, double* mean, double* axes) {
    /* exact integer sums (any order), the upper triangle, per thread then combined */
    int64_t* s1 = (int64_t*)calloc(128, sizeof(int64_t));
    int64_t* s2 = (int64_t*)calloc(128 * 128, sizeof(int64_t));
    #pragma omp parallel num_threads(g_fthreads)
    {
        int64_t* t1 = (int64_t*)calloc(128, sizeof(int64_t));
        int64_t* t2 = (int64_t*)calloc(128 * 128, sizeof(int64_t));
        #pragma omp for schedule(static)
        for (int64_t p = 0; p < n_desc; p++) {
            const uint8_t* q = desc + p * 128;
            for (int i = 0; i < 128; i++) {
                const int64_t qi = q[i];
                t1[i] += qi;
                for (int j = i; j < 128; j++) t2[i * 128 + j] += qi * q[j];
            }
        }
        #pragma omp critical
        {
            for (int i = 0; i < 128; i++) s1[i] += t1[i];
            for (int k = 0; k < 128 * 128; k++) s2[k] += t2[k];
        }
        free(t1);
        free(t2);
    }
    for (int i = 0; i < 128; i++)
        for (int j = 0; j < i; j++) s2[i * 128 + j] = s2[j * 128 + i];
    double C[128 * 128];
    for (int i = 0; i < 128; i++) mean[i] = (double)s1[i] / (double)n_desc;
    for (int i = 0; i < 128; i++)
        for (int j = 0; j < 128; j++) C[i * 128 + j] = (double)s2[i * 128 + j] / (double)n_desc - mean[i] * mean[j];
    for (int c = 0; c < 3; c++) {
        double v[128], wv[128];
        for (int i = 0; i < 128; i++) v[i] = 1.0;
        for (int it = 0; it < 200; it++) {
            for (int i = 0; i < 128; i++) wv[i] = dot128(C + i * 128, v);
            for (int e = 0; e < c; e++) {
                const double d = dot128(axes + e * 128, wv);
                for (int i = 0; i < 128; i++) wv[i] = wv[i] - d * axes[e * 128 + i];
            }
            const double nr = sqrt(dot128(wv, wv));
            for (int i = 0; i < 128; i++) v[i] = nr > 0.0 ? wv[i] / nr : 0.0;
        }
        int big = 0;
        for (int i = 1; i < 128; i++)
            if (fabs(v[i]) > fabs(v[big])) big = i;
        const double sg = v[big] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < 128; i++) axes[c * 128 + i] = sg * v[i];
    }
    free(s1);
    free(s2);
}

/* phi [n_desc][4] of descriptors [n_desc][128] on the axes. */
void sfft_project(const uint8_t* desc, int64_t n_desc, const double* mean, const double* axes, float* phi) {
    float a32[3][128], bias[3];
    for (int c = 0; c < 3; c++) {
        double b = 0.0;
        for (int k = 0; k < 128; k++) {
            a32[c][k] = (float)axes[c * 128 + k];
            b = b + axes[c * 128 + k] * mean[k];
        }
        bias[c] = (float)b;
    }
    #pragma omp parallel for num_threads(g_fthreads) schedule(static)
    for (int64_t p = 0; p < n_desc; p++) {
        const uint8_t* q = desc + p * 128;
        for (int c = 0; c < 3; c++) {
            float t = 0.0f;
            for (int k = 0; k < 128; k++) t = t + a32[c][k] * (float)q[k];
            phi[p * 4 + c] = t - bias[c];
        }
        phi[p * 4 + 3] = 0.0f;
    }
}

/* phi of the four images at every scale: rgb[4] H x W x 3, phi[4] each
 * [S][H][W][4]; mean / axes out (may be NULL). */
void sfft_phi(const uint8_t* const* rgb, int w, int h, int S, float* const* phi, double* mean_out,
              double* axes_out) {
    const size_t np = (size_t)w * h;
    uint8_t* sm = (uint8_t*)malloc(np * 3);
    uint8_t* desc = (uint8_t*)malloc(np * 128 * 4);
    double mean[128], axes[3 * 128];
    for (int s = 0; s < S; s++) {
        for (int v = 0; v < 4; v++) {
            sffo_smooth(rgb[v], w, h, s, sm);
            sfft_descriptors(sm, w, h, s, desc + (size_t)v * np * 128);
        }
        if (s == 0) sfft_pca(desc, (int64_t)np * 4, mean, axes);
        for (int v = 0; v < 4; v++)
            sfft_project(desc + (size_t)v * np * 128, (int64_t)np, mean, axes, phi[v] + (size_t)s * np * 4);
    }
    if (mean_out) memcpy(mean_out, mean, sizeof mean);
    if (axes_out) memcpy(axes_out, axes, sizeof axes);
    free(sm);
    free(desc);
}

static float dist3(const float* a, const float* b) {
    const float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrtf((dx * dx + dy * dy) + dz * dz);
}

/* Eq. 1 with SIFT-PCA features at one scale: phi_* [H][W][4] of the scale,
 * n its stride, sigma +1 (forward) or -1 (inverse field); the float cost. */
float sfft_cost(const float* ref, const float* tmp, const float* ste, const float* crs, int w, int h, int n,
                int sigma, int px, int py, const int16_t* u) {
    float c = 0.0f;
    for (int j = -3; j <= 3; j++)
        for (int i = -3; i <= 3; i++) {
            const int x = px + i * n, y = py + j * n;
            const float* a = ref + ((size_t)clampi(y, 0, h - 1) * w + clampi(x, 0, w - 1)) * 4;
            const float* t = tmp + ((size_t)clampi(y + u[1], 0, h - 1) * w + clampi(x + u[0], 0, w - 1)) * 4;
            const float* s = ste + ((size_t)clampi(y, 0, h - 1) * w + clampi(x - sigma * u[2], 0, w - 1)) * 4;
            const float* r = crs + ((size_t)clampi(y + u[1], 0, h - 1) * w + clampi(x + u[0] - sigma * u[3], 0, w - 1)) * 4;
            c = c + dist3(a, t);
            c = c + dist3(a, s);
            c = c + dist3(a, r);
        }
    return c;
}
