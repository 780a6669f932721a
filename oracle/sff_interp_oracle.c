/*
 * Plain CPU oracle of SceneFlowFields' dense interpolation of the seeds
 * (Schuster et al., WACV 2018, Sec. 3.2 "Interpolation Models" and
 * "Edge-Aware Neighborhood"), with a Euclidean neighbourhood in place of
 * the geodesic one (the trained boundary detector is not available).
 *
 * TEST INFRASTRUCTURE ONLY: the slow statement of what the CUDA path
 * computes, loaded by the tests and the benchmark's CPU leg.  It shares no
 * source with the CUDA path.
 *
 * For every seed s (the sparse matches of Sec. 3.2), two local models:
 *   geometry: the plane d0 = a1 x + a2 y + a3 fitted by weighted least
 *     squares through its k_geo nearest seeds;
 *   motion: the affine map x1 = A x0 + t of 3D points (12 unknowns) fitted
 *     by weighted least squares through its k_motion nearest motion seeds,
 *     x0 triangulated from (x, y, d0), x1 from (x + u, y + v, d1) with a
 *     pinhole camera (focal f px, principal point (cx, cy), baseline B):
 *     Z = f B / d, X = (x - cx) Z / f, Y = (y - cy) Z / f.
 * The weight of a neighbour at Euclidean distance D px is exp(-alpha D /
 * dist_unit) (the Gaussian kernel g(D) = exp(-alpha D) with D in units of
 * dist_unit pixels).  Every pixel takes the models of its closest seed
 * (the approximation of [revaud2015epic] the paper follows) and evaluates
 * them at its own position: d0 from the plane, then reproject, transform and
 * project back to get u, v, d1.
 *
 * Readings (stated once, implemented identically by the CUDA path):
 *   - neighbours: the k nearest seeds by squared pixel distance, ties to
 *     the lower seed index; a seed is its own nearest neighbour; motion
 *     seeds are the seeds with d0 >= 1 and d1 >= 1 (triangulable);
 *   - closest seed of a pixel: over all seeds, same order;
 *   - coordinates are centred: the plane at its seed's position, the affine
 *     map at the weighted centroid c of its neighbours' 3D points
 *     (x1 = A (x0 - c) + t); the linear part gets a ridge of
 *     1e-9 * trace / dimension towards a flat plane and towards A = I, so
 *     that every system is solvable and too few seeds give a constant
 *     disparity and a translation; the systems are solved by a Cholesky
 *     factorisation in double precision;
 *   - a pixel's disparity used for the reprojection is max(d0, 1);
 *     if the transformed point is not in front of the camera (Z1 <= 0) or
 *     the seed has no motion neighbours, u = v = 0 and d1 = d0;
 *   - output: float [H][W][4] (u, v, d0, d1).
 * Pins: tests/test_oracle_interp.py (an exact plane and an exact affine 3D
 * motion reproduced at every pixel, the weighted mean of a symmetric star,
 * lattice neighbourhoods and ties, motion-seed selection, the one-seed
 * defaults, and on random seeds the fits against numpy's weighted least
 * squares and its solve of the same normal equations).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

typedef struct {
    int16_t x, y, u, v, d0, d1;
    int32_t cost;
    uint8_t cerr;
    uint8_t kind;
    uint8_t pad[2];
} sffi_seed;

typedef struct {
    int32_t k_geo, k_motion;
    double alpha, dist_unit;
    double focal, baseline, cx, cy;
} sffi_params;

static int g_ithreads = 1;
void sffi_set_threads(int n) { g_ithreads = n < 1 ? 1 : n; }

typedef struct {
    int64_t d2;
    int32_t idx;
} nb_t;

static int cmp_nb(const void* a, const void* b) {
    const nb_t* p = (const nb_t*)a;
    const nb_t* q = (const nb_t*)b;
    if (p->d2 != q->d2) return p->d2 < q->d2 ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

static int motion_seed(const sffi_seed* s) { return s->d0 >= 1 && s->d1 >= 1; }

/* The k nearest seeds to (x, y) among those passing `want` (NULL: all):
 * all distances, sorted by (d2, index).  Returns the count (<= k). */
static int nearest(const sffi_seed* seeds, int n, int x, int y, int k, int (*want)(const sffi_seed*),
                   nb_t* buf, nb_t* out) {
    int m = 0;
    for (int i = 0; i < n; i++) {
        if (want && !want(seeds + i)) continue;
        const int64_t dx = seeds[i].x - x, dy = seeds[i].y - y;
        buf[m].d2 = dx * dx + dy * dy;
        buf[m].idx = i;
        m++;
    }
    qsort(buf, (size_t)m, sizeof(nb_t), cmp_nb);
    const int c = m < k ? m : k;
    memcpy(out, buf, (size_t)c * sizeof(nb_t));
    return c;
}

void sffi_nearest(const sffi_seed* seeds, int n, int x, int y, int k, int motion_only, int32_t* idx_out,
                  int64_t* d2_out, int32_t* count_out) {
    nb_t* buf = (nb_t*)malloc(sizeof(nb_t) * (size_t)(n > 0 ? n : 1));
    nb_t* out = (nb_t*)malloc(sizeof(nb_t) * (size_t)(k > 0 ? k : 1));
    const int c = nearest(seeds, n, x, y, k, motion_only ? motion_seed : NULL, buf, out);
    for (int i = 0; i < c; i++) {
        idx_out[i] = out[i].idx;
        d2_out[i] = out[i].d2;
    }
    *count_out = c;
    free(buf);
    free(out);
}

/* Solves M x = b for a symmetric positive definite M (dim n, row-major)
 * with `nr` right-hand sides b[r][n]; x overwrites b. */
static void solve_spd(double* M, int n, double* b, int nr) {
    /* Cholesky M = L L^T, L in the lower triangle */
    for (int j = 0; j < n; j++) {
        double s = M[j * n + j];
        for (int k = 0; k < j; k++) s -= M[j * n + k] * M[j * n + k];
        const double ljj = sqrt(s > 0.0 ? s : 1e-300);
        M[j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = M[i * n + j];
            for (int k = 0; k < j; k++) t -= M[i * n + k] * M[j * n + k];
            M[i * n + j] = t / ljj;
        }
    }
    for (int r = 0; r < nr; r++) {
        double* x = b + r * n;
        for (int i = 0; i < n; i++) {  /* L y = b */
            double t = x[i];
            for (int k = 0; k < i; k++) t -= M[i * n + k] * x[k];
            x[i] = t / M[i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {  /* L^T x = y */
            double t = x[i];
            for (int k = i + 1; k < n; k++) t -= M[k * n + i] * x[k];
            x[i] = t / M[i * n + i];
        }
    }
}

static void triangulate(const sffi_params* P, double x, double y, double d, double* X) {
    const double Z = P->focal * P->baseline / d;
    X[0] = (x - P->cx) * Z / P->focal;
    X[1] = (y - P->cy) * Z / P->focal;
    X[2] = Z;
}

/* Ridge of the linear part: lambda = 1e-9 * trace / n added to the first
 * nl diagonal entries (the constant term is never penalised). */
static double ridge_of(const double* M, int n) {
    double tr = 0.0;
    for (int i = 0; i < n; i++) tr += M[i * n + i];
    return 1e-9 * tr / n + 1e-300;
}

/* Models of seed s: plane[3] (a1, a2, a3 of d0 = a1 (x - xs) + a2 (y - ys)
 * + a3), affine[15] (rows of [A | t], then the centre c);
 * has_motion = number of motion neighbours (0: none). */
static void fit_seed(const sffi_seed* seeds, int n, const sffi_params* P, int s, nb_t* buf, nb_t* nb,
                     double* plane, double* affine, int32_t* has_motion) {
    const int sx = seeds[s].x, sy = seeds[s].y;
    /* geometry: plane through the k_geo nearest seeds */
    int c = nearest(seeds, n, sx, sy, P->k_geo, NULL, buf, nb);
    double M[9] = {0}, b[3] = {0};
    for (int i = 0; i < c; i++) {
        const sffi_seed* g = seeds + nb[i].idx;
        const double w = exp(-P->alpha * sqrt((double)nb[i].d2) / P->dist_unit);
        const double r[3] = {(double)(g->x - sx), (double)(g->y - sy), 1.0};
        for (int a = 0; a < 3; a++) {
            for (int e = 0; e < 3; e++) M[a * 3 + e] += w * r[a] * r[e];
            b[a] += w * r[a] * g->d0;
        }
    }
    {
        const double lam = ridge_of(M, 3);
        M[0] += lam;
        M[4] += lam;
    }
    solve_spd(M, 3, b, 1);
    memcpy(plane + 3 * (size_t)s, b, sizeof b);
    /* motion: affine map through the k_motion nearest motion seeds */
    c = nearest(seeds, n, sx, sy, P->k_motion, motion_seed, buf, nb);
    double N[16] = {0}, rhs[12] = {0}, cen[3] = {0, 0, 0}, wsum = 0.0;
    for (int i = 0; i < c; i++) {  /* weighted centroid of the x0 */
        const sffi_seed* g = seeds + nb[i].idx;
        const double w = exp(-P->alpha * sqrt((double)nb[i].d2) / P->dist_unit);
        double X0[3];
        triangulate(P, g->x, g->y, g->d0, X0);
        for (int j = 0; j < 3; j++) cen[j] += w * X0[j];
        wsum += w;
    }
    for (int j = 0; j < 3 && c > 0; j++) cen[j] /= wsum;
    for (int i = 0; i < c; i++) {
        const sffi_seed* g = seeds + nb[i].idx;
        const double w = exp(-P->alpha * sqrt((double)nb[i].d2) / P->dist_unit);
        double X0[3], X1[3];
        triangulate(P, g->x, g->y, g->d0, X0);
        triangulate(P, g->x + g->u, g->y + g->v, g->d1, X1);
        const double r[4] = {X0[0] - cen[0], X0[1] - cen[1], X0[2] - cen[2], 1.0};
        for (int a = 0; a < 4; a++) {
            for (int e = 0; e < 4; e++) N[a * 4 + e] += w * r[a] * r[e];
            for (int j = 0; j < 3; j++) rhs[j * 4 + a] += w * r[a] * X1[j];
        }
    }
    if (c > 0) {
        const double lam = ridge_of(N, 4);
        for (int a = 0; a < 3; a++) {
            N[a * 4 + a] += lam;
            rhs[a * 4 + a] += lam;  /* towards A = I */
        }
        solve_spd(N, 4, rhs, 3);
    }
    memcpy(affine + 15 * (size_t)s, rhs, sizeof rhs);
    memcpy(affine + 15 * (size_t)s + 12, cen, sizeof cen);
    has_motion[s] = c;
}

/* Models of the seeds listed in which[0 .. m) (NULL: of all n seeds); the
 * other entries of plane / affine / has_motion are left untouched. */
void sffi_seed_models_of(const sffi_seed* seeds, int n, const sffi_params* P, const int32_t* which, int m,
                         double* plane, double* affine, int32_t* has_motion) {
    const int cnt = which ? m : n;
    #pragma omp parallel num_threads(g_ithreads)
    {
        nb_t* buf = (nb_t*)malloc(sizeof(nb_t) * (size_t)(n > 0 ? n : 1));
        const int kmax = P->k_geo > P->k_motion ? P->k_geo : P->k_motion;
        nb_t* nb = (nb_t*)malloc(sizeof(nb_t) * (size_t)(kmax > 0 ? kmax : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int k = 0; k < cnt; k++) fit_seed(seeds, n, P, which ? which[k] : k, buf, nb, plane, affine, has_motion);
        free(buf);
        free(nb);
    }
}

void sffi_seed_models(const sffi_seed* seeds, int n, const sffi_params* P, double* plane, double* affine,
                      int32_t* has_motion) {
    sffi_seed_models_of(seeds, n, P, NULL, 0, plane, affine, has_motion);
}

/* The models of seed s evaluated at pixel (x, y): out[4] = (u, v, d0, d1). */
static void evaluate(const sffi_params* P, const sffi_seed* sd, const double* pl, const double* af, int motion,
                     int x, int y, float* out) {
    const double d0 = pl[0] * (x - sd->x) + pl[1] * (y - sd->y) + pl[2];
    out[2] = (float)d0;
    if (!motion) {
        out[0] = out[1] = 0.f;
        out[3] = (float)d0;
        return;
    }
    double X0[3], X1[3];
    triangulate(P, x, y, d0 > 1.0 ? d0 : 1.0, X0);
    const double* c = af + 12;
    for (int j = 0; j < 3; j++)
        X1[j] = af[4 * j] * (X0[0] - c[0]) + af[4 * j + 1] * (X0[1] - c[1]) + af[4 * j + 2] * (X0[2] - c[2]) + af[4 * j + 3];
    if (!(X1[2] > 0.0)) {
        out[0] = out[1] = 0.f;
        out[3] = (float)d0;
        return;
    }
    const double x1 = P->focal * X1[0] / X1[2] + P->cx, y1 = P->focal * X1[1] / X1[2] + P->cy;
    out[0] = (float)(x1 - x);
    out[1] = (float)(y1 - y);
    out[3] = (float)(P->focal * P->baseline / X1[2]);
}

/* Closest seed of every listed pixel (brute force) and its models evaluated
 * there.  pixels: [m][2] (x, y); out: [m][4]; closest_out: [m] (or NULL). */
void sffi_interpolate_pixels(const sffi_seed* seeds, int n, const sffi_params* P, const double* plane,
                             const double* affine, const int32_t* has_motion, const int32_t* pixels, int m,
                             float* out, int32_t* closest_out) {
    #pragma omp parallel for num_threads(g_ithreads) schedule(static)
    for (int k = 0; k < m; k++) {
        const int x = pixels[2 * k], y = pixels[2 * k + 1];
        int best = -1;
        int64_t bd = 0;
        for (int i = 0; i < n; i++) {
            const int64_t dx = seeds[i].x - x, dy = seeds[i].y - y, d2 = dx * dx + dy * dy;
            if (best < 0 || d2 < bd) { best = i; bd = d2; }  /* ascending index: ties keep the lower */
        }
        if (closest_out) closest_out[k] = best;
        if (best < 0) { out[4 * k] = out[4 * k + 1] = out[4 * k + 2] = out[4 * k + 3] = 0.f; continue; }
        evaluate(P, seeds + best, plane + 3 * (size_t)best, affine + 15 * (size_t)best, has_motion[best] > 0, x, y,
                 out + 4 * k);
    }
}
