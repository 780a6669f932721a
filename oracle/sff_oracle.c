/*
 * Plain CPU oracle of SceneFlowFields' sparse four-view matching stage
 * (Schuster et al., "SceneFlowFields: Dense Interpolation of Sparse Scene
 * Flow Correspondences", WACV 2018, Sec. 3.1 "Sparse Correspondences" and
 * Sec. 3.2 "Sparsification").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the CUDA path computes.  Only the tests, the package's
 * smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * source, header, table or helper with the CUDA path.
 *
 * Every step is plain loops over pixels in the paper's order:
 *   box smoothing of the scale space            (Sec. 3.1 "Multi-Scale Propagation")
 *   Walsh-Hadamard patch features, H P H^T      (Sec. 3.1 "Initialization", [hel2005real])
 *   matching cost summed over three views       (Eq. 1, with the feature reading below)
 *   exact nearest-neighbour initialisation      (Sec. 3.1 "Initialization")
 *   per-scale propagation + random search       (Sec. 3.1 "Multi-Scale Propagation")
 *   inverse field, consistency + region filter  (Sec. 3.1 "Consistency Check")
 *   3x3-block sparsification into seeds         (Sec. 3.2 "Sparsification")
 *
 * Readings of points the paper leaves open (all shared with the CUDA path by
 * specification, never by code):
 *   - features: 16 AC Walsh-Hadamard coefficients per colour channel of an
 *     8x8 patch (offsets -3..+4 times the scale stride), ordered by total
 *     sequency then vertical sequency, quantised by an arithmetic right shift
 *     and saturated to int8; the cost is the integer sum of squared
 *     differences (SSD) over the three views, no extra window;
 *   - scale space: integer n x n box smoothing at full resolution
 *     (window -n/2 .. n/2-1, round half up) instead of area downsampling plus
 *     Lanczos upsampling;
 *   - initialisation: exact K nearest neighbours over the coarsest grid
 *     (K_T temporal over the whole image, K_E epipolar on a row), all K_T*K_E*K_E
 *     combinations scored with the full cost;
 *   - propagation: synchronous two-colour (checkerboard) half-steps; each
 *     grid pixel considers its own vector and the vectors of its two
 *     predecessors along the sweep direction; replace on strictly lower cost,
 *     ties to the lower candidate index;
 *   - random search: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *     counter (pixel index, iteration, scale + 4 * field, 0); offsets are the
 *     rounded value of a uniform draw on ]-n, n[ full-resolution pixels;
 *   - d0, d1 >= 0; correspondence positions are clamped to the image;
 *   - inverse field: reference R1, temporal R0, stereo L1, cross L0, with the
 *     stereo offset acting towards +x (sigma = -1);
 *   - consistency: round trip of all three correspondences, reject when any
 *     of the four differences exceeds tau_c; cerr = sum of |differences|;
 *   - region filter: 4-connected regions with max-norm vector difference
 *     <= tau_r; a region that a rejected neighbour could join and that is
 *     smaller than s_c is removed;
 *   - seeds: per 3x3 block the kept pixel with the lowest (cerr, cost,
 *     raster index), emitted in block raster order.
 *
 * Parity pins live in tests/test_oracle_*.py: Walsh-Hadamard identities on
 * hand-built patches, Philox known-answer vectors and the numpy Philox4x64
 * structure, brute-force nearest neighbours and exhaustive search on tiny
 * images, exact recovery of integer shifts, and consistency/region/seed
 * invariants.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 48            /* features per pixel: 3 channels x 16 coefficients */
#define NCOEF 16         /* AC coefficients kept per channel */
#define EMPTY_COST INT32_MAX

typedef struct {
    int32_t num_scales;    /* k + 1 = 4 (Sec. 5: k = 3 subscales + full res) */
    int32_t iterations;    /* 12 per scale (Sec. 5) */
    int32_t tau_c;         /* consistency threshold, 1 px (Sec. 5) */
    int32_t region_min;    /* s_c = 150 px (Sec. 5) */
    int32_t tau_r;         /* "approximately the same" vector: max-norm <= tau_r */
    int32_t quant_shift;   /* feature quantisation shift */
    int32_t knn_temporal;  /* K_T leaves of the temporal tree */
    int32_t knn_epipolar;  /* K_E leaves of each epipolar tree */
    int32_t order_mode;    /* 0: the readings above (what the CUDA path computes); bits switch
                              readings back towards the paper's own procedure, for the
                              quality comparison only: 1 = in-place sequential scans (D4),
                              2 = approximate kD-tree leaves (D3), 4 = sequential random
                              stream (D5) */
} sffo_params;

#define SFFO_SEQUENTIAL_SCAN 1
#define SFFO_KDTREE_INIT 2
#define SFFO_SEQUENTIAL_RNG 4

typedef struct {
    int16_t x, y, u, v, d0, d1;
    int32_t cost;
    uint8_t cerr;
    uint8_t pad[3];
} sffo_seed;

static int g_threads = 1;

void sffo_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int sffo_get_threads(void) { return g_threads; }

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* floor(a / 2^s) for any sign of a */
static int32_t floor_shift(int32_t a, int s) {
    int32_t d = (int32_t)1 << s;
    int32_t q = a / d;            /* C division truncates towards zero */
    if (a % d != 0 && a < 0) q -= 1;
    return q;
}

/* ---------------------------------------------------------------------------
 * Scale space (Sec. 3.1 "Multi-Scale Propagation"): the image at scale s is
 * smoothed with an n x n box (n = 2^s), every pixel kept at full resolution.
 */
void sffo_smooth(const uint8_t* img, int w, int h, int s, uint8_t* out) {
    int n = 1 << s;
    if (s == 0) { memcpy(out, img, (size_t)w * h * 3); return; }
    #pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++)
            for (int c = 0; c < 3; c++) {
                int sum = 0;
                for (int j = -n / 2; j <= n / 2 - 1; j++)
                    for (int i = -n / 2; i <= n / 2 - 1; i++) {
                        int xx = clampi(x + i, 0, w - 1), yy = clampi(y + j, 0, h - 1);
                        sum += img[((size_t)yy * w + xx) * 3 + c];
                    }
                out[((size_t)y * w + x) * 3 + c] = (uint8_t)((sum + n * n / 2) / (n * n));
            }
}

/* ---------------------------------------------------------------------------
 * Walsh-Hadamard basis in sequency order: the Sylvester Hadamard matrix of
 * order 8 with its rows sorted by their number of sign changes.
 */
static int g_walsh[8][8];
static int g_walsh_ready = 0;

static void build_walsh(void) {
    if (g_walsh_ready) return;
    int had[8][8];
    had[0][0] = 1;
    for (int size = 1; size < 8; size *= 2)          /* Sylvester: [[H, H], [H, -H]] */
        for (int i = 0; i < size; i++)
            for (int j = 0; j < size; j++) {
                had[i][j + size] = had[i][j];
                had[i + size][j] = had[i][j];
                had[i + size][j + size] = -had[i][j];
            }
    for (int r = 0; r < 8; r++) {
        int changes = 0;
        for (int j = 1; j < 8; j++) changes += had[r][j] != had[r][j - 1];
        for (int j = 0; j < 8; j++) g_walsh[changes][j] = had[r][j];   /* sequency = #changes */
    }
    g_walsh_ready = 1;
}

void sffo_walsh_matrix(int32_t* out /* [8][8] */) {
    build_walsh();
    for (int i = 0; i < 8; i++) for (int j = 0; j < 8; j++) out[i * 8 + j] = g_walsh[i][j];
}

/* The 16 kept coefficients (ky, kx): AC entries sorted by kx+ky, then ky. */
void sffo_coef_order(int32_t* ky_out, int32_t* kx_out) {
    int m = 0;
    for (int t = 1; t <= 14 && m < NCOEF; t++)
        for (int ky = 0; ky <= t && m < NCOEF; ky++) {
            int kx = t - ky;
            if (ky > 7 || kx > 7) continue;
            ky_out[m] = ky; kx_out[m] = kx; m++;
        }
}

/* Full 2-D transform T = H P H^T of one 8x8 patch (rows i = y, columns j = x). */
void sffo_wht8x8(const int32_t* patch, int32_t* coef) {
    build_walsh();
    int32_t r[8][8];
    for (int i = 0; i < 8; i++)                        /* r = P H^T */
        for (int kx = 0; kx < 8; kx++) {
            int32_t acc = 0;
            for (int j = 0; j < 8; j++) acc += patch[i * 8 + j] * g_walsh[kx][j];
            r[i][kx] = acc;
        }
    for (int ky = 0; ky < 8; ky++)                     /* T = H r */
        for (int kx = 0; kx < 8; kx++) {
            int32_t acc = 0;
            for (int i = 0; i < 8; i++) acc += g_walsh[ky][i] * r[i][kx];
            coef[ky * 8 + kx] = acc;
        }
}

/*
 * Features of one image at all scales.  feat: [S][H][W][48] int8,
 * norm: [S][H][W] int32 (sum of squared features).
 * Patch of pixel (x, y) at scale s: P_c[i][j] = S_s(x + n(j-3), y + n(i-3))_c,
 * coordinates clamped to the image (boundary replication, Sec. 3.1).
 */
void sffo_features(const uint8_t* img, int w, int h, const sffo_params* prm, int8_t* feat, int32_t* norm) {
    build_walsh();
    int ky[NCOEF], kx[NCOEF];
    sffo_coef_order(ky, kx);
    uint8_t* sm = (uint8_t*)malloc((size_t)w * h * 3);
    for (int s = 0; s < prm->num_scales; s++) {
        int n = 1 << s;
        sffo_smooth(img, w, h, s, sm);
        int8_t* fs = feat + (size_t)s * w * h * NF;
        int32_t* ns = norm + (size_t)s * w * h;
        #pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                int8_t* f = fs + ((size_t)y * w + x) * NF;
                int32_t nn = 0;
                for (int c = 0; c < 3; c++) {
                    int32_t patch[64], coef[64];
                    for (int i = 0; i < 8; i++)
                        for (int j = 0; j < 8; j++) {
                            int xx = clampi(x + n * (j - 3), 0, w - 1);
                            int yy = clampi(y + n * (i - 3), 0, h - 1);
                            patch[i * 8 + j] = sm[((size_t)yy * w + xx) * 3 + c];
                        }
                    sffo_wht8x8(patch, coef);
                    for (int m = 0; m < NCOEF; m++) {
                        int32_t q = floor_shift(coef[ky[m] * 8 + kx[m]], prm->quant_shift);
                        q = clampi(q, -128, 127);
                        f[c * NCOEF + m] = (int8_t)q;
                        nn += q * q;
                    }
                }
                ns[(size_t)y * w + x] = nn;
            }
    }
    free(sm);
}

/* ---------------------------------------------------------------------------
 * Matching cost (Eq. 1 with the feature reading): for u = (u, v, d0, d1) at p,
 *   temporal  T at p + (u, v)
 *   stereo    S at p + (-sigma d0, 0)
 *   cross     X at p + (u - sigma d1, v)
 * each position clamped to the image; cost = sum of the three SSDs.
 */
typedef struct {
    const int8_t* ref; const int8_t* tmp; const int8_t* ste; const int8_t* crs;
    int w, h, sigma;
    /* the paper's own cost instead (Eq. 1 with SIFT-PCA features, see
       sff_sift_oracle.c): phi planes of the four views at this scale, NULL
       for the WHT cost; n the scale's stride */
    const float* pref; const float* ptmp; const float* pste; const float* pcrs;
    int n;
} views_t;

float sfft_cost(const float* ref, const float* tmp, const float* ste, const float* crs, int w, int h, int n,
                int sigma, int px, int py, const int16_t* u);

static int32_t ssd(const int8_t* a, const int8_t* b) {
    int32_t acc = 0;
    for (int k = 0; k < NF; k++) { int32_t d = (int32_t)a[k] - (int32_t)b[k]; acc += d * d; }
    return acc;
}

static const int8_t* fat(const int8_t* f, int w, int h, int x, int y) {
    x = clampi(x, 0, w - 1); y = clampi(y, 0, h - 1);
    return f + ((size_t)y * w + x) * NF;
}

static int32_t cost_at(const views_t* V, int px, int py, const int16_t* u) {
    if (V->pref) {
        /* a non-negative float's bit pattern orders like the float */
        const float c = sfft_cost(V->pref, V->ptmp, V->pste, V->pcrs, V->w, V->h, V->n, V->sigma, px, py, u);
        int32_t b;
        memcpy(&b, &c, sizeof b);
        return b;
    }
    const int8_t* a = V->ref + ((size_t)py * V->w + px) * NF;
    int32_t c = 0;
    c += ssd(a, fat(V->tmp, V->w, V->h, px + u[0], py + u[1]));
    c += ssd(a, fat(V->ste, V->w, V->h, px - V->sigma * u[2], py));
    c += ssd(a, fat(V->crs, V->w, V->h, px + u[0] - V->sigma * u[3], py + u[1]));
    return c;
}

/* Exported for tests: cost of one vector at one pixel, features at one scale. */
int32_t sffo_cost(const int8_t* ref, const int8_t* tmp, const int8_t* ste, const int8_t* crs,
                  int w, int h, int mirror, int px, int py, const int16_t* u) {
    views_t V = {ref, tmp, ste, crs, w, h, mirror ? -1 : 1, NULL, NULL, NULL, NULL, 1};
    return cost_at(&V, px, py, u);
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of a
 * multiply-based S-box on four 32-bit words, the key bumped by a Weyl
 * sequence between rounds.
 */
void sffo_philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k[0] += W0; k[1] += W1; }
        uint64_t p0 = (uint64_t)M0 * c[0];
        uint64_t p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Random-search offset in full-resolution pixels: the nearest integer to a
 * uniform draw on ]-n, n[, realised from r as floor((floor(r*4n/2^32)+1)/2) - n. */
int32_t sffo_rs_offset(uint32_t r, int n) {
    uint32_t j = (uint32_t)(((uint64_t)r * (uint64_t)(4 * n)) >> 32);
    return (int32_t)((j + 1) / 2) - n;
}

/* ---------------------------------------------------------------------------
 * Exact K nearest neighbours: the K smallest (distance, raster index) pairs.
 */
typedef struct { int32_t d; int32_t idx; } cand_t;

static void knn_insert(cand_t* list, int* count, int K, int32_t d, int32_t idx) {
    /* keep list sorted ascending by (d, idx) */
    if (*count == K) {
        cand_t last = list[K - 1];
        if (d > last.d || (d == last.d && idx > last.idx)) return;
        (*count)--;
    }
    int pos = *count;
    while (pos > 0 && (list[pos - 1].d > d || (list[pos - 1].d == d && list[pos - 1].idx > idx))) {
        list[pos] = list[pos - 1]; pos--;
    }
    list[pos].d = d; list[pos].idx = idx;
    (*count)++;
}

static void init_coarsest(const views_t* V, int s, const sffo_params* prm, int16_t* field, int32_t* cost) {
    int w = V->w, h = V->h, n = 1 << s;
    int KT = prm->knn_temporal, KE = prm->knn_epipolar;
    #pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int py = 0; py < h; py += n) {
        cand_t tl[64], sl[64], xl[64];
        for (int px = 0; px < w; px += n) {
            const int8_t* a = V->ref + ((size_t)py * w + px) * NF;
            /* temporal tree: whole coarsest grid */
            int nt = 0;
            for (int qy = 0; qy < h; qy += n)
                for (int qx = 0; qx < w; qx += n)
                    knn_insert(tl, &nt, KT, ssd(a, V->tmp + ((size_t)qy * w + qx) * NF), qy * w + qx);
            /* stereo epipolar tree: row py, d0 = sigma (px - qx) >= 0 */
            int ns = 0;
            for (int qx = 0; qx < w; qx += n)
                if (V->sigma * (px - qx) >= 0)
                    knn_insert(sl, &ns, KE, ssd(a, V->ste + ((size_t)py * w + qx) * NF), py * w + qx);
            int32_t best_c = EMPTY_COST;
            int16_t best_u[4] = {0, 0, 0, 0};
            for (int it = 0; it < nt; it++) {
                int tx = tl[it].idx % w, ty = tl[it].idx / w;
                /* cross epipolar tree: row ty, d1 = sigma (tx - qx) >= 0 */
                int nx = 0;
                for (int qx = 0; qx < w; qx += n)
                    if (V->sigma * (tx - qx) >= 0)
                        knn_insert(xl, &nx, KE, ssd(a, V->crs + ((size_t)ty * w + qx) * NF), ty * w + qx);
                for (int is = 0; is < ns; is++)
                    for (int ix = 0; ix < nx; ix++) {
                        int sx = sl[is].idx % w, cx = xl[ix].idx % w;
                        int16_t u[4];
                        u[0] = (int16_t)(tx - px);
                        u[1] = (int16_t)(ty - py);
                        u[2] = (int16_t)(V->sigma * (px - sx));
                        u[3] = (int16_t)(V->sigma * (tx - cx));
                        int32_t c = cost_at(V, px, py, u);
                        if (c < best_c) { best_c = c; memcpy(best_u, u, sizeof best_u); }
                    }
            }
            memcpy(field + ((size_t)py * w + px) * 4, best_u, sizeof best_u);
            cost[(size_t)py * w + px] = best_c;
        }
    }
}

/* ---------------------------------------------------------------------------
 * The paper's approximate initialisation (Sec. 3.1 "Initialization"), for the
 * quality comparison of reading D3: kD-trees over the coarsest-grid features
 * of the temporal image and, per grid row, of the stereo and cross images
 * ("epipolar" trees); a query descends to one leaf and all combinations of
 * the leaves' points are scored with the full cost.  Trees: median split on
 * the dimension of largest spread, leaves of at most 8 points, single
 * descent without backtracking.
 */
typedef struct { int dim, split, left, right, start, count; } kdnode;

typedef struct {
    kdnode* nodes; int nn, cap;
    int* idx;          /* raster indices, permuted so that leaves are contiguous */
    const int8_t* f;   /* feature plane [H][W][48] */
} kdtree;

static const int8_t* g_sort_f;
static int g_sort_dim;
static int cmp_dim(const void* a, const void* b) {
    int ia = *(const int*)a, ib = *(const int*)b;
    int va = g_sort_f[(size_t)ia * NF + g_sort_dim], vb = g_sort_f[(size_t)ib * NF + g_sort_dim];
    if (va != vb) return va < vb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib);
}

static int kd_build(kdtree* T, int start, int count) {
    if (T->nn == T->cap) { T->cap = T->cap ? 2 * T->cap : 64; T->nodes = (kdnode*)realloc(T->nodes, T->cap * sizeof(kdnode)); }
    int id = T->nn++;
    kdnode nd = {0, 0, -1, -1, start, count};
    if (count > 8) {
        int best_dim = 0, best_spread = -1;
        for (int d = 0; d < NF; d++) {
            int lo = 127, hi = -128;
            for (int k = 0; k < count; k++) {
                int v = T->f[(size_t)T->idx[start + k] * NF + d];
                if (v < lo) lo = v;
                if (v > hi) hi = v;
            }
            if (hi - lo > best_spread) { best_spread = hi - lo; best_dim = d; }
        }
        g_sort_f = T->f; g_sort_dim = best_dim;
        qsort(T->idx + start, count, sizeof(int), cmp_dim);
        int m = count / 2;
        nd.dim = best_dim;
        nd.split = T->f[(size_t)T->idx[start + m] * NF + best_dim];
        int l = kd_build(T, start, m);
        int r = kd_build(T, start + m, count - m);
        nd.left = l; nd.right = r;
    }
    T->nodes[id] = nd;
    return id;
}

static void kd_init(kdtree* T, const int8_t* f, const int* pts, int n) {
    T->nodes = NULL; T->nn = T->cap = 0; T->f = f;
    T->idx = (int*)malloc((n > 0 ? n : 1) * sizeof(int));
    memcpy(T->idx, pts, n * sizeof(int));
    if (n > 0) kd_build(T, 0, n);
}

static void kd_free(kdtree* T) { free(T->nodes); free(T->idx); }

/* the leaf a query descends to: its points T->idx[*start .. *start + *count) */
static void kd_leaf(const kdtree* T, const int8_t* q, int* start, int* count) {
    int node = 0;
    while (T->nodes[node].left >= 0) node = q[T->nodes[node].dim] < T->nodes[node].split ? T->nodes[node].left : T->nodes[node].right;
    *start = T->nodes[node].start; *count = T->nodes[node].count;
}

static void init_kdtree(const views_t* V, int s, const sffo_params* prm, int16_t* field, int32_t* cost) {
    int w = V->w, h = V->h, n = 1 << s;
    int gw = (w + n - 1) / n, gh = (h + n - 1) / n;
    int* pts = (int*)malloc((size_t)gw * gh * sizeof(int));
    int np = 0;
    for (int y = 0; y < h; y += n) for (int x = 0; x < w; x += n) pts[np++] = y * w + x;
    kdtree tt; kd_init(&tt, V->tmp, pts, np);
    kdtree* st = (kdtree*)malloc(gh * sizeof(kdtree));
    kdtree* xt = (kdtree*)malloc(gh * sizeof(kdtree));
    for (int r = 0; r < gh; r++) { kd_init(&st[r], V->ste, pts + r * gw, gw); kd_init(&xt[r], V->crs, pts + r * gw, gw); }
    int KT = prm->knn_temporal, KE = prm->knn_epipolar;
    #pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int py = 0; py < h; py += n) {
        cand_t tl[64], sl[64], xl[64];
        for (int px = 0; px < w; px += n) {
            const int8_t* a = V->ref + ((size_t)py * w + px) * NF;
            int ls, lc, nt = 0, ns = 0;
            kd_leaf(&tt, a, &ls, &lc);
            for (int k = 0; k < lc; k++) { int q = tt.idx[ls + k]; knn_insert(tl, &nt, KT, ssd(a, V->tmp + (size_t)q * NF), q); }
            const kdtree* S = &st[py / n];
            kd_leaf(S, a, &ls, &lc);
            for (int k = 0; k < lc; k++) {
                int q = S->idx[ls + k];
                if (V->sigma * (px - q % w) >= 0) knn_insert(sl, &ns, KE, ssd(a, V->ste + (size_t)q * NF), q);
            }
            if (ns == 0) /* no leaf point satisfies d0 >= 0: the pixel's own column is always valid */
                knn_insert(sl, &ns, KE, ssd(a, V->ste + ((size_t)py * w + px) * NF), py * w + px);
            int32_t best_c = EMPTY_COST;
            int16_t best_u[4] = {0, 0, 0, 0};
            for (int it = 0; it < nt; it++) {
                int tx = tl[it].idx % w, ty = tl[it].idx / w, nx = 0;
                const kdtree* X = &xt[ty / n];
                kd_leaf(X, a, &ls, &lc);
                for (int k = 0; k < lc; k++) {
                    int q = X->idx[ls + k];
                    if (V->sigma * (tx - q % w) >= 0) knn_insert(xl, &nx, KE, ssd(a, V->crs + (size_t)q * NF), q);
                }
                if (nx == 0) knn_insert(xl, &nx, KE, ssd(a, V->crs + ((size_t)ty * w + tx) * NF), ty * w + tx);
                for (int is = 0; is < ns; is++)
                    for (int ix = 0; ix < nx; ix++) {
                        int sx = sl[is].idx % w, cx = xl[ix].idx % w;
                        int16_t u[4] = {(int16_t)(tx - px), (int16_t)(ty - py), (int16_t)(V->sigma * (px - sx)),
                                        (int16_t)(V->sigma * (tx - cx))};
                        int32_t c = cost_at(V, px, py, u);
                        if (c < best_c) { best_c = c; memcpy(best_u, u, sizeof best_u); }
                    }
            }
            memcpy(field + ((size_t)py * w + px) * 4, best_u, sizeof best_u);
            cost[(size_t)py * w + px] = best_c;
        }
    }
    kd_free(&tt);
    for (int r = 0; r < gh; r++) { kd_free(&st[r]); kd_free(&xt[r]); }
    free(st); free(xt); free(pts);
}

/* Sequential random stream for reading D5's comparison: splitmix64 (Steele,
 * Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA'14). */
static uint64_t splitmix64(uint64_t* st) {
    uint64_t z = (*st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------------------------
 * Field estimation for one reference view (forward: mirror = 0, reference L0,
 * temporal L1, stereo R0, cross R1; inverse: mirror = 1, reference R1,
 * temporal R0, stereo L1, cross L0).  feat_*: [S][H][W][48] from sffo_features.
 * field: [H][W][4] int16 (u, v, d0, d1), cost: [H][W] int32 (INT32_MAX = empty).
 */
static void match_views(const int8_t* f_ref, const int8_t* f_tmp, const int8_t* f_ste, const int8_t* f_crs,
                        const float* const* phi, int w, int h, int mirror, uint64_t seed, const sffo_params* prm,
                        int16_t* field, int32_t* cost);

void sffo_match_views(const int8_t* f_ref, const int8_t* f_tmp, const int8_t* f_ste, const int8_t* f_crs,
                      int w, int h, int mirror, uint64_t seed, const sffo_params* prm,
                      int16_t* field, int32_t* cost) {
    match_views(f_ref, f_tmp, f_ste, f_crs, NULL, w, h, mirror, seed, prm, field, cost);
}

/* The same with the paper's own cost (Eq. 1, SIFT-PCA features): phi_*
 * [S][H][W][4] of the four views in the roles of the field; the WHT
 * features still drive the initialisation's nearest-neighbour search (Sec.
 * 3.1 "Initialization"), whose combinations are scored with this cost.
 * cost: the float costs as int32 bit patterns. */
void sffo_match_views_sift(const int8_t* f_ref, const int8_t* f_tmp, const int8_t* f_ste, const int8_t* f_crs,
                           const float* phi_ref, const float* phi_tmp, const float* phi_ste, const float* phi_crs,
                           int w, int h, int mirror, uint64_t seed, const sffo_params* prm, int16_t* field,
                           int32_t* cost) {
    const float* phi[4] = {phi_ref, phi_tmp, phi_ste, phi_crs};
    match_views(f_ref, f_tmp, f_ste, f_crs, phi, w, h, mirror, seed, prm, field, cost);
}

static void match_views(const int8_t* f_ref, const int8_t* f_tmp, const int8_t* f_ste, const int8_t* f_crs,
                        const float* const* phi, int w, int h, int mirror, uint64_t seed, const sffo_params* prm,
                        int16_t* field, int32_t* cost) {
    const int S = prm->num_scales;
    const size_t np = (size_t)w * h;
    static const int DIRS[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int16_t* snap_f = (int16_t*)malloc(np * 4 * sizeof(int16_t));
    int32_t* snap_c = (int32_t*)malloc(np * sizeof(int32_t));

    for (size_t i = 0; i < np; i++) { cost[i] = EMPTY_COST; field[4 * i] = field[4 * i + 1] = field[4 * i + 2] = field[4 * i + 3] = 0; }

    for (int s = S - 1; s >= 0; s--) {
        int n = 1 << s;
        size_t off = (size_t)s * np * NF;
        views_t V = {f_ref + off, f_tmp + off, f_ste + off, f_crs + off, w, h, mirror ? -1 : 1, NULL, NULL, NULL, NULL, n};
        if (phi) {
            const size_t po = (size_t)s * np * 4;
            V.pref = phi[0] + po;
            V.ptmp = phi[1] + po;
            V.pste = phi[2] + po;
            V.pcrs = phi[3] + po;
        }

        if (s == S - 1) {
            /* initialisation on the coarsest scale only (Sec. 3.1) */
            if (prm->order_mode & SFFO_KDTREE_INIT) init_kdtree(&V, s, prm, field, cost);
            else init_coarsest(&V, s, prm, field, cost);
        } else {
            /* points of the coarser grid keep their vector, re-scored at this
               scale; all other points of this grid start empty */
            #pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int y = 0; y < h; y += n)
                for (int x = 0; x < w; x += n) {
                    size_t i = (size_t)y * w + x;
                    int coarse = (x % (2 * n) == 0) && (y % (2 * n) == 0);
                    if (coarse && cost[i] != EMPTY_COST) {
                        cost[i] = cost_at(&V, x, y, field + 4 * i);
                    } else {
                        cost[i] = EMPTY_COST;
                        field[4 * i] = field[4 * i + 1] = field[4 * i + 2] = field[4 * i + 3] = 0;
                    }
                }
        }

        for (int it = 0; it < prm->iterations; it++) {
            int dx = DIRS[it % 4][0], dy = DIRS[it % 4][1];
            if (prm->order_mode & SFFO_SEQUENTIAL_SCAN) {
                /* the paper's order: one in-place raster sweep in the
                   iteration's direction; each pixel sees its predecessors'
                   values of this sweep */
                int gw = (w + n - 1) / n, gh = (h + n - 1) / n;
                for (int gyk = 0; gyk < gh; gyk++)
                    for (int gxk = 0; gxk < gw; gxk++) {
                        int x = (dx > 0 ? gxk : gw - 1 - gxk) * n, y = (dy > 0 ? gyk : gh - 1 - gyk) * n;
                        size_t i = (size_t)y * w + x;
                        int qx[2] = {x - dx * n, x}, qy[2] = {y, y - dy * n};
                        for (int k = 0; k < 2; k++) {
                            if (qx[k] < 0 || qx[k] >= w || qy[k] < 0 || qy[k] >= h) continue;
                            size_t j = (size_t)qy[k] * w + qx[k];
                            if (cost[j] == EMPTY_COST) continue;
                            int32_t c = cost_at(&V, x, y, field + 4 * j);
                            if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, field + 4 * j, 4 * sizeof(int16_t)); }
                        }
                    }
            } else
            /* propagation: two synchronous half-steps over the grid colours */
            for (int colour = 0; colour < 2; colour++) {
                memcpy(snap_f, field, np * 4 * sizeof(int16_t));
                memcpy(snap_c, cost, np * sizeof(int32_t));
                #pragma omp parallel for num_threads(g_threads) schedule(static)
                for (int y = 0; y < h; y += n)
                    for (int x = 0; x < w; x += n) {
                        if (((x / n + y / n) & 1) != colour) continue;
                        size_t i = (size_t)y * w + x;
                        int32_t best_c = snap_c[i];
                        int16_t best_u[4];
                        memcpy(best_u, snap_f + 4 * i, sizeof best_u);
                        int qx[2] = {x - dx * n, x}, qy[2] = {y, y - dy * n};
                        for (int k = 0; k < 2; k++) {
                            if (qx[k] < 0 || qx[k] >= w || qy[k] < 0 || qy[k] >= h) continue;
                            size_t j = (size_t)qy[k] * w + qx[k];
                            if (snap_c[j] == EMPTY_COST) continue;
                            int32_t c = cost_at(&V, x, y, snap_f + 4 * j);
                            if (c < best_c) { best_c = c; memcpy(best_u, snap_f + 4 * j, sizeof best_u); }
                        }
                        memcpy(field + 4 * i, best_u, sizeof best_u);
                        cost[i] = best_c;
                    }
            }
            /* random search after the iteration: every non-empty grid pixel */
            if (prm->order_mode & SFFO_SEQUENTIAL_RNG) {
                /* one sequential stream in raster order */
                uint64_t st = seed ^ ((uint64_t)(s + 4 * mirror) << 40) ^ ((uint64_t)it << 48);
                for (int y = 0; y < h; y += n)
                    for (int x = 0; x < w; x += n) {
                        size_t i = (size_t)y * w + x;
                        if (cost[i] == EMPTY_COST) continue;
                        uint64_t r0 = splitmix64(&st), r1 = splitmix64(&st);
                        uint32_t r[4] = {(uint32_t)r0, (uint32_t)(r0 >> 32), (uint32_t)r1, (uint32_t)(r1 >> 32)};
                        int32_t cu[4];
                        for (int k = 0; k < 4; k++) cu[k] = field[4 * i + k] + sffo_rs_offset(r[k], n);
                        if (cu[2] < 0) cu[2] = 0;
                        if (cu[3] < 0) cu[3] = 0;
                        int16_t cand[4] = {(int16_t)cu[0], (int16_t)cu[1], (int16_t)cu[2], (int16_t)cu[3]};
                        int32_t c = cost_at(&V, x, y, cand);
                        if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }
                    }
                continue;
            }
            #pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int y = 0; y < h; y += n)
                for (int x = 0; x < w; x += n) {
                    size_t i = (size_t)y * w + x;
                    if (cost[i] == EMPTY_COST) continue;
                    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u}, r[4];
                    sffo_philox4x32_10(ctr, key, r);
                    int32_t cu[4];
                    for (int k = 0; k < 4; k++) cu[k] = field[4 * i + k] + sffo_rs_offset(r[k], n);
                    if (cu[2] < 0) cu[2] = 0;
                    if (cu[3] < 0) cu[3] = 0;
                    int16_t cand[4] = {(int16_t)cu[0], (int16_t)cu[1], (int16_t)cu[2], (int16_t)cu[3]};
                    int32_t c = cost_at(&V, x, y, cand);
                    if (c < cost[i]) { cost[i] = c; memcpy(field + 4 * i, cand, sizeof cand); }
                }
        }
    }
    free(snap_f);
    free(snap_c);
}

/* ---------------------------------------------------------------------------
 * Consistency check and region filter (Sec. 3.1 "Consistency Check").
 * fwd/inv: [H][W][4] fields of L0 and R1; *_cost: INT32_MAX marks empty.
 * keep: [H][W] 1 = kept; cerr: [H][W] sum of |round-trip differences|
 * (255 when rejected without a comparison).
 */
static int vec_close(const int16_t* a, const int16_t* b, int tau) {
    for (int k = 0; k < 4; k++) if (abs((int)a[k] - (int)b[k]) > tau) return 0;
    return 1;
}

void sffo_consistency_check(const int16_t* fwd, const int32_t* fwd_cost, const int16_t* inv, const int32_t* inv_cost,
                            int w, int h, const sffo_params* prm, uint8_t* keep, uint8_t* cerr) {
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            size_t i = (size_t)y * w + x;
            keep[i] = 0; cerr[i] = 255;
            if (fwd_cost[i] == EMPTY_COST) continue;
            const int16_t* u = fwd + 4 * i;
            int qx = x + u[0] - u[3], qy = y + u[1];          /* the cross correspondence in R1 */
            if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
            size_t j = (size_t)qy * w + qx;
            if (inv_cost[j] == EMPTY_COST) continue;
            const int16_t* iu = inv + 4 * j;
            int dlt[4];
            dlt[0] = iu[0] + u[0] - u[3] + u[2];   /* right-camera flow R0->R1 vs inverse R1->R0 */
            dlt[1] = iu[1] + u[1];
            dlt[2] = iu[2] - u[3];                 /* disparity at t1 */
            dlt[3] = iu[3] - u[2];                 /* disparity at t0 */
            int mx = 0, sum = 0;
            for (int k = 0; k < 4; k++) { int a = abs(dlt[k]); if (a > mx) mx = a; sum += a; }
            cerr[i] = (uint8_t)(sum > 255 ? 255 : sum);
            keep[i] = mx <= prm->tau_c;
        }
}

void sffo_region_filter(const int16_t* fwd, const int32_t* fwd_cost, int w, int h, const sffo_params* prm,
                        uint8_t* keep /* in: consistency result, out: filtered */) {
    size_t np = (size_t)w * h;
    int32_t* label = (int32_t*)malloc(np * sizeof(int32_t));
    int32_t* queue = (int32_t*)malloc(np * sizeof(int32_t));
    uint8_t* rejected = (uint8_t*)malloc(np);
    for (size_t i = 0; i < np; i++) { label[i] = -1; rejected[i] = !keep[i] && fwd_cost[i] != EMPTY_COST; }
    static const int NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    for (size_t start = 0; start < np; start++) {
        if (!keep[start] || label[start] >= 0) continue;
        /* breadth-first growth of one region */
        int head = 0, tail = 0, joinable = 0;
        queue[tail++] = (int32_t)start;
        label[start] = (int32_t)start;
        while (head < tail) {
            int32_t i = queue[head++];
            int x = i % w, y = i / w;
            for (int k = 0; k < 4; k++) {
                int nx = x + NB[k][0], ny = y + NB[k][1];
                if (nx < 0 || nx >= w || ny < 0 || ny >= h) continue;
                int32_t j = ny * w + nx;
                if (!vec_close(fwd + 4 * (size_t)i, fwd + 4 * (size_t)j, prm->tau_r)) continue;
                if (keep[j]) {
                    if (label[j] < 0) { label[j] = (int32_t)start; queue[tail++] = j; }
                } else if (rejected[j]) {
                    joinable = 1;   /* a removed outlier could join this region */
                }
            }
        }
        if (joinable && tail < prm->region_min)
            for (int k = 0; k < tail; k++) keep[queue[k]] = 0;
    }
    free(label); free(queue); free(rejected);
}

void sffo_consistency_filter(const int16_t* fwd, const int32_t* fwd_cost, const int16_t* inv, const int32_t* inv_cost,
                             int w, int h, const sffo_params* prm, uint8_t* keep, uint8_t* cerr) {
    sffo_consistency_check(fwd, fwd_cost, inv, inv_cost, w, h, prm, keep, cerr);
    sffo_region_filter(fwd, fwd_cost, w, h, prm, keep);
}

/* ---------------------------------------------------------------------------
 * Sparsification (Sec. 3.2): per non-overlapping 3x3 block, the kept match
 * with the lowest consistency error (then cost, then raster index).
 * Returns the number of seeds; writes at most `capacity`.
 */
int sffo_emit_seeds(const int16_t* fwd, const int32_t* fwd_cost, const uint8_t* keep, const uint8_t* cerr,
                    int w, int h, sffo_seed* out, int capacity) {
    int count = 0;
    for (int by = 0; by < h; by += 3)
        for (int bx = 0; bx < w; bx += 3) {
            int best = -1;
            for (int y = by; y < by + 3 && y < h; y++)
                for (int x = bx; x < bx + 3 && x < w; x++) {
                    int i = y * w + x;
                    if (!keep[i]) continue;
                    if (best < 0 || cerr[i] < cerr[best] ||
                        (cerr[i] == cerr[best] && fwd_cost[i] < fwd_cost[best]))
                        best = i;   /* raster order visits lower indices first: ties keep them */
                }
            if (best < 0) continue;
            if (count < capacity) {
                sffo_seed* sd = out + count;
                memset(sd, 0, sizeof *sd);
                sd->x = (int16_t)(best % w); sd->y = (int16_t)(best / w);
                sd->u = fwd[4 * (size_t)best]; sd->v = fwd[4 * (size_t)best + 1];
                sd->d0 = fwd[4 * (size_t)best + 2]; sd->d1 = fwd[4 * (size_t)best + 3];
                sd->cost = fwd_cost[best]; sd->cerr = cerr[best];
            }
            count++;
        }
    return count;
}
