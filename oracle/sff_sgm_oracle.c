/*
 * Plain CPU oracle of SceneFlowFields' disparity fill (Schuster et al., WACV
 * 2018, Sec. 3.1, last paragraph): a second disparity map of L0/R0 by
 * semi-global matching (Hirschmueller, PAMI 2008), the matching's own d0
 * kept as a disparity-only value wherever it agrees with that map within
 * tau_c, and disparity-only seeds for the 3x3 blocks that hold no jointly
 * consistent match (Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY: the slow statement of what the CUDA path
 * computes, loaded by the tests and the benchmark's CPU leg.  It shares no
 * source with the CUDA path.
 *
 * The paper names SGM and the shared threshold tau_c but no SGM details.
 * Readings (implemented identically by the CUDA path):
 *   - grey value (R + 2G + B + 2) >> 2;
 *   - census transform over a 9 x 7 window (width 9, height 7): bit k, k in
 *     row-major window order with the centre skipped, is set when the
 *     neighbour is darker than the centre; coordinates clamped to the image;
 *   - matching cost C(p, d) = number of differing census bits between L0 at
 *     (x, y) and R0 at (max(x - d, 0), y), d = 0 .. D - 1;
 *   - aggregation along 8 directions r (the 4 axes and the 4 diagonals):
 *       L_r(p, d) = C(p, d) + min(L_r(p-r, d), L_r(p-r, d-1) + P1,
 *                                 L_r(p-r, d+1) + P1, min_k L_r(p-r, k) + P2)
 *                   - min_k L_r(p-r, k),
 *     L_r(p, d) = C(p, d) where p - r is outside the image;
 *   - disparity = argmin_d sum_r L_r(p, d), ties to the lowest d; no
 *     left-right or uniqueness check (the check that matters is against the
 *     matching's d0);
 *   - a pixel holding a vector (cost not empty) is disparity-valid when
 *     |d0 - d_sgm| <= tau_c;
 *   - seeds: per 3x3 block the jointly consistent seed of Sec. 3.2 when the
 *     block has one; otherwise the disparity-valid pixel with the lowest
 *     |d0 - d_sgm|, then cost, then raster index, as a disparity-only seed
 *     (kind 1, u = v = d1 = 0, cerr = |d0 - d_sgm|).
 * Pins: tests/test_oracle_sgm.py (census of closed-form images, every path
 * value against brute force over all disparity sequences, the P1 = P2 = 0
 * reduction to per-pixel winner-takes-all, integer-shift images, hand-built
 * seed blocks).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

typedef struct {
    int32_t max_disp, p1, p2;
} sffs_params;

typedef struct {
    int16_t x, y, u, v, d0, d1;
    int32_t cost;
    uint8_t cerr;
    uint8_t kind;
    uint8_t pad[2];
} sffs_seed;

static int g_sthreads = 1;
void sffs_set_threads(int n) { g_sthreads = n < 1 ? 1 : n; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

void sffs_grey(const uint8_t* rgb, int pitch, int W, int H, uint8_t* grey) {
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const uint8_t* p = rgb + (size_t)y * pitch + 3 * x;
            grey[(size_t)y * W + x] = (uint8_t)((p[0] + 2 * p[1] + p[2] + 2) >> 2);
        }
}

void sffs_census(const uint8_t* grey, int W, int H, uint64_t* out) {
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const int c = grey[(size_t)y * W + x];
            uint64_t bits = 0;
            int k = 0;
            for (int j = -3; j <= 3; j++)
                for (int i = -4; i <= 4; i++) {
                    if (i == 0 && j == 0) continue;
                    const int q = grey[(size_t)clampi(y + j, 0, H - 1) * W + clampi(x + i, 0, W - 1)];
                    if (q < c) bits |= (uint64_t)1 << k;
                    k++;
                }
            out[(size_t)y * W + x] = bits;
        }
}

static int popcount64(uint64_t v) {
    int n = 0;
    while (v) {
        v &= v - 1;
        n++;
    }
    return n;
}

void sffs_cost_volume(const uint64_t* cL, const uint64_t* cR, int W, int H, int D, uint8_t* C) {
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < D; d++) {
                const int xr = x - d < 0 ? 0 : x - d;
                C[((size_t)y * W + x) * D + d] = (uint8_t)popcount64(cL[(size_t)y * W + x] ^ cR[(size_t)y * W + xr]);
            }
}

/* L_r of one direction (rx, ry) in {-1, 0, 1}^2 \ {0} over a cost volume
 * C[y][x][d]; L out as [y][x][d].  Pixels are visited so that p - r comes
 * before p: rows in the direction of ry, within a row in the direction of rx. */
void sffs_path(const uint8_t* C, int W, int H, int D, int P1, int P2, int rx, int ry, uint16_t* L) {
    for (int t = 0; t < H; t++) {
        const int y = ry >= 0 ? t : H - 1 - t;
        for (int s = 0; s < W; s++) {
            const int x = rx >= 0 ? s : W - 1 - s;
            const size_t i = ((size_t)y * W + x) * D;
            const int px = x - rx, py = y - ry;
            if (px < 0 || py < 0 || px >= W || py >= H) {
                for (int d = 0; d < D; d++) L[i + d] = C[i + d];
                continue;
            }
            const uint16_t* prev = L + ((size_t)py * W + px) * D;
            int m = prev[0];
            for (int d = 1; d < D; d++)
                if (prev[d] < m) m = prev[d];
            for (int d = 0; d < D; d++) {
                int best = prev[d];
                if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
                if (d + 1 < D && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
                if (m + P2 < best) best = m + P2;
                L[i + d] = (uint16_t)(C[i + d] + best - m);
            }
        }
    }
}

static const int kDirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

/* Winner-takes-all over the sum of the 8 directions of a cost volume. */
void sffs_sgm_from_cost(const uint8_t* C, int W, int H, int D, int P1, int P2, int16_t* disp) {
    const size_t n = (size_t)W * H * D;
    uint32_t* S = (uint32_t*)calloc(n, sizeof(uint32_t));
    uint16_t* L[8];
    #pragma omp parallel for num_threads(g_sthreads) schedule(static, 1)
    for (int r = 0; r < 8; r++) {
        L[r] = (uint16_t*)malloc(n * sizeof(uint16_t));
        sffs_path(C, W, H, D, P1, P2, kDirs[r][0], kDirs[r][1], L[r]);
    }
    for (int r = 0; r < 8; r++) {
        for (size_t i = 0; i < n; i++) S[i] += L[r][i];
        free(L[r]);
    }
    for (size_t p = 0; p < (size_t)W * H; p++) {
        int best = 0;
        for (int d = 1; d < D; d++)
            if (S[p * D + d] < S[p * D + best]) best = d;
        disp[p] = (int16_t)best;
    }
    free(S);
}

/* The SGM disparity map of L0 (left) against R0 (right), both H x W x 3
 * uint8 with row pitch `pitch` bytes. */
void sffs_sgm(const uint8_t* left, const uint8_t* right, int pitch, int W, int H, const sffs_params* P,
              int16_t* disp) {
    const size_t np = (size_t)W * H;
    uint8_t* gl = (uint8_t*)malloc(np);
    uint8_t* gr = (uint8_t*)malloc(np);
    uint64_t* cl = (uint64_t*)malloc(np * 8);
    uint64_t* cr = (uint64_t*)malloc(np * 8);
    uint8_t* C = (uint8_t*)malloc(np * P->max_disp);
    sffs_grey(left, pitch, W, H, gl);
    sffs_grey(right, pitch, W, H, gr);
    sffs_census(gl, W, H, cl);
    sffs_census(gr, W, H, cr);
    sffs_cost_volume(cl, cr, W, H, P->max_disp, C);
    sffs_sgm_from_cost(C, W, H, P->max_disp, P->p1, P->p2, disp);
    free(gl);
    free(gr);
    free(cl);
    free(cr);
    free(C);
}

/* Seeds with the disparity fill: fwd [H][W][4] int16, fwd_cost [H][W]
 * int32 (INT32_MAX = no vector), keep / cerr [H][W] uint8, sgm [H][W]
 * int16.  Writes up to `cap` seeds in block raster order; returns the
 * number of seeds. */
int sffs_emit_seeds_geo(const int16_t* fwd, const int32_t* fcost, const uint8_t* keep, const uint8_t* cerr,
                        const int16_t* sgm, int W, int H, int tau_c, sffs_seed* out, int cap) {
    int n = 0;
    for (int by = 0; by < H; by += 3)
        for (int bx = 0; bx < W; bx += 3) {
            int bj = -1, bje = 0, bjc = 0;  /* jointly consistent: (cerr, cost, raster) */
            int bg = -1, bge = 0, bgc = 0;  /* disparity-only: (|d0 - sgm|, cost, raster) */
            for (int y = by; y < by + 3 && y < H; y++)
                for (int x = bx; x < bx + 3 && x < W; x++) {
                    const int i = y * W + x;
                    if (keep[i]) {
                        if (bj < 0 || cerr[i] < bje || (cerr[i] == bje && fcost[i] < bjc)) {
                            bj = i;
                            bje = cerr[i];
                            bjc = fcost[i];
                        }
                    } else if (fcost[i] != INT32_MAX) {
                        const int e = abs(fwd[4 * i + 2] - sgm[i]);
                        if (e <= tau_c && (bg < 0 || e < bge || (e == bge && fcost[i] < bgc))) {
                            bg = i;
                            bge = e;
                            bgc = fcost[i];
                        }
                    }
                }
            const int i = bj >= 0 ? bj : bg;
            if (i < 0) continue;
            if (n < cap) {
                sffs_seed s;
                memset(&s, 0, sizeof s);
                s.x = (int16_t)(i % W);
                s.y = (int16_t)(i / W);
                s.d0 = fwd[4 * i + 2];
                s.cost = fcost[i];
                if (bj >= 0) {
                    s.u = fwd[4 * i];
                    s.v = fwd[4 * i + 1];
                    s.d1 = fwd[4 * i + 3];
                    s.cerr = cerr[i];
                } else {
                    s.cerr = (uint8_t)bge;
                    s.kind = 1;
                }
                out[n] = s;
            }
            n++;
        }
    return n;
}
