/*
 * sff.h -- C ABI of the GB300 (sm_103a) implementation of SceneFlowFields'
 * sparse four-view matching stage (Schuster, Wasenmueller, Kuschk, Bailer,
 * Stricker, "SceneFlowFields: Dense Interpolation of Sparse Scene Flow
 * Correspondences", WACV 2018).
 *
 * Problem statement (Sec. 3): two rectified stereo pairs L0 = I_l^0,
 * R0 = I_r^0 (time t0) and L1 = I_l^1, R1 = I_r^1 (time t1).  For every pixel
 * p of the reference view the stage estimates the scene flow vector
 * u = (u, v, d0, d1): optical flow (u, v) to L1 and the disparities d0 (to R0)
 * and d1 (L1 to R1), so that the three correspondences of Eq. 1 are
 *     temporal  L1 at p + (u, v)
 *     stereo    R0 at p + (-d0, 0)
 *     cross     R1 at p + (u - d1, v).
 * The four calls below are the four parts of Sec. 3.1-3.2:
 *     sff_features            Walsh-Hadamard patch features on a scale space
 *     sff_match_views         initialisation + multi-scale propagation + random search
 *     sff_consistency_filter  forward/inverse consistency check + region filter
 *     sff_emit_seeds          3x3 sparsification into seeds (Sec. 3.2)
 * the paper's own cost (Sec. 3.1, Eq. 1 with SIFT-PCA features):
 *     sff_sift_features, sff_match_views_sift
 * the disparity fill (Sec. 3.1, last paragraph):
 *     sff_sgm, sff_emit_seeds_geo   SGM disparity map, disparity-only seeds
 * and the dense interpolation of the seeds (Sec. 3.2):
 *     sff_interpolate         per-seed plane and affine 3D motion, per-pixel evaluation
 *
 * Conventions for every call:
 *   - Pointers named *_dev, and every image/pyramid/field buffer, are DEVICE
 *     pointers owned by the caller; the library never allocates, frees or
 *     retains them.  `params` is a HOST pointer read during the call only.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued asynchronously on it; results are valid once the stream has
 *     reached the point of the call.  No call synchronises the host.
 *   - `workspace`/`workspace_bytes` is caller-owned device scratch of at
 *     least sff_workspace_bytes() bytes, 256-byte aligned; its contents are
 *     undefined between calls.  Calls that share one workspace must be
 *     ordered (same stream or event-ordered).
 *   - Images are W x H with 8 <= W, H and W, H <= 16384; all four images of a
 *     quad have the same size.  Rows of images are `pitch_bytes` apart,
 *     pixels are 3 interleaved uint8 channels (RGB).
 *   - Return value: SFF_OK (0) or a negative SFF_ERR_* code.  Argument errors
 *     are detected on the host before anything is enqueued.  SFF_ERR_CUDA
 *     reports a launch failure (cudaGetLastError()).
 */
#ifndef SFF_H
#define SFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFF_OK 0
#define SFF_ERR_ARG (-1)        /* invalid argument (null pointer, size, alignment, params) */
#define SFF_ERR_CUDA (-2)       /* a CUDA launch or API call failed */
#define SFF_ERR_WORKSPACE (-3)  /* workspace smaller than sff_workspace_bytes() */
#define SFF_ERR_TIMEOUT (-4)    /* a bounded device-side wait gave up (sff_device_status) */
#define SFF_ERR_CAPACITY (-5)   /* a seed buffer was too small (sff_device_status) */

#define SFF_FEATURES 48         /* int8 features per pixel and scale: 3 channels x 16 */
#define SFF_FEATURE_BYTES 48    /* bytes of one feature record */
#define SFF_PYRAMID_PIXEL_BYTES 52 /* pyramid bytes per pixel and scale: record + int32 norm */
#define SFF_MAX_SCALES 4
#define SFF_MAX_KNN 8
#define SFF_EMPTY_COST 2147483647 /* cost of a pixel that holds no vector yet */

/* Method parameters.  Defaults (sff_default_params) are the paper's values
 * (Sec. 5: k = 3 subscales, 12 iterations, tau_c = 1, s_c = 150) and the
 * readings of the points the paper leaves open. */
typedef struct sff_params {
    int32_t num_scales;   /* k + 1 scales, stride 2^s at scale s; 1..4 (Sec. 3.1, Sec. 5: k = 3) */
    int32_t iterations;   /* propagation + random-search iterations per scale; 0..64 (Sec. 5: 12) */
    int32_t tau_c;        /* consistency threshold in px; 0..255 (Sec. 3.1, Sec. 5: 1) */
    int32_t region_min;   /* minimum region size s_c; >= 0 (Sec. 3.1, Sec. 5: 150) */
    int32_t tau_r;        /* region rule: max-norm vector difference <= tau_r; 0..255 (default 1) */
    int32_t quant_shift;  /* feature quantisation: floor(coef / 2^quant_shift), 0..8 (default 4) */
    int32_t knn_temporal; /* K_T nearest neighbours of the temporal search; 1..8 (default 4) */
    int32_t knn_epipolar; /* K_E nearest neighbours per epipolar row; 1..8 (default 2) */
} sff_params;

/* Work distribution of the propagation kernels (no counterpart in the paper).
 * Every supported setting gives bit-identical results; only speed differs.
 * A variant of the iteration kernel is (lanes, slots, tile_x, tile_y, min_ctas):
 *   slots = 0: the throughput form, `lanes` in {1, 2, 4} threads sharing one
 *              pixel's feature loads, tile in {(64, 16), (32, 16), (64, 8),
 *              (32, 8), (16, 8), (8, 8)} grid pixels, min_ctas 0; and with one
 *              lane, (tile, min_ctas) in {(64 x 16, 2), (32 x 16, 3), (32 x 16,
 *              4), (32 x 8, 6), (32 x 8, 7), (32 x 8, 8), (16 x 8, 12)}:
 *              registers budgeted for that many resident CTAs per SM;
 *   slots = 1 or 4: the latency form (the next pixel's loads and the random
 *              draws issued up front, the colour-1 random search scored with
 *              the propagation candidates), each candidate of an update on
 *              `slots` == 4 ? its own `lanes` lanes : all lanes; only the
 *              tiles for which lanes * slots * (tile_x / 2 + 1) * (tile_y + 1)
 *              threads (one group per colour-0 slot of the tile and its halo)
 *              fit 1024; min_ctas 0.
 * Scale 0 takes (lanes_per_pixel, slots, tile_x, tile_y, min_ctas).  Scale
 * s >= 1 takes coarse[s - 1] = {lanes, slots, tile_x, tile_y, min_ctas}; all zero means
 * derived from the grid size: (1, 4, 16, 8, 0) below 200 grid pixels per SM
 * over all fields of the launch, else (1, 0, 32, 16, 0).
 * sff_tuning_supported() checks a setting. */
typedef struct sff_tuning {
    int32_t lanes_per_pixel; /* threads that share one pixel's feature loads */
    int32_t tile_x, tile_y;  /* grid pixels per CTA of the iteration kernel */
    int32_t slots;           /* 0: throughput form; 1 or 4: latency form */
    int32_t min_ctas;        /* throughput form compiled for >= this many resident CTAs per SM (0: none) */
    int32_t coarse[3][5];    /* scales 1..3: {lanes, slots, tile_x, tile_y, min_ctas}, or all 0 */
    int32_t group_mb;        /* sweep schedule of scale 0 when a launch holds several quads
                              * (sff_run_batch): 0 = every iteration launch covers all of them;
                              * > 0 = all iterations for one group of consecutive quads, then
                              * the next, each group's four-image records and field state at
                              * most group_mb MiB (a quad larger than that alone); 0..2^20 */
    int32_t pair_fields;     /* CTA order of the iteration kernel: 0 = field after field;
                              * 1 = a quad's forward and inverse field alternate tile by tile
                              * (their CTAs read the same four images side by side) */
    int32_t alternate_order; /* bit s set (s = 0..3): at scale s every other iteration launch
                              * visits its tiles last-to-first, so that it starts on what the
                              * previous launch read last (still in L2); 0..15 */
    int32_t features_form;   /* transform of the whole-stage calls (sff_run_batch): 0 = separable
                              * butterflies (sff_features), 1 = tensor cores (sff_features_tc),
                              * 2 = butterflies per pixel pair (sff_features_pairs); identical
                              * features */
    int32_t pdl;             /* bit s set (s = 0..3): the iteration launches of scale s use
                              * programmatic dependent launch: each is scheduled while the previous
                              * one's last CTAs run and waits in the kernel for its completion
                              * (same results); 0..15 */
    int32_t fuse;            /* bit s set (s = 1..3): all iterations of scale s run in one
                              * cooperative launch (every CTA resident, each taking tiles
                              * blockIdx.x + k * gridDim.x), a bounded grid barrier between
                              * iterations instead of a launch boundary (same results).  The
                              * scale's variant must have a fused form: a derived one (all-zero
                              * coarse entry) or (lanes, slots, tile_x x tile_y, min_ctas) one of
                              * (1,0,32x16,0), (1,0,32x16,4), (1,0,32x8,0), (1,0,32x8,7),
                              * (2,0,32x8,0), (1,1,32x16,0), (1,1,32x8,0), (1,1,16x8,0),
                              * (1,1,8x8,0), (2,1,32x8,0), (2,1,16x8,0), (2,1,8x8,0),
                              * (1,4,16x8,0), (1,4,8x8,0), (2,4,8x8,0); bit 0 clear, and no
                              * bit shared with pdl or alternate_order; 0..14.  A
                              * barrier wait that runs out (1 s) raises SFF_ERR_TIMEOUT in
                              * sff_device_status. */
    int32_t tma;             /* 1: at scale 0 each CTA of the iteration kernel stages its
                              * region's reference records in shared memory with one tensor
                              * copy (TMA) instead of per-thread loads (same results); the
                              * scale-0 variant must be (1, 0, 32x16 or 32x8) with min_ctas
                              * 0, or 32x16 with 3, or 32x8 with 7; 0 or 1 */
    int32_t overlap;         /* 1: in sff_run_batch, the features of the scales below the
                              * coarsest are computed on a second stream of the library (one
                              * per device and caller stream), forked once the coarsest grid
                              * is gathered, while the K-NN and the coarse scales match; each
                              * scale's inheritance waits for its features.  0: every launch
                              * on the caller's stream.  Same results; under stream capture
                              * the second stream forks from and joins back into the captured
                              * stream.  0 or 1 */
} sff_tuning;

/* One seed of Sec. 3.2: pixel (x, y) of L0, its vector and its scores. 20 bytes.
 * kind 0: a jointly consistent scene flow match.  kind 1 (only from
 * sff_emit_seeds_geo): a disparity-only seed of the disparity fill, with
 * u = v = d1 = 0 and cerr = |d0 - d_sgm|. */
typedef struct sff_seed {
    int16_t x, y, u, v, d0, d1;
    int32_t cost;   /* matching cost at scale 0 */
    uint8_t cerr;   /* consistency error: sum of |round-trip differences| */
    uint8_t kind;   /* 0 scene flow seed, 1 disparity-only seed */
    uint8_t pad[2];
} sff_seed;

/* Fills *out with the default parameters.  Returns SFF_ERR_ARG if out is NULL. */
int sff_default_params(sff_params* out);

/* Bytes of one image's feature pyramid: num_scales * H * W * 52.
 * Layout: per scale s, H * W 48-byte int8 feature records (16 coefficients
 * per channel, channel-major, in the order of sff_features): for scale 0 as
 * three planes of 16-byte chunks ([chunk][y][x], chunk = channel), for the
 * coarser scales as whole records ([y][x][48]); then
 * [scale][y][x] int32 norms (the sum of squared features of each record).
 * Returns 0 for invalid arguments. */
size_t sff_pyramid_bytes(int32_t width, int32_t height, const sff_params* params);

/* Device scratch needed by any call below for a W x H quad.  0 if invalid. */
size_t sff_workspace_bytes(int32_t width, int32_t height, const sff_params* params);

/* Walsh-Hadamard patch features of one image at every scale (Sec. 3.1,
 * "Initialization": WHT features as in FlowFields; "Multi-Scale
 * Propagation": scale s smooths the image and samples every n = 2^s-th
 * pixel, all positions staying at full resolution).
 *   Scale space: S_s = round-half-up mean of the n x n box with offsets
 *   -n/2..n/2-1 around each pixel, edges replicated; S_0 = image.
 *   Patch of pixel (x, y): P_c[i][j] = S_s(x + n(j-3), y + n(i-3))_c,
 *   i, j = 0..7, coordinates clamped to the image (boundary replication).
 *   Coefficients T_c = H P_c H^T with H the 8x8 Walsh matrix in sequency
 *   order; the 16 AC coefficients (ky, kx) with the lowest ky+kx (ties: lower
 *   ky) are kept per channel and quantised to clamp(floor(T / 2^quant_shift),
 *   -128, 127).
 * Computed separably: the 8-point Walsh transform of each row segment (an
 * image row at one patch's 8 sample columns) once, shared through shared
 * memory by the 8 pixels whose patches contain it, then per pixel the column
 * transforms of the kept coefficients only (integer sums, exact in any order).
 * rgb_dev: W x H x 3 uint8, rows pitch_bytes apart (pitch >= 3W).
 * pyramid_dev: sff_pyramid_bytes() bytes, 16-byte aligned; fully overwritten. */
int sff_features(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                 const sff_params* params, uint8_t* pyramid_dev,
                 void* workspace, size_t workspace_bytes, void* stream);

/* sff_features with the transform on the tensor cores: per scale and
 * channel, the kept coefficients of 128 pixels of a row as one matrix product
 * of their 8x8 patches (fp16, exact integers 0..255) with the 16 kept
 * Walsh-Hadamard basis products (+-1), accumulated in fp32 (exact: every
 * partial sum is an integer of magnitude <= 16320).  Same arguments, same
 * pyramid, bit for bit, as sff_features (Sec. 3.1, "Initialization").  Its
 * only device waits (for the MMAs of a tile) are bounded: a wait that gives
 * up leaves that image's records of the scale incomplete and raises
 * SFF_ERR_TIMEOUT in sff_device_status. */
int sff_features_tc(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                    const sff_params* params, uint8_t* pyramid_dev,
                    void* workspace, size_t workspace_bytes, void* stream);

/* sff_features with the transform per pair of vertically adjacent pixels
 * (x, y), (x, y + n): one thread computes the 9 row transforms of their two
 * patches and folds each into both pixels' kept coefficients.  The earlier
 * form, kept for comparison: same arguments, same pyramid, bit for bit, as
 * sff_features (Sec. 3.1, "Initialization"). */
int sff_features_pairs(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                       const sff_params* params, uint8_t* pyramid_dev,
                       void* workspace, size_t workspace_bytes, void* stream);

/* One dense scene-flow field (Sec. 3.1, "Initialization" and "Multi-Scale
 * Propagation"; "Consistency Check" for the inverse field).
 *   Cost of u at p (Eq. 1, with squared L2 distances of the WHT features of
 *   the pixel's patch in place of the summed Euclidean SIFTFlow distances):
 *   SSD(ref(p), temporal(p + (u, v))) + SSD(ref(p), stereo(p + (-sigma d0, 0)))
 *   + SSD(ref(p), cross(p + (u - sigma d1, v))), each position clamped to
 *   the image; sigma = +1 (mirror = 0) or -1 (mirror = 1).
 *   Forward field: ref = L0, temporal = L1, stereo = R0, cross = R1, mirror 0.
 *   Inverse field: ref = R1, temporal = R0, stereo = L1, cross = L0, mirror 1
 *   ("temporal order as well as points of view are swapped").
 *   Initialisation on the coarsest grid only: exact K_T nearest temporal
 *   grid points, K_E nearest stereo points on the pixel's row (d0 >= 0) and
 *   K_E nearest cross points on each temporal candidate's row (d1 >= 0); all
 *   combinations scored, lowest cost wins (ties: first combination).
 *   Then for each scale from coarse to fine: points of the coarser grid keep
 *   their vector (cost re-scored), the other grid points start empty; then
 *   `iterations` times: two synchronous half-steps over the two grid colours
 *   ((x + y) / n even first), each grid pixel taking the lowest-cost of its
 *   own vector and those of its two predecessors along the sweep direction
 *   (cycling (+x,+y), (-x,-y), (+x,-y), (-x,+y)), replaced only on strictly
 *   lower cost; then random search: every non-empty grid pixel adds to each
 *   component the rounded value of a uniform draw on ]-n, n[ (Philox4x32-10,
 *   key = seed, counter = (y W + x, iteration, scale + 4 mirror, 0)),
 *   clamps d0, d1 >= 0 and keeps the candidate if its cost is strictly lower.
 * pyr_*_dev: pyramids from sff_features of the same size and params.
 * field_dev: [H][W][4] int16 (u, v, d0, d1), 8-byte aligned; cost_dev: [H][W]
 * int32, SFF_EMPTY_COST where a pixel holds no vector.  Both overwritten. */
int sff_match_views(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                    const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev,
                    int32_t width, int32_t height, int32_t mirror, uint64_t seed,
                    const sff_params* params, int16_t* field_dev, int32_t* cost_dev,
                    void* workspace, size_t workspace_bytes, void* stream);

/* sff_match_views with the paper's own propagation order (Sec. 3.1,
 * "Multi-Scale Propagation": the pixels are visited in scan order, each
 * taking the better of its predecessors' current vectors, in place).  Each
 * iteration is one raster sweep over the grid in the iteration's direction
 * (rows in y direction, pixels in x direction), every pixel comparing first
 * its horizontal, then its vertical predecessor's vector as updated earlier
 * in the same sweep (replaced only on strictly lower cost), followed by the
 * random search of sff_match_views over every non-empty grid pixel.
 * Everything else (initialisation, inheritance, costs, random draws) is that
 * of sff_match_views.  A sweep has one dependent step per anti-diagonal of
 * the grid (W/n + H/n - 1 of them), so this call is much slower than
 * sff_match_views; it reproduces the sequential scan exactly.  Same
 * arguments, alignment, workspace and errors as sff_match_views. */
int sff_match_views_sequential(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                               const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev,
                               int32_t width, int32_t height, int32_t mirror, uint64_t seed,
                               const sff_params* params, int16_t* field_dev, int32_t* cost_dev,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Both fields of a quad in one pass (Sec. 3.1: the matching field of L0 and
 * the inverse field of R1 used by "Consistency Check").  Identical results to
 *   sff_match_views(L0, L1, R0, R1, mirror 0) -> fwd, fwd_cost
 *   sff_match_views(R1, R0, L1, L0, mirror 1) -> inv, inv_cost
 * with the same seed and params; the two fields share every kernel launch
 * (half the launches, one L2 fill of each scale's features for both).
 * pyr_*_dev: pyramids of L0, R0, L1, R1; outputs as in sff_match_views. */
int sff_match_quad(const uint8_t* pyr_l0_dev, const uint8_t* pyr_r0_dev,
                   const uint8_t* pyr_l1_dev, const uint8_t* pyr_r1_dev,
                   int32_t width, int32_t height, uint64_t seed, const sff_params* params,
                   int16_t* fwd_dev, int32_t* fwd_cost_dev, int16_t* inv_dev, int32_t* inv_cost_dev,
                   void* workspace, size_t workspace_bytes, void* stream);

/* sff_match_quad with an explicit work distribution (identical results). */
int sff_match_quad_tuned(const uint8_t* pyr_l0_dev, const uint8_t* pyr_r0_dev,
                         const uint8_t* pyr_l1_dev, const uint8_t* pyr_r1_dev,
                         int32_t width, int32_t height, uint64_t seed, const sff_params* params,
                         const sff_tuning* tuning,
                         int16_t* fwd_dev, int32_t* fwd_cost_dev, int16_t* inv_dev, int32_t* inv_cost_dev,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Fills *out with the default tuning; SFF_ERR_ARG if out is NULL. */
int sff_default_tuning(sff_tuning* out);

/* 1 if the tuning is one of the supported settings, else 0. */
int sff_tuning_supported(const sff_tuning* tuning);

/* Consistency check and region filter (Sec. 3.1, "Consistency Check").
 *   For L0 pixel p with forward vector u, q = p + (u - d1, v) in R1 and w the
 *   inverse vector at q: differences (w.u + u - d1 + d0, w.v + v, w.d0 - d1,
 *   w.d1 - d0); p is kept iff all |differences| <= tau_c; cerr = min(255,
 *   sum |differences|).  Pixels without a vector, with q outside the image
 *   or without an inverse vector at q are rejected with cerr = 255.
 *   Region filter: kept pixels form 4-connected regions where neighbours
 *   differ by at most tau_r in every component; a region that a rejected
 *   4-neighbour (with a vector) could join by the same rule and that has
 *   fewer than region_min pixels is removed.
 * keep_dev: [H][W] uint8 0/1; cerr_dev: [H][W] uint8.  Both overwritten. */
int sff_consistency_filter(const int16_t* fwd_dev, const int32_t* fwd_cost_dev,
                           const int16_t* inv_dev, const int32_t* inv_cost_dev,
                           int32_t width, int32_t height, const sff_params* params,
                           uint8_t* keep_dev, uint8_t* cerr_dev,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Sparsification (Sec. 3.2): for each non-overlapping 3x3 block (anchored at
 * (0, 0), partial blocks at the right/bottom edges included) the kept pixel
 * with the lowest cerr, then lowest cost, then lowest raster index becomes a
 * seed.  Seeds are written in block raster order.
 * seeds_dev: room for `capacity` seeds; seeds past `capacity` are dropped.
 * count_dev: device int32, receives the total number of seeds (which may
 * exceed capacity).  ceil(W/3) * ceil(H/3) is always enough. */
int sff_emit_seeds(const int16_t* fwd_dev, const int32_t* fwd_cost_dev,
                   const uint8_t* keep_dev, const uint8_t* cerr_dev,
                   int32_t width, int32_t height, sff_seed* seeds_dev, int32_t capacity,
                   int32_t* count_dev, void* workspace, size_t workspace_bytes, void* stream);

/* Disparity fill (Sec. 3.1, last paragraph): the joint filtering removes
 * more disparities than necessary, so a second disparity map of L0/R0 from
 * semi-global matching verifies the matching's own d0 where the joint check
 * failed.  The paper names SGM and the shared threshold tau_c only; this
 * library's SGM is:
 *   - grey = (R + 2G + B + 2) >> 2; census over a 9 x 7 window (bit k, in
 *     row-major window order without the centre, set when the neighbour is
 *     darker than the centre), coordinates clamped to the image;
 *   - cost C(p, d) = Hamming distance of the census words of L0 at (x, y)
 *     and R0 at (max(x - d, 0), y), 0 <= d < max_disp;
 *   - aggregation along the 4 axes and 4 diagonals:
 *     L_r(p, d) = C(p, d) + min(L_r(p - r, d), L_r(p - r, d +- 1) + p1,
 *                               min_k L_r(p - r, k) + p2) - min_k L_r(p - r, k);
 *   - disparity = argmin_d sum_r L_r(p, d), ties to the lowest d; no
 *     left-right check. */
typedef struct sff_sgm_params {
    int32_t max_disp;  /* disparity range D: 32, 64, 128 or 256 */
    int32_t p1, p2;    /* penalties, 0 <= p1 <= p2 <= 193 (L_r then fits 8 bits) */
} sff_sgm_params;

/* Defaults: max_disp 128, p1 10, p2 120.  SFF_ERR_ARG if out is NULL. */
int sff_default_sgm_params(sff_sgm_params* out);

/* Scratch of sff_sgm: two census words of 8 bytes, max_disp bytes of
 * matching costs and 8 * max_disp bytes of path costs per pixel; 0 for
 * invalid arguments. */
size_t sff_sgm_workspace_bytes(int32_t width, int32_t height, const sff_sgm_params* params);

/* SGM disparity map of left_dev (L0) against right_dev (R0), H x W x 3 uint8
 * images with row pitch `pitch_bytes` (>= 3 W), into disp_dev: [H][W] int16
 * (device, 2-byte aligned). */
int sff_sgm(const uint8_t* left_dev, const uint8_t* right_dev, int32_t pitch_bytes, int32_t width, int32_t height,
            const sff_sgm_params* params, int16_t* disp_dev, void* workspace, size_t workspace_bytes, void* stream);

/* Seeds with the disparity fill: as sff_emit_seeds, except that a 3x3 block
 * without a kept (jointly consistent) match takes, among its pixels that hold
 * a vector and whose d0 agrees with sgm_dev within params->tau_c, the one
 * with the lowest |d0 - d_sgm| (then cost, then raster index) as a
 * disparity-only seed (kind 1).  sgm_dev: [H][W] int16 (sff_sgm).  Workspace
 * as sff_emit_seeds (sff_workspace_bytes suffices). */
int sff_emit_seeds_geo(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const uint8_t* keep_dev,
                       const uint8_t* cerr_dev, const int16_t* sgm_dev, int32_t width, int32_t height,
                       const sff_params* params, sff_seed* seeds_dev, int32_t capacity, int32_t* count_dev,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free variant of sff_emit_seeds.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. code that only receives device pointers from another component and
 * has no allocator of its own, or a latency-critical loop where a
 * cudaMalloc (which may synchronise the device) is not acceptable.  It
 * computes exactly what sff_emit_seeds computes, with the same arguments
 * except the workspace: its scratch (one int32 per 3x3 block and one per
 * 256 blocks) is a static device array of SFF_NOALLOC_MAX_BLOCKS + 2048
 * int32 (about 2 MiB) inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   - Calls no cudaMalloc/cudaFree or allocating routine.
 *   - Images with ceil(W/3) * ceil(H/3) > SFF_NOALLOC_MAX_BLOCKS (about
 *     4.7 million pixels) are rejected with SFF_ERR_ARG before any work.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture on the device.  The cache is per device number and does
 *     not survive cudaDeviceReset (the module is loaded again, possibly at
 *     another address): do not call this entry point on a device after
 *     resetting it in the same process.
 *   - All calls share the one array: calls that may overlap on the GPU (other
 *     streams, other threads) race and must be ordered by the caller.  The
 *     array keeps the previous call's contents; every entry a call reads is
 *     first written by the same call. */
#define SFF_NOALLOC_MAX_BLOCKS (1 << 19)
int sff_emit_seeds_noalloc(const int16_t* fwd_dev, const int32_t* fwd_cost_dev,
                           const uint8_t* keep_dev, const uint8_t* cerr_dev,
                           int32_t width, int32_t height, sff_seed* seeds_dev, int32_t capacity,
                           int32_t* count_dev, void* stream);

/* The paper's own matching cost (Sec. 3.1 "Matching Cost", Eq. 1): the sum
 * over a 7 x 7 window (pixel stride n = 2^s at scale s) of the Euclidean
 * distances between the first three principal components phi of a dense
 * SIFT descriptor of the reference view and of each of the three other
 * views; the principal axes are computed over the descriptors of all four
 * images.  A float mode beside the WHT-SSD cost of sff_match_views.  This
 * library's dense SIFT (the paper relies on SIFTFlow's without restating
 * it): grey (R + 2G + B + 2) >> 2 of the scale's smoothed image; gradients
 * by central differences at stride n; 8 orientation sectors of 45 degrees
 * (exact integer tests); 4 x 4 cells of 3 x 3 samples at stride n; L2
 * normalisation, clipping at 0.2, renormalisation, quantisation to uint8
 * (x 512).  Axes: covariance of the four images' full-resolution descriptors
 * from exact integer sums, 200 power iterations per axis in double
 * precision, each dot product of an iteration as four partial sums over the
 * indices mod 4 (fused multiply-adds in index order) combined as
 * (s0 + s1) + (s2 + s3); the same axes at every scale.  Every floating-point
 * operation follows this fixed order, fused multiply-adds only there, so
 * results are reproducible bit for bit. */

/* Scratch of sff_sift_features: about 650 bytes per pixel; 0 for invalid sizes. */
size_t sff_sift_workspace_bytes(int32_t width, int32_t height);

/* phi of the four images at every scale.  rgb_dev4: host array of 4 device
 * pointers to H x W x 3 uint8 images with row pitch pitch_bytes; phi_dev4:
 * host array of 4 device pointers, each to [num_scales][H][W][4] float
 * (16-byte aligned; the fourth component is 0).  The principal axes are
 * computed over all four images, so their order does not matter. */
int sff_sift_features(const uint8_t* const* rgb_dev4, int32_t pitch_bytes, int32_t width, int32_t height,
                      const sff_params* params, float* const* phi_dev4, void* workspace, size_t workspace_bytes,
                      void* stream);

/* sff_match_views with the cost of Eq. 1 on phi (sff_sift_features) instead
 * of the WHT features.  The WHT pyramids still drive the initialisation's
 * nearest-neighbour search (Sec. 3.1 "Initialization"); all K_T x K_E x K_E
 * combinations are then scored with this cost, the first minimum in
 * (temporal, stereo, cross) rank order winning.  phi_*_dev: [S][H][W][4]
 * float of the views in the field's roles.  cost_dev receives each float
 * cost as its int32 bit pattern (non-negative floats order like their bit
 * patterns; SFF_EMPTY_COST stays the empty marker).  Workspace as
 * sff_match_views. */
int sff_match_views_sift(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                         const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev, const float* phi_ref_dev,
                         const float* phi_temporal_dev, const float* phi_stereo_dev, const float* phi_cross_dev,
                         int32_t width, int32_t height, int32_t mirror, uint64_t seed, const sff_params* params,
                         int16_t* field_dev, int32_t* cost_dev, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Dense interpolation of the seeds (Sec. 3.2, "Interpolation Models" and
 * "Edge-Aware Neighborhood"), with Euclidean pixel distances in place of the
 * geodesic ones (the edge map comes from a trained boundary detector, which
 * is not part of this library).
 *   - Every seed gets two local models, fitted by weighted least squares over
 *     its nearest seeds, weight exp(-alpha * D / dist_unit) for a neighbour D
 *     pixels away, ties in the distance order to the lower seed index:
 *       geometry: the plane d0 = a1 (x - xs) + a2 (y - ys) + a3 over the k_geo
 *       nearest seeds;
 *       motion: the affine map X1 = A (X0 - c) + t of 3D points over the
 *       k_motion nearest motion seeds (d0 >= 1 and d1 >= 1), X0 triangulated
 *       from (x, y, d0) and X1 from (x + u, y + v, d1) with the pinhole camera
 *       Z = focal * baseline / d, X = (x - cx) Z / focal, Y = (y - cy) Z / focal,
 *       c the weighted centroid of the X0.
 *     The linear parts get a ridge of 1e-9 * trace / dimension towards a flat
 *     plane and A = I (too few seeds: a constant disparity, a translation).
 *     Systems are solved by Cholesky factorisation in double precision.
 *   - Every pixel takes the models of its closest seed (same order) and
 *     evaluates them: d0 from the plane, then X0 from (x, y, max(d0, 1)),
 *     X1 = A (X0 - c) + t projected back gives u, v and d1.  Without motion
 *     neighbours, or when Z1 <= 0, u = v = 0 and d1 = d0.
 *   - No seeds: the field is all zeros. */
typedef struct sff_interp_params {
    int32_t k_geo, k_motion;   /* neighbourhood sizes, 1 ... 1024 */
    double alpha, dist_unit;   /* weight exp(-alpha * D / dist_unit) */
    double focal, baseline;    /* pixels; any unit of length */
    double cx, cy;             /* principal point, pixels */
} sff_interp_params;

/* Defaults: k_geo 160, k_motion 80, alpha 2.2, dist_unit 20 px, principal
 * point at the image centre ((W - 1) / 2, (H - 1) / 2).  SFF_ERR_ARG for a
 * NULL out, a size below 1 or a focal length or baseline that is not > 0. */
int sff_default_interp_params(int32_t width, int32_t height, double focal, double baseline,
                              sff_interp_params* out);

/* Scratch of sff_interpolate: 4 bytes per 3x3 block, 468 bytes per seed of
 * `capacity` (points, normal equations, models), 8 bytes per pixel and a
 * 512 KiB weight table; 0 for invalid arguments. */
size_t sff_interp_workspace_bytes(int32_t width, int32_t height, int32_t capacity);

/* Interpolates the seeds of sff_emit_seeds (seeds_dev, count_dev: device;
 * min(*count_dev, capacity) seeds are used) into field_dev: [H][W][4] float
 * (u, v, d0, d1), device, 16-byte aligned, overwritten.  params: host, read
 * during the call.  The seeds must lie in the image with at most one seed per
 * 3x3 block anchored at (0, 0), as sff_emit_seeds writes them.
 * Errors found on the GPU (a second seed in one block, a seed outside the
 * image, or more than 6 * max(k_geo, k_motion) + 224 neighbour candidates of
 * one seed tied at the k-th distances, which the candidate buffer's
 * compaction cannot reduce) set bits of a status word in the workspace (read
 * it with sff_interp_status) and the field is all zeros. */
int sff_interpolate(const sff_seed* seeds_dev, const int32_t* count_dev, int32_t capacity, int32_t width,
                    int32_t height, const sff_interp_params* params, float* field_dev, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Copies the status word of the last sff_interpolate on `workspace` into
 * *status_out (host) after a synchronous device-to-host copy (it waits for
 * the work on the legacy default stream): 0 = no error, bit 0 = a duplicate
 * or out-of-image seed, bit 1 = too many neighbour candidates. */
int sff_interp_status(const void* workspace, int32_t width, int32_t height, int32_t capacity, uint32_t* status_out);

/* One quad of a batch: its images, outputs and scratch (device pointers).
 * The four images share one pitch; seeds are written as by sff_emit_seeds. */
#define SFF_MAX_BATCH 32
typedef struct sff_quad {
    const uint8_t* rgb[4];     /* L0, R0, L1, R1: H x W x 3 uint8 */
    int32_t pitch_bytes;       /* row pitch of the four images (>= 3 W) */
    int32_t width, height;
    uint64_t seed;             /* random-search seed of this quad */
    uint8_t* pyramid[4];       /* sff_pyramid_bytes() each, 16-byte aligned */
    int16_t* fwd;              /* [H][W][4] forward field of L0 */
    int32_t* fwd_cost;
    int16_t* inv;              /* [H][W][4] inverse field of R1 */
    int32_t* inv_cost;
    uint8_t* keep;             /* [H][W] filter result */
    uint8_t* cerr;             /* [H][W] consistency error */
    sff_seed* seeds;           /* room for `capacity` seeds */
    int32_t capacity;
    int32_t* count;            /* device int32: number of seeds */
    void* workspace;           /* sff_quad_workspace_bytes(), 256-byte aligned */
    size_t workspace_bytes;
} sff_quad;

/* Scratch one quad of sff_run_batch needs; 0 for invalid arguments. */
size_t sff_quad_workspace_bytes(int32_t width, int32_t height, const sff_params* params);

/* The whole stage (Sec. 3.1-3.2: sff_features on the four images,
 * sff_match_quad, sff_consistency_filter, sff_emit_seeds) for n <= 32 quads
 * of any sizes, each phase in shared kernel launches.  Every quad's outputs
 * are identical to running those calls on it alone with its own seed.
 * `quads` is a host array read during the call; tuning NULL = default.
 * The enqueued work has no host synchronisation and can be captured into a
 * CUDA graph. */
int sff_run_batch(const sff_quad* quads, int32_t n, const sff_params* params, const sff_tuning* tuning,
                  void* stream);

/* Per-kernel timing (no counterpart in the paper: measurement support).
 * While enabled, every kernel launch of the library is bracketed by two
 * CUDA events recorded on the launch's stream.  Enabling or disabling
 * discards what was recorded.  Not usable while a stream is being captured
 * into a CUDA graph: keep it disabled around stream capture. */
typedef struct sff_kernel_time {
    char name[40];       /* kernel name */
    int32_t launches;    /* launches recorded */
    int32_t units;       /* work units they covered: iterations for the iteration kernel
                          * (a fused scale is one launch of all its iterations), else
                          * the launches */
    double total_ms;     /* summed event-to-event time */
} sff_kernel_time;

int sff_profile_enable(int32_t on);

/* Waits for the recorded events, writes up to `capacity` per-kernel totals
 * (first-launch order) and the number of distinct kernels to *n_out, then
 * clears the record.  Host pointers. */
int sff_profile_collect(sff_kernel_time* out, int32_t capacity, int32_t* n_out);

/* Number of device-side bounded waits (on the completion of the library's own
 * asynchronous copies and tensor-core operations) that gave up since the last
 * reset; nonzero means a result is invalid.  reset also clears the drain count
 * below.  Synchronises the current device.  Host pointer. */
int sff_device_timeouts(uint32_t* out, int32_t reset);

/* Of those, the drains that gave up: waits, after a failure, for copies and
 * MMAs already issued (which always complete) before the tensor memory is
 * released.  Each drain waits ten times the normal limit; a nonzero count
 * means the hardware did not finish issued work within it.  Host pointer. */
int sff_device_drain_timeouts(uint32_t* out);

/* Integer throughput of the current device, measured (no counterpart in the
 * paper; the roofline of the integer cost evaluations): kind 0 = dp4a (one
 * 4-way int8 dot product with int32 accumulate per op), kind 1 = 32-bit
 * integer multiply-add.  Eight independent chains per thread, 8 CTAs of 256
 * threads per SM, best of three timed launches (CUDA events on `stream`)
 * after a warm-up; *ops_per_s receives the operations per second.
 * Synchronises `stream`; allocates nothing.  SFF_ERR_ARG for another kind or
 * a NULL pointer. */
int sff_int_peak(int32_t kind, double* ops_per_s, void* stream);

/* Device-side error status, read at synchronisation (the calls themselves
 * only enqueue work and cannot see it).  Waits for the work enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream), then reports the
 * conditions that kernels of this library raised on the current device since
 * the last reset:
 *   SFF_ERR_TIMEOUT   a bounded device wait gave up (the temporal K-NN's
 *                     waits on its bulk copies and MMAs): the fields, and
 *                     everything computed from them, of the calls since the
 *                     last reset are invalid (their pixels may be empty,
 *                     never out of bounds);
 *   SFF_ERR_CAPACITY  otherwise, if sff_emit_seeds / sff_emit_seeds_geo /
 *                     sff_run_batch found more seeds than a seed buffer's
 *                     capacity: the first `capacity` seeds were written and
 *                     the count holds the number needed;
 *   SFF_OK            neither;  SFF_ERR_CUDA if the read or the
 *                     synchronisation failed.
 * reset != 0 clears both conditions after reading them.  The conditions are
 * per device and shared by all streams: a condition may come from another
 * stream's call that completed first.  Not for use while `stream` is being
 * captured into a CUDA graph (it synchronises). */
int sff_device_status(void* stream, int32_t reset);

/* Failure injection for tests of the device-side error path (no counterpart
 * in the paper).  step >= 0: in every later launch of the temporal K-NN
 * kernel the thread that issues the tensor-core MMAs stops before the MMAs of
 * that step (tile visit; 2 per candidate tile) and issues nothing further, so
 * the waits on that step's results run out; nothing issued is left in
 * flight.  step = -1: off.  wait_limit_us > 0 sets the time limit of every
 * bounded device wait (drains: ten times it); 0 restores the default of 1 s.
 * Applies to the current device; synchronous.  SFF_ERR_ARG for step < -1 or
 * wait_limit_us < 0. */
int sff_debug_knn_withhold(int32_t step, int32_t wait_limit_us);

/* Failure injection for the grid barrier of the fused iteration launches
 * (sff_tuning.fuse; no counterpart in the paper).  barrier >= 0: in every
 * later fused launch, CTA 0 leaves before arriving at that barrier (after
 * iteration `barrier`), so the other CTAs' bounded waits run out and raise
 * SFF_ERR_TIMEOUT; nothing is left in flight.  barrier = -1: off.
 * wait_limit_us as in sff_debug_knn_withhold (the same limit).  Applies to
 * the current device; synchronous.  SFF_ERR_ARG for barrier < -1 or
 * wait_limit_us < 0. */
int sff_debug_barrier_withhold(int32_t barrier, int32_t wait_limit_us);

/* Human-readable name of a status code (static string). */
const char* sff_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SFF_H */
