// Dense scene-flow fields: exact nearest-neighbour initialisation on the
// coarsest grid, then per scale inheritance + propagation half-steps with
// random search (Sec. 3.1, "Initialization", "Multi-Scale Propagation").
//
// Every kernel works on one or two fields at once (blockIdx.z): the forward
// field of L0 and the inverse field of R1 read the same four pyramids, so
// running them in the same launches halves the launch count, doubles the
// parallelism of the small coarse-scale launches and lets one L2 fill of a
// scale's features serve both fields.
//
// k_gather_grid:  writes the coarsest-grid points of the reference and
//                 temporal images as augmented bf16 rows whose products are
//                 the squared feature distances, in the tensor-core tile
//                 layout.
// k_knn_tc:       temporal K-NN, all-pairs over the coarsest grid: the
//                 distance matrix on the tensor cores (tcgen05.mma into
//                 tensor memory, operands streamed by TMA bulk copies),
//                 two scans of it -- a bound from 128 bucket minima, then
//                 exact top-8 lists under that bound.
// k_init_select:  one warp per query: takes the temporal top-K, finds
//                 the nearest epipolar stereo / cross points and keeps the
//                 best combination.  The cost is the sum of the three
//                 independent distances, so for a given temporal leaf the
//                 first-ranked epipolar leaves give the lowest cost and win
//                 every tie; the result equals scoring all K_T x K_E x K_E
//                 combinations in order.
// inheritance:    grid points of the coarser scale keep their vector and are
//                 re-scored at this scale; the others start empty.  Done by
//                 the first iteration of each finer scale (TileStep::inherit),
//                 or by k_inherit for the sequential sweeps and for runs
//                 without iterations.
// k_iteration:    one whole iteration (both colours of the checkerboard)
//                 over a tile, L lanes per pixel.  Fused with the random
//                 search: the search after iteration i of colour 1 runs at
//                 the end of its half-step of iteration i, the search of
//                 colour 0 at the start of its half-step of iteration i+1
//                 (or, after a scale's last iteration, in a third phase of
//                 that launch).  Both orders read the same values as the
//                 plain order "half-step 0, half-step 1, random search",
//                 because a half-step only reads the other colour and the
//                 search only reads the pixel itself.
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda.h>  // CUtensorMap and its encoder's signature (resolved at run time)

#include "sff_internal.cuh"
#include "sff_tc.cuh"

namespace sff {
namespace {

std::mutex g_fields_mu;  // guards the host staging of the Fields parameter


// One field: its views and grid at the current scale, its state and, for
// the double-buffered iteration kernel, the buffer it writes; plus its
// coarsest-scale K-NN scratch.
struct Field {
    Views V;
    uint2* field;  // state read (and written in place by the other kernels)
    int* cost;
    uint2* field_out;  // state written by k_iteration
    int* cost_out;
    int mirror;
    int gw, gh;  // grid of the current scale
    int gq;  // coarsest grid points
    int2* best8;  // [gq][8] temporal top-8 (distance, grid index)
    uint8_t* tk;  // [2 roles][rows] augmented bf16 rows in MMA tile layout: queries, candidates
    int4* rec;    // [2][gq][3] int8 records of the stereo and cross images' coarsest grid
    int* rec_n;   // [2][gq] their norms
    uint2 key;  // Philox key: the seed of the field's quad
    unsigned* sync;  // grid-barrier counter of a fused iteration launch (zeroed before each scale)
    uint8_t* stamp;  // change stamps of the current scale's grid (stamp_limits), one plane for all scales
};

// Up to kMaxFields fields of any sizes share every launch (blockIdx.z picks
// the field); passed by value as a __grid_constant__ kernel parameter.
constexpr int kMaxFields = kMaxBatchFields;
struct Fields {
    Field f[kMaxFields];
};

__device__ __forceinline__ const Field& pick(const Fields& F) { return F.f[blockIdx.z]; }




// ---------------------------------------------------------------------------
// Temporal K-NN on the tensor cores.
//
// The squared distance |q - c|^2 = |q|^2 + |c|^2 - 2 q.c of every
// (query, candidate) pair of the coarsest grid is one entry of a matrix
// product D = C Q^T with augmented rows
//     candidate c:  [ c_0..c_47,  P(|c|^2),  1, 1, 1,  0 ... ]
//     query q:      [ -2q_0..-2q_47,  1, 1, 1,  P(|q|^2),  0 ... ]
// where P(n) = (n & 0xff0000, n & 0xff00, n & 0xff) splits a norm
// (< 2^20) into three parts of at most 8 significant bits.  Every entry is
// an integer that bf16 holds exactly, every product and partial sum is an
// integer below 2^22 in magnitude, so the fp32 accumulation gives the exact
// distance whatever the order of its sums.  K = 54 is padded to 64.
//
// Operands sit in global memory already in the tcgen05 "no swizzle,
// K-major" shared-memory layout, 128 rows per 16 KB tile: core matrix
// (row group m, K group k) of 8 rows x 8 bf16 at byte
//     k * kTcKGroupStride + m * 128 + (row % 8) * 16 + (col % 8) * 2,
// so one bulk copy moves a tile.
constexpr int kTcRows = 128;                        // candidates per tile (M) = queries per CTA (N)
constexpr int kTcK = 64;                            // augmented row length (bf16)
constexpr int kTcTileBytes = kTcRows * kTcK * 2;    // 16 KB
constexpr int kTcKGroupStride = kTcRows * 16;       // bytes between K groups of 8 columns
constexpr int kTcStages = 6;                        // candidate tiles in shared memory
constexpr int kTcAcc = 4;                           // fp32 accumulators in tensor memory
constexpr int kTcScanWarps = 16;                    // warps reading the accumulators
constexpr int kTcScanCols = kTcRows * 4 / kTcScanWarps;  // query columns per scanning warp (32)
constexpr int kTcMmaWarp = kTcScanWarps;            // issues the MMAs
constexpr int kTcTmaWarp = kTcScanWarps + 1;        // issues the bulk copies
constexpr int kTcThreads = (kTcScanWarps + 2) * 32;
static_assert(kTcScanCols == 32, "one 32-column TMEM load per warp and step");
constexpr int kTcCols = kTcAcc * kTcRows;           // TMEM columns (all 512)
// instruction descriptor, kind::f16: fp32 D (bits 4-5 = 1), bf16 A (7-9 = 1)
// and B (10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcRows >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);
// shared memory: queries | candidate stages | scratch (bucket minima, then
// the per-lane-group candidate buffers) | limits | counts | barriers
constexpr int kTcOffQ = 0;
constexpr int kTcOffA = kTcOffQ + kTcTileBytes;
constexpr int kTcOffScratch = kTcOffA + kTcStages * kTcTileBytes;
constexpr int kTcMinStride = kTcRows + 1;                         // padded row: conflict-free both ways
constexpr int kTcScratchBytes = kTcRows * kTcMinStride * 4;      // [query][bucket] minima
constexpr int kTcCap = 16;                                       // buffered candidates per (lane group, query)
constexpr int kTcOffLim = kTcOffScratch + kTcScratchBytes;
constexpr int kTcOffCnt = kTcOffLim + 4 * kTcRows * 4;
constexpr int kTcOffBar = kTcOffCnt + 4 * kTcRows * 4;
constexpr int kTcSmemBytes = kTcOffBar + 256 + 1024;            // + alignment slack
static_assert(4 * kTcRows * kTcCap * 8 <= kTcScratchBytes, "candidate buffers fit the scratch");
constexpr unsigned kInfBits = 0x7f800000u;   // +inf
constexpr int kMaxFiniteBits = 0x7f7fffff;   // largest finite float

__host__ __device__ __forceinline__ int tc_rows(int gq) { return (gq + kTcRows - 1) / kTcRows * kTcRows; }

// Writes the augmented bf16 rows of the reference (role 0: queries) and
// temporal (role 1: candidates) coarsest-grid points; rows past gq are zero.
// One thread per 8-column group of a row.  Roles 2 and 3 copy the stereo
// and cross images' grid records into compact rows.
__global__ void k_gather_grid(const __grid_constant__ Fields F, int n) {
    const Field& A = pick(F);
    const int role = blockIdx.y;
    const int rows = tc_rows(A.gq);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (role >= 2) {
        // roles 2, 3: compact int8 records of the stereo and cross images
        // (row-major grid), scanned row by row by k_init_select
        const int c = t >> 2, part = t & 3;
        if (c >= A.gq) return;
        const Plane& P = role == 2 ? A.V.ste : A.V.crs;
        const size_t i = pix(A.V.w, (c % A.gw) * n, (c / A.gw) * n);
        const size_t slot = (size_t)(role - 2) * A.gq + c;
        if (part < 3)
            A.rec[slot * 3 + part] = chunk_of(P, i, part);
        else
            A.rec_n[slot] = __ldg(P.nrm + i);
        return;
    }
    const int r = t >> 3, kg = t & 7;
    if (r >= rows) return;
    float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (r < A.gq) {
        const Plane& P = role ? A.V.tmp : A.V.ref;
        const size_t i = pix(A.V.w, (r % A.gw) * n, (r / A.gw) * n);
        if (kg < 6) {
            const int2 f = __ldg(reinterpret_cast<const int2*>(chunk_ptr(P, i, kg >> 1)) + (kg & 1));
            const int8_t* b = reinterpret_cast<const int8_t*>(&f);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = role ? (float)b[k] : (float)(-2 * b[k]);
        } else if (kg == 6) {
            const int nr = __ldg(P.nrm + i);
            const float p2 = (float)(nr & 0xff0000), p1 = (float)(nr & 0xff00), p0 = (float)(nr & 0xff);
            const int norm_at = role ? 0 : 3;  // candidates: norm then ones; queries: ones then norm
            v[norm_at] = p2;
            v[norm_at + 1] = p1;
            v[norm_at + 2] = p0;
            v[3 - norm_at] = v[4 - norm_at] = v[5 - norm_at] = 1.f;
        }
    }
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint8_t* base = A.tk + (size_t)role * rows * (kTcK * 2);
    const size_t off = (size_t)(r / kTcRows) * kTcTileBytes + (size_t)kg * kTcKGroupStride + ((r % kTcRows) >> 3) * 128 +
                       (r & 7) * 16;
    *reinterpret_cast<uint4*>(base + off) = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ unsigned int g_wait_timeouts;  // bounded waits that gave up (read by sff_device_timeouts)
__device__ unsigned int g_drain_timeouts;  // drains that gave up (work in flight not seen to finish)
// Conditions raised since the last reset (read by sff_device_status):
// bit 0 a bounded wait gave up (the field of that call is invalid).
constexpr unsigned kStatusTimeout = 1u;
__device__ unsigned int g_match_status;
// Failure injection for tests (sff_debug_knn_withhold): the MMA issuer of
// k_knn_tc stops before the MMAs of this step (-1: never), and the limit of
// every bounded wait (0: kDefaultWaitNs).
__device__ int g_withhold_step = -1;
__device__ unsigned long long g_wait_limit_ns = 0;

__device__ __forceinline__ void note_timeout() {
    atomicAdd(&g_wait_timeouts, 1u);
    atomicOr(&g_match_status, kStatusTimeout);
}

// Reduces a buffer of `cnt` (<= kTcCap) candidates of one (lane group,
// query) to its 8 best in (distance, index) order, at the front in order;
// returns the limit they imply: the float bits just below the 8th distance
// (a candidate that comes later has a larger index, so it needs a strictly
// smaller distance).  The whole warp calls it.
__device__ __forceinline__ int tc_compact(int2* buf, int cnt, int lane) {
    const int2 x = lane < cnt ? buf[lane] : make_int2(0x7fffffff, 0x7fffffff);
    int rank = 0;
#pragma unroll
    for (int m = 0; m < kTcCap; ++m) {
        const int od = __shfl_sync(0xffffffffu, x.x, m), oi = __shfl_sync(0xffffffffu, x.y, m);
        rank += m < cnt && (od < x.x || (od == x.x && oi < x.y));
    }
    __syncwarp();
    if (lane < cnt && rank < 8) buf[rank] = x;
    const unsigned at7 = __ballot_sync(0xffffffffu, lane < cnt && rank == 7);
    const int d7 = __shfl_sync(0xffffffffu, x.x, at7 ? __ffs(at7) - 1 : 0);
    __syncwarp();
    return at7 ? __float_as_int((float)d7) - 1 : 0x7fffffff;
}

// Appends the lanes of `enter` (lane order = increasing candidate index) to
// a full-enough buffer, compacting it to its 8 best whenever it fills;
// every compaction lowers the limit, which drops the lanes no longer
// within it.  Rare: only when a column brings more candidates than the
// buffer holds (ties at the bound).
__device__ __noinline__ void tc_append_slow(unsigned enter, int mine, int idx, int cnt, int2* buf, int* cntp, int* limp,
                                            int lane) {
    const unsigned lt = (1u << lane) - 1u;
    while (enter) {
        const int room = kTcCap - cnt;
        const bool mine_in = (enter >> lane) & 1u;
        const int rank = __popc(enter & lt);
        if (mine_in && rank < room) buf[cnt + rank] = make_int2((int)__int_as_float(mine), idx);
        const int took = min(room, __popc(enter));
        enter = __ballot_sync(0xffffffffu, mine_in && rank >= room);
        cnt += took;
        __syncwarp();
        if (cnt == kTcCap) {
            const int nl = tc_compact(buf, cnt, lane);
            cnt = 8;
            const int l = min(*limp, nl);
            __syncwarp();
            if (lane == 0) *limp = l;
            enter &= __ballot_sync(0xffffffffu, mine <= l);
        }
    }
    __syncwarp();
    if (lane == 0) *cntp = cnt;
    __syncwarp();
}

// v[j] for a warp-uniform j in 0..31: a tree of selects on the bits of j
// (31 selects; a register array cannot be indexed at run time).
__device__ __forceinline__ uint32_t select32(const uint32_t (&v)[32], int j) {
    uint32_t a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (j & 1) ? v[2 * k + 1] : v[2 * k];
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        const bool hi = (j & (32 / (2 * w))) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) a[k] = hi ? a[2 * k + 1] : a[2 * k];
    }
    return a[0];
}

// Bounded wait on an accumulator for a whole warp (lane 0 polls); false
// (and the CTA's failure flag raised) on a timeout or when another warp
// already failed.
__device__ __forceinline__ bool scan_wait(uint64_t* bar, unsigned parity, volatile int* fail, int lane,
                                          unsigned long long wait_ns) {
    bool ok = true;
    if (lane == 0) ok = mbar_wait(bar, parity, wait_ns) && *fail == 0;
    const bool failed = __shfl_sync(0xffffffffu, (int)ok, 0) == 0;
    if (failed && lane == 0) {
        *fail = 1;
        note_timeout();
    }
    return !failed;
}

// Reads the warp's 32 candidates x 32 queries of accumulator b and releases it.
__device__ __forceinline__ void scan_load(uint32_t trow, int b, uint32_t (&v)[32], uint64_t* bar_free, int lane) {
    tc_fence_after();
    tmem_ld32(trow + (uint32_t)(b * kTcRows), v, 0);
    tmem_ld_wait(v);
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bar_free[b]);
}

// Temporal K-NN of the kTcRows queries of one CTA over every candidate of
// the field, exact in (distance, candidate index) order.
//
// Warp 17 streams candidate tiles into kTcStages shared-memory stages with
// bulk copies; warp 16 issues, per tile, four M128 N128 K16 MMAs into one of
// kTcAcc TMEM accumulators (rows = candidates, columns = queries) and
// commits them to the accumulator's and the stage's barriers.  Warps 0-15
// read an accumulator (warp w: lanes 32 (w % 4).., query columns
// 32 (w / 4)..), release it and scan it while the MMAs of the next tiles
// run.  Every tile is visited twice:
//   pass 1: each lane keeps, per query, the minimum over its candidates
//           ("bucket" = candidate index mod 128); the 8th smallest of the
//           128 bucket minima is reached by 8 distinct candidates, so it
//           bounds the query's 8th-nearest distance from above -- exactly
//           it, unless two of the 8 nearest share a bucket;
//   pass 2: candidates within the bound are appended to a buffer per lane
//           group and query (compacted to its 8 best if it fills, which
//           lowers the limit); the four buffers of a query are merged at
//           the end.
// Every wait is bounded; a timeout raises the CTA's failure flag, after
// which the warps skip their work but still reach every barrier, and the
// copy and MMA threads let their work in flight land before the tensor
// memory is released.
__global__ void __launch_bounds__(kTcThreads, 1) k_knn_tc(const __grid_constant__ Fields F) {
    extern __shared__ uint8_t smem_raw[];
    const Field& A = pick(F);
    const int gq = A.gq;
    const int q0 = blockIdx.x * kTcRows;
    if (q0 >= gq) return;  // CTA-uniform, before any barrier or allocation
    uint8_t* sm = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    uint8_t* sQ = sm + kTcOffQ;
    uint8_t* sA = sm + kTcOffA;
    int* scratch = reinterpret_cast<int*>(sm + kTcOffScratch);
    int* lim = reinterpret_cast<int*>(sm + kTcOffLim);  // [4 lane groups][kTcRows queries]
    int* count = reinterpret_cast<int*>(sm + kTcOffCnt);  // [4 lane groups][kTcRows queries]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kTcOffBar);
    uint64_t* bar_q = bars;
    uint64_t* bar_a = bars + 1;                                  // [kTcStages] tile landed
    uint64_t* bar_empty = bars + 1 + kTcStages;                  // [kTcStages] tile read by its MMAs
    uint64_t* bar_mma = bars + 1 + 2 * kTcStages;                // [kTcAcc] accumulator written
    uint64_t* bar_free = bars + 1 + 2 * kTcStages + kTcAcc;      // [kTcAcc] accumulator read
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 1 + 2 * kTcStages + 2 * kTcAcc);
    volatile int* fail = reinterpret_cast<volatile int*>(bars + 2 + 2 * kTcStages + 2 * kTcAcc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long wait_ns = g_wait_limit_ns ? g_wait_limit_ns : kDefaultWaitNs;
    const unsigned long long drain_ns = kDrainFactor * wait_ns;
    const int nt = (gq + kTcRows - 1) / kTcRows;  // candidate tiles
    const int steps = 2 * nt;                      // two passes
    const int rows = nt * kTcRows;
    const uint8_t* gQ = A.tk + (size_t)q0 * (kTcK * 2);
    const uint8_t* gC = A.tk + (size_t)rows * (kTcK * 2);

    if (threadIdx.x == 0) {
        mbar_init(bar_q, 1);
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&bar_a[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < kTcAcc; ++b) {
            mbar_init(&bar_mma[b], 1);
            mbar_init(&bar_free[b], kTcScanWarps);
        }
        *fail = 0;
        mbar_fence_init();
    }
    if (warp == kTcMmaWarp) tmem_alloc(tmem_slot, kTcCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kTcTmaWarp) {
        // ---- bulk copies (one thread): the queries once, then the
        // candidate tiles of both passes through the stages
        if (lane == 0) {
            mbar_expect_tx(bar_q, kTcTileBytes);
            bulk_copy_g2s(sQ, gQ, kTcTileBytes, bar_q);
            int issued = 0;
            bool ok = true;
            for (; issued < steps; ++issued) {
                const int u = issued, s = u % kTcStages;
                if (u >= kTcStages &&
                    (*fail ||
                     !(ok = mbar_wait(&bar_empty[s], (unsigned)((u - kTcStages) / kTcStages) & 1u, wait_ns))))
                    break;
                mbar_expect_tx(&bar_a[s], kTcTileBytes);
                bulk_copy_g2s(sA + s * kTcTileBytes, gC + (size_t)(u % nt) * kTcTileBytes, kTcTileBytes, &bar_a[s]);
            }
            if (!ok) {
                *fail = 1;
                note_timeout();
            }
            // drain: the copies in flight land before the CTA releases its
            // memory (issued copies always complete)
            bool drained = mbar_wait(bar_q, 0, drain_ns);
            for (int u = max(0, issued - kTcStages); u < issued; ++u)
                drained = mbar_wait(&bar_a[u % kTcStages], (unsigned)(u / kTcStages) & 1u, drain_ns) && drained;
            if (!drained) {
                atomicAdd(&g_drain_timeouts, 1u);
                note_timeout();
            }
        }
        __syncwarp();
    } else if (warp == kTcMmaWarp) {
        // ---- MMAs (one thread)
        if (lane == 0) {
            int committed = 0;
            const int withhold = g_withhold_step;
            bool ok = mbar_wait(bar_q, 0, wait_ns);
            const uint32_t qaddr = smem_addr(sQ);
            for (int u = 0; ok && u < steps; ++u) {
                if (*fail) {
                    ok = false;
                    break;
                }
                if (u == withhold) break;  // failure injection: nothing of this step is issued
                const int s = u % kTcStages, b = u % kTcAcc;
                if (!(ok = mbar_wait(&bar_a[s], (unsigned)(u / kTcStages) & 1u, wait_ns))) break;
                if (u >= kTcAcc && !(ok = mbar_wait(&bar_free[b], (unsigned)((u - kTcAcc) / kTcAcc) & 1u, wait_ns)))
                    break;
                tc_fence_after();
                const uint32_t aaddr = smem_addr(sA + s * kTcTileBytes);
#pragma unroll
                for (int kk = 0; kk < kTcK / 16; ++kk)
                    tc_mma(tmem + (uint32_t)(b * kTcRows), smem_desc(aaddr + kk * 2 * kTcKGroupStride, kTcKGroupStride, 128),
                           smem_desc(qaddr + kk * 2 * kTcKGroupStride, kTcKGroupStride, 128), kTcIdesc, kk > 0);
                tc_commit(&bar_mma[b]);
                tc_commit(&bar_empty[s]);
                committed = u + 1;
            }
            if (!ok) {
                *fail = 1;
                note_timeout();
            }
            // drain: the MMAs in flight finish before the tensor memory is
            // released (the last commit tracks every earlier MMA)
            if (committed > 0 &&
                !mbar_wait(&bar_mma[(committed - 1) % kTcAcc], (unsigned)((committed - 1) / kTcAcc) & 1u, drain_ns)) {
                atomicAdd(&g_drain_timeouts, 1u);
                note_timeout();
            }
        }
        __syncwarp();
    } else {
        // ---- scanners: warp w reads TMEM lanes 32 (w % 4).. (its candidates)
        // and query columns 32 (w / 4)..
        const int g = warp & 3, h = warp >> 2;
        const uint32_t trow = tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(kTcScanCols * h);
        const int qc = kTcScanCols * h;  // first query column of the warp
        int* mylim = lim + g * kTcRows + qc;
        int* mycnt = count + g * kTcRows + qc;
        int2* bufs = reinterpret_cast<int2*>(scratch);  // [4][kTcRows][kTcCap] in pass 2
        int2* mybuf = bufs + ((size_t)g * kTcRows + qc) * kTcCap;
        bool live = true;
        {
            // pass 1: bucket minima
            uint32_t mins[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) mins[j] = kInfBits;
            for (int u = 0; u < nt && live; ++u) {
                if (!(live = scan_wait(&bar_mma[u % kTcAcc], (unsigned)(u / kTcAcc) & 1u, fail, lane, wait_ns)))
                    break;
                uint32_t v[32];
                scan_load(trow, u % kTcAcc, v, bar_free, lane);
                if (u * kTcRows + 32 * g + lane < gq) {  // not a padding row of the last tile
#pragma unroll
                    for (int j = 0; j < 32; ++j) mins[j] = min(mins[j], v[j]);  // unsigned: a -0 never lowers a bound
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) scratch[(qc + j) * kTcMinStride + 32 * g + lane] = (int)mins[j];
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kTcScanWarps * 32) : "memory");
        {
            // bounds: four threads per query, each the 8 smallest of 32 bucket
            // minima (branch-free sorted insertion), then two merges; the 8th
            // smallest of the 128 is the inclusive bound
            const int q = threadIdx.x >> 2, part = threadIdx.x & 3;
            uint32_t a[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = 0xffffffffu;
            const int* row = scratch + q * kTcMinStride + 32 * part;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                uint32_t x = (uint32_t)row[i];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t lo = min(a[k], x);
                    x = max(a[k], x);
                    a[k] = lo;
                }
            }
#pragma unroll
            for (int o = 1; o <= 2; o <<= 1) {
                uint32_t b8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) b8[k] = __shfl_xor_sync(0xffffffffu, a[k], o);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint32_t x = b8[i];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t lo = min(a[k], x);
                        x = max(a[k], x);
                        a[k] = lo;
                    }
                }
            }
            // capped below +inf so that padding never enters
            lim[part * kTcRows + q] = (int)min(a[7], (uint32_t)kMaxFiniteBits);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kTcScanWarps * 32) : "memory");
        for (int e = threadIdx.x; e < 4 * kTcRows * kTcCap; e += kTcScanWarps * 32)
            bufs[e] = make_int2(0x7fffffff, 0x7fffffff);
        for (int e = threadIdx.x; e < 4 * kTcRows; e += kTcScanWarps * 32) count[e] = 0;
        asm volatile("bar.sync 1, %0;" ::"r"(kTcScanWarps * 32) : "memory");
        // pass 2: every candidate within its query's limit goes to the
        // buffer of (lane group, query), in increasing index order
        const unsigned lt = (1u << lane) - 1u;
        for (int u = nt; u < steps && live; ++u) {
            if (!(live = scan_wait(&bar_mma[u % kTcAcc], (unsigned)(u / kTcAcc) & 1u, fail, lane, wait_ns))) break;
            uint32_t v[32];
            scan_load(trow, u % kTcAcc, v, bar_free, lane);
            const int idx = (u - nt) * kTcRows + 32 * g + lane;
            unsigned m = 0;  // columns where this lane's candidate is within the limit
            if (idx < gq) {  // not a padding row of the last tile
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const int4 l4 = *reinterpret_cast<const int4*>(mylim + j);
                    m |= (unsigned)((int)v[j] <= l4.x) << j | (unsigned)((int)v[j + 1] <= l4.y) << (j + 1) |
                         (unsigned)((int)v[j + 2] <= l4.z) << (j + 2) | (unsigned)((int)v[j + 3] <= l4.w) << (j + 3);
                }
            }
            unsigned cols = __reduce_or_sync(0xffffffffu, m);
            while (cols) {
                const int j = __ffs(cols) - 1;
                cols &= cols - 1;
                const int mine = (int)select32(v, j);
                const unsigned ent = __ballot_sync(0xffffffffu, (m >> j) & 1u);
                const int c = mycnt[j];
                if (c + __popc(ent) <= kTcCap) {
                    if ((m >> j) & 1u) mybuf[j * kTcCap + c + __popc(ent & lt)] = make_int2((int)__int_as_float(mine), idx);
                    if (lane == 0) mycnt[j] = c + __popc(ent);
                } else {
                    tc_append_slow(ent, mine, idx, c, mybuf + j * kTcCap, mycnt + j, mylim + j, lane);
                }
            }
            __syncwarp();
        }
        // each buffer holding more than 8 candidates down to its 8 best
        for (int j = 0; j < kTcScanCols; ++j) {
            const int c = mycnt[j];
            if (c > 8) tc_compact(mybuf + j * kTcCap, c, lane);
        }
        // ---- merge the four lane-group buffers (8 best each, in any order)
        // of each query (warp w: kTcRows / kTcScanWarps queries)
        asm volatile("bar.sync 1, %0;" ::"r"(kTcScanWarps * 32) : "memory");
        for (int qq = 0; qq < kTcRows / kTcScanWarps; ++qq) {
            const int q = warp * (kTcRows / kTcScanWarps) + qq;
            if (q0 + q >= gq) break;
            if (!live) {
                // after a failed wait the lists are empty: the queries start
                // empty instead of reading stale candidate indices
                if (lane < 8) A.best8[(size_t)(q0 + q) * 8 + lane] = make_int2(0x7fffffff, 0x7fffffff);
                continue;
            }
            const int2 e = bufs[((size_t)(lane >> 3) * kTcRows + q) * kTcCap + (lane & 7)];
            int rank = 0;
#pragma unroll
            for (int o = 0; o < 32; ++o) {
                const int od = __shfl_sync(0xffffffffu, e.x, o), oi = __shfl_sync(0xffffffffu, e.y, o);
                rank += (od < e.x) || (od == e.x && (oi < e.y || (oi == e.y && o < lane)));
            }
            if (rank < 8) A.best8[(size_t)(q0 + q) * 8 + rank] = e;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kTcMmaWarp) tmem_dealloc(tmem, kTcCols);
}

// Nearest grid point of grid row gy by (distance, x), constrained by sigma,
// found by one warp over the compact row (records rec[gy * gw ..]): lane l
// scans grid columns l, l+32, ...; then a warp argmin.
__device__ __forceinline__ void warp_row_nearest(const RefFeat& r, const int4* rec, const int* rec_n, int n, int gw,
                                                 int gy, int xlim, int sigma, int lane, int& best_d, int& best_x) {
    int bd = 0x7fffffff, bx = 0x7fffffff;
    const int4* row = rec + (size_t)gy * gw * 3;
    const int* row_n = rec_n + (size_t)gy * gw;
    for (int g = lane; g < gw; g += 32) {
        const int x = g * n;
        if (sigma * (xlim - x) < 0) continue;
        const int4 q0 = __ldg(row + 3 * g), q1 = __ldg(row + 3 * g + 1), q2 = __ldg(row + 3 * g + 2);
        int dot = 0;
        dot = __dp4a(r.a[0], q0.x, dot); dot = __dp4a(r.a[1], q0.y, dot);
        dot = __dp4a(r.a[2], q0.z, dot); dot = __dp4a(r.a[3], q0.w, dot);
        dot = __dp4a(r.a[4], q1.x, dot); dot = __dp4a(r.a[5], q1.y, dot);
        dot = __dp4a(r.a[6], q1.z, dot); dot = __dp4a(r.a[7], q1.w, dot);
        dot = __dp4a(r.a[8], q2.x, dot); dot = __dp4a(r.a[9], q2.y, dot);
        dot = __dp4a(r.a[10], q2.z, dot); dot = __dp4a(r.a[11], q2.w, dot);
        const int d = r.n + __ldg(row_n + g) - 2 * dot;
        if (d < bd) {  // ascending x within the lane: ties keep the lower x
            bd = d;
            bx = x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int od = __shfl_xor_sync(0xffffffffu, bd, o), ox = __shfl_xor_sync(0xffffffffu, bx, o);
        if (od < bd || (od == bd && ox < bx)) {
            bd = od;
            bx = ox;
        }
    }
    best_d = bd;
    best_x = bx;
}

__global__ void k_init_select(const __grid_constant__ Fields F, int n, int knn) {
    const Field& A = pick(F);
    const Views& V = A.V;
    // the grid-barrier counters of every scale's fused iterations (one each)
    if (blockIdx.x == 0 && threadIdx.x < SFF_MAX_SCALES) A.sync[threadIdx.x] = 0u;
    const int gw = A.gw;
    const int qi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qi >= A.gq) return;  // warp-uniform
    const int px = (qi % gw) * n, py = (qi / gw) * n;
    RefFeat r;
    load_ref(V.ref, pix(V.w, px, py), r);
    // the query's temporal top-8 (every lane the same, reads broadcast), read
    // one entry at a time
    const int2* src = A.best8 + (size_t)qi * 8;
    int ds, sx;
    warp_row_nearest(r, A.rec, A.rec_n, n, gw, qi / gw, px, V.sigma, lane, ds, sx);
    int best_c = 0x7fffffff;
    Vec4 best = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k >= knn) break;
        const int2 e = src[k];
        const int bdk = e.x, bik = e.y;
        if (bdk == 0x7fffffff || bik < 0 || bik >= A.gq) break;
        const int tx = (bik % gw) * n, ty = (bik / gw) * n;
        int dxc, cx;
        warp_row_nearest(r, A.rec + (size_t)A.gq * 3, A.rec_n + A.gq, n, gw, bik / gw, tx, V.sigma, lane, dxc, cx);
        const int c = bdk + ds + dxc;
        if (c < best_c) {
            best_c = c;
            best.u = tx - px;
            best.v = ty - py;
            best.d0 = V.sigma * (px - sx);
            best.d1 = V.sigma * (tx - cx);
        }
    }
    if (lane == 0) {
        A.field[qi] = pack_vec(best);  // compact: grid row-major
        A.cost[qi] = best_c;
    }
}

__global__ void k_inherit(const __grid_constant__ Fields F, int n) {
    const Field& A = pick(F);
    const Views& V = A.V;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= A.gw || gy >= A.gh) return;
    const int x = gx * n, y = gy * n;
    const bool coarse = ((gx | gy) & 1) == 0;
    const size_t ic = (size_t)(gy >> 1) * ((A.gw + 1) >> 1) + (gx >> 1);  // coarser scale's compact state
    const size_t io = (size_t)gy * A.gw + gx;                              // this scale's
    const int c = coarse ? A.cost[ic] : kEmpty;
    if (c != kEmpty) {
        RefFeat r;
        load_ref(V.ref, pix(V.w, x, y), r);
        const uint2 w = A.field[ic];
        const Vec4 a = unpack_vec(w);
        A.field_out[io] = w;
        A.cost_out[io] = cost_of(V, r, x, y, a.u, a.v, a.d0, a.d1);
    } else {
        A.cost_out[io] = kEmpty;
        A.field_out[io] = make_uint2(0u, 0u);
    }
}


// Pixels are processed by groups of L lanes (L = 1, 2 or 4, a tuning knob
// that never changes results).  Lane q of a group holds the 16-byte chunks j
// of a 48-byte record with j % L == q; every target record is loaded the
// same way, so with L = 4 one warp-wide load fetches eight whole records.
// The norms are not loaded: each lane computes its chunks' part of |b|^2
// with dp4a (exact), which saves the norm plane's sector per record -- the
// iteration kernels are bound by L1 sector traffic, not by issue.  Partial
// sums |a|^2 + |b|^2 - 2 a.b of the three views are combined with log2(L)
// shuffles inside the group.
template <int L>
struct Slice {
    static constexpr int kChunks = (3 + L - 1) / L;
    int4 c[kChunks];
    int nrm;  // this lane's part of the record's squared norm
};

__device__ __forceinline__ int dot4(const int4& a, const int4& b, int d) {
    d = __dp4a(a.x, b.x, d);
    d = __dp4a(a.y, b.y, d);
    d = __dp4a(a.z, b.z, d);
    return __dp4a(a.w, b.w, d);
}

template <int L>
__device__ __forceinline__ void load_slice(const Plane& P, size_t i, int q, Slice<L>& s) {
    s.nrm = 0;
#pragma unroll
    for (int k = 0; k < Slice<L>::kChunks; ++k) {
        const int j = q + k * L;
        s.c[k] = j < 3 ? chunk_of(P, i, j) : make_int4(0, 0, 0, 0);
        s.nrm = dot4(s.c[k], s.c[k], s.nrm);
    }
}

template <int L>
__device__ __forceinline__ int slice_part(const Slice<L>& a, const Plane& P, size_t i, int q) {
    Slice<L> t;
    load_slice<L>(P, i, q, t);
    int d = 0;
#pragma unroll
    for (int k = 0; k < Slice<L>::kChunks; ++k) d = dot4(a.c[k], t.c[k], d);
    return a.nrm + t.nrm - 2 * d;
}

// This lane's part of the cost of vector c at (px, py).
template <int L>
__device__ __forceinline__ int group_part(const Views& V, const Slice<L>& a, int q, int px, int py, const Vec4& c) {
    const int tx = clampi(px + c.u, 0, V.w - 1);
    const int ty = clampi(py + c.v, 0, V.h - 1);
    const int sx = clampi(px - V.sigma * c.d0, 0, V.w - 1);
    const int cx = clampi(px + c.u - V.sigma * c.d1, 0, V.w - 1);
    return slice_part<L>(a, V.tmp, pix(V.w, tx, ty), q) + slice_part<L>(a, V.ste, pix(V.w, sx, py), q) +
           slice_part<L>(a, V.crs, pix(V.w, cx, ty), q);
}

template <int L>
__device__ __forceinline__ int group_sum(int part, unsigned gmask) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) part += __shfl_xor_sync(gmask, part, o);
    return part;
}

template <int L>
__device__ __forceinline__ unsigned group_mask() {
    return L == 1 ? (1u << (threadIdx.x & 31)) : (((1u << L) - 1u) << (threadIdx.x & 31 & ~(L - 1)));
}

// Random-search candidate of iteration `it` around `cur`; false when it
// equals `cur` (its cost could not be strictly lower).
__device__ __forceinline__ bool rs_candidate(int n, int s, uint2 key, int mirror, int it, uint32_t pixel,
                                             const Vec4& cur, Vec4& cand) {
    const uint4 rnd = philox4x32_10(make_uint4(pixel, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u), key);
    cand.u = (int)(int16_t)(cur.u + rs_offset(rnd.x, n));
    cand.v = (int)(int16_t)(cur.v + rs_offset(rnd.y, n));
    cand.d0 = (int)(int16_t)max(0, cur.d0 + rs_offset(rnd.z, n));
    cand.d1 = (int)(int16_t)max(0, cur.d1 + rs_offset(rnd.w, n));
    return !(cand.u == cur.u && cand.v == cur.v && cand.d0 == cur.d0 && cand.d1 == cur.d1);
}

__device__ __forceinline__ bool same_vec(const Vec4& a, const Vec4& b) {
    return a.u == b.u && a.v == b.v && a.d0 == b.d0 && a.d1 == b.d1;
}

// Change stamps: one byte per grid pixel of the scale (Field::stamp) saying
// when the pixel's state last changed within the scale:
//     0           not since the scale's first iteration began,
//     2 it + 1    a colour-0 pixel, in the first half-step of iteration it
//                 (its propagation, or the random search of iteration
//                 it - 1, which the kernels run at that point),
//     2 it + 2    a colour-1 pixel, in the second half-step of iteration it
//                 (its propagation or its random search).
// A candidate taken from a predecessor whose vector has not changed since
// this pixel last took a candidate from the same neighbour cannot be strictly
// lower than the pixel's cost: that vector's cost here was computed then (or
// equalled the pixel's own or the other predecessor's, which were), the
// pixel kept a cost no higher, and a pixel's cost never rises within a
// scale.  Such a stale candidate is not evaluated; the results are those of
// evaluating it.  The horizontal predecessor (the sweep's dx) was last
// consulted in iteration it - 2 (dx alternates), the vertical one in it - 1
// for even it and it - 3 for odd it (dy runs +, -, -, +).  A colour-0
// pixel of iteration i' read its predecessors' states as of the end of
// iteration i' - 1 (stamps <= 2 i'), a colour-1 pixel read its colour-0
// predecessors after their half-step of i' (stamps <= 2 i' + 1).  Iteration
// 0 of a scale writes every grid pixel's stamp; later ones write it only on
// a change.  The plane is not double-buffered: a stamp read while its owner
// rewrites it in the same iteration is either the old value or a newer,
// larger one, which only makes the test fail (the candidate is scored as
// usual); a pixel computed in another tile's halo reads its own stamp only
// to pass it on when unchanged, and then no tile rewrites it.
struct StampLimits {
    int h, v;  // largest stale stamp of the horizontal / vertical predecessor (-1: none)
};
__device__ __forceinline__ StampLimits stamp_limits(int it, int colour) {
    const int ih = it - 2, iv = (it & 1) ? it - 3 : it - 1;
    return StampLimits{ih >= 0 ? 2 * ih + colour : -1, iv >= 0 ? 2 * iv + colour : -1};
}
template <bool kCg>
__device__ __forceinline__ int ld_stamp(const uint8_t* p) {
    if constexpr (kCg) return __ldcg(p);
    else return *p;
}
template <bool kCg>
__device__ __forceinline__ void st_stamp(uint8_t* p, int v) {
    if constexpr (kCg) __stcg(p, (unsigned char)v);
    else *p = (uint8_t)v;
}

// One half-step of one pixel with own state (cur, c) and predecessor states
// (va, ca), (vb, cb) (ca/cb = kEmpty when absent).  The costs of the
// candidates that do not depend on each other -- the random-search candidate
// that precedes the propagation (colour 0) and the two predecessors -- are
// evaluated with all their loads in flight together; the
// strict-less-than comparisons then run in the order random search,
// horizontal, vertical, exactly as if evaluated one after the other.  The
// random search that follows the propagation (colour 1) depends on its
// result and comes last.  rs_before / rs_after < 0: no search.
// stale_a / stale_b: the predecessor's vector is one this pixel has already
// scored (change stamps, below), so it cannot be strictly lower either.
template <int L>
__device__ __forceinline__ bool update_pixel(const Views& V, const Slice<L>& a, int q, unsigned gmask, int n, int s,
                                             uint2 key, int mirror, int x, int y, uint32_t pixel, int rs_before,
                                             int rs_after, const Vec4& va, int ca, const Vec4& vb, int cb, Vec4& cur,
                                             int& c, bool stale_a = false, bool stale_b = false) {
    bool changed = false;
    Vec4 cr;
    const bool do_rs = rs_before >= 0 && c != kEmpty && rs_candidate(n, s, key, mirror, rs_before, pixel, cur, cr);
    // A predecessor holding the pixel's own vector, or the same vector as the
    // other predecessor, has exactly that candidate's cost and can never be
    // strictly lower: it is not evaluated (the result is unchanged).
    const bool own_valid = c != kEmpty;
    const bool do_a = ca != kEmpty && !stale_a && !(own_valid && same_vec(va, cur));
    const bool do_b = cb != kEmpty && !stale_b && !(own_valid && same_vec(vb, cur)) &&
                      !(ca != kEmpty && same_vec(vb, va));
    const int pr = do_rs ? group_part<L>(V, a, q, x, y, cr) : 0;
    const int pa = do_a ? group_part<L>(V, a, q, x, y, va) : 0;
    const int pb = do_b ? group_part<L>(V, a, q, x, y, vb) : 0;
    if (do_rs) {
        const int cc = group_sum<L>(pr, gmask);
        if (cc < c) {
            c = cc;
            cur = cr;
            changed = true;
        }
    }
    if (do_a) {
        const int cc = group_sum<L>(pa, gmask);
        if (cc < c) {
            c = cc;
            cur = va;
            changed = true;
        }
    }
    if (do_b) {
        const int cc = group_sum<L>(pb, gmask);
        if (cc < c) {
            c = cc;
            cur = vb;
            changed = true;
        }
    }
    if (rs_after >= 0 && c != kEmpty && rs_candidate(n, s, key, mirror, rs_after, pixel, cur, cr)) {
        const int cc = group_sum<L>(group_part<L>(V, a, q, x, y, cr), gmask);
        if (cc < c) {
            c = cc;
            cur = cr;
            changed = true;
        }
    }
    return changed;
}

// One whole iteration (both colours) over a TX x TY tile of grid pixels.
// Phase 1 updates the colour-0 pixels of the tile and of a one-pixel halo on
// the sides the colour-1 pixels read from (the predecessor sides of the
// sweep), keeping the results in shared memory; phase 2 updates the
// colour-1 pixels of the tile from them.  The state is read from `field` and
// written to `field_out` (double buffering), so a CTA never sees another
// CTA's writes of the same iteration; halo pixels are computed redundantly
// and only written by the CTA that owns them.  At scale 0 the records of
// the two colours share cache lines, so the second phase mostly hits L1.
// Threads of the iteration kernel: enough L-lane groups for one colour-0
// cell of the region (tile + halo) each, so that both phases finish in one
// round and no thread waits at the barrier for a second pixel of another;
// at most 1024 (larger settings take more rounds).
template <int L, int TX, int TY>
__host__ __device__ constexpr int iter_threads() {
    return ((L * (((TX + 1) * (TY + 1) + 1) / 2)) + 31) / 32 * 32 > 1024
               ? 1024
               : ((L * (((TX + 1) * (TY + 1) + 1) / 2)) + 31) / 32 * 32;
}

struct IterStep {
    int n, s, dx, dy, it;
    int last;  // the scale's last iteration: also the colour-0 search of this iteration (phase 3)
    int f0;    // first field of the launch
    int pair;  // 0: blockIdx.z picks field f0 + z; 1: fields f0 + 2z and f0 + 2z + 1 (one quad's
               // forward and inverse) alternate along blockIdx.x, so their CTAs of one tile
               // position run side by side
    int rev;   // the block indices taken in reverse: CTAs are issued in increasing linear
               // index, so a launch with rev = 1 visits the tiles last-to-first and first reads
               // what the previous launch read last (still in L2)
    int inherit;  // first iteration of a scale that inherits (TileStep::inherit)
};

// Block indices of this CTA in visiting order.
__device__ __forceinline__ int3 iter_block(const IterStep& H) {
    if (!H.rev) return make_int3((int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
    return make_int3((int)(gridDim.x - 1 - blockIdx.x), (int)(gridDim.y - 1 - blockIdx.y),
                     (int)(gridDim.z - 1 - blockIdx.z));
}
// Field and tile column of this CTA.
__device__ __forceinline__ int iter_field(const IterStep& H, int3 b) {
    return H.f0 + (H.pair ? 2 * b.z + (b.x & 1) : b.z);
}
__device__ __forceinline__ int iter_tile_x(const IterStep& H, int3 b) { return H.pair ? (b.x >> 1) : b.x; }

// State of one iteration of a tile: the buffers it reads and writes and the
// step's scale, sweep direction and iteration.
struct TileStep {
    const uint2* fin;
    const int* cin;
    uint2* fout;
    int* cout;
    int n, s, dx, dy, it, last;
    // 1: the first iteration of a scale below the coarsest, which also does
    // the scale inheritance: fin / cin hold the coarser scale's final state
    // (its compact grid), a grid pixel with both coordinates even starts
    // from its coarser counterpart's vector with that vector's cost at this
    // scale (empty if the counterpart is), and every other pixel starts
    // empty -- in particular the predecessors of a colour-0 pixel, which are
    // of colour 1
    int inherit;
    uint8_t* stamp;  // change stamps (stamp_limits); nullptr: every candidate is scored
};

// The inherited state of grid pixel (gx, gy) (TileStep::inherit): the
// coarser scale's state where both coordinates are even, else empty; the
// cost is still the coarser scale's (the caller evaluates it at this scale).
template <bool kCg>
__device__ __forceinline__ int inherited_state(const TileStep& T, int gx, int gy, int gw, uint2& w) {
    w = make_uint2(0u, 0u);
    if ((gx | gy) & 1) return kEmpty;
    const size_t ic = (size_t)(gy >> 1) * ((gw + 1) >> 1) + (gx >> 1);
    const int c = kCg ? __ldcg(T.cin + ic) : T.cin[ic];
    if (c != kEmpty) w = kCg ? __ldcg(T.fin + ic) : T.fin[ic];
    return c;
}

// State loads and stores of the latency form.  kCg: through L2 only
// (ld/st.global.cg), for a launch whose CTAs read in one iteration what other
// CTAs wrote in the previous one (the fused form): an L1 line kept from an
// earlier iteration could hold stale state.
template <bool kCg>
__device__ __forceinline__ int ld_cost(const int* p) {
    if constexpr (kCg) return __ldcg(p);
    else return *p;
}
template <bool kCg>
__device__ __forceinline__ uint2 ld_vec(const uint2* p) {
    if constexpr (kCg) return __ldcg(p);
    else return *p;
}
template <bool kCg>
__device__ __forceinline__ void st_state(const TileStep& T, size_t i, uint2 v, int c) {
    if constexpr (kCg) {
        __stcg(T.fout + i, v);
        __stcg(T.cout + i, c);
    } else {
        T.fout[i] = v;
        T.cout[i] = c;
    }
}

// One iteration of the throughput form over the tile at grid (tx0, ty0) of
// field A, with the shared-memory region s_vec / s_cost.  Every thread of
// the CTA calls it; it contains one __syncthreads.  kTma: the reference
// records of the region (tile + halo) come from s_ref, where a tensor copy
// completing on `bar` stages them as [chunk][region row][region column];
// each thread waits for it (bounded by wait_ns) before its first read.
template <int L, int TX, int TY, bool kCg, bool kTma = false>
__device__ __forceinline__ void iter_tile(const Field& A, const TileStep& T, int tx0, int ty0, uint2* s_vec,
                                          int* s_cost, uint8_t* s_stamp, const int4* s_ref = nullptr,
                                          uint64_t* bar = nullptr, unsigned long long wait_ns = 0) {
    constexpr int kRegX = TX + 1, kRegY = TY + 1;
    constexpr int kGroups = iter_threads<L, TX, TY>() / L;
    const Views& V = A.V;
    const int q = threadIdx.x & (L - 1);
    const unsigned gmask = group_mask<L>();
    const int grp = threadIdx.x / L;
    const int gw = A.gw, gh = A.gh;
    if (tx0 >= gw || ty0 >= gh) return;  // tile beyond this field's grid (whole CTA)
    const int rx0 = tx0 - (T.dx > 0 ? 1 : 0), ry0 = ty0 - (T.dy > 0 ? 1 : 0);  // region origin
    const int n = T.n;
    const bool stamps = T.stamp != nullptr, read_st = stamps && T.it >= 2;
    const StampLimits lim = stamp_limits(T.it, 0);  // colour 0; colour 1 is one higher
    bool staged = false;  // this thread has seen the tensor copy complete
    // reference record of image pixel i, region cell r
    auto ref_slice = [&](size_t i, int r, Slice<L>& a) {
        if constexpr (kTma) {
            if (!staged) {
                if (!mbar_wait(bar, 0, wait_ns)) note_timeout();
                staged = true;
            }
            a.nrm = 0;
#pragma unroll
            for (int k = 0; k < Slice<L>::kChunks; ++k) {
                const int j = q + k * L;
                a.c[k] = j < 3 ? s_ref[j * (kRegX * kRegY) + r] : make_int4(0, 0, 0, 0);
                a.nrm = dot4(a.c[k], a.c[k], a.nrm);
            }
        } else {
            load_slice<L>(V.ref, i, q, a);
        }
    };

    // phase 1: colour-0 pixels of the region (tile + halo)
    constexpr int kHalfRow = (kRegX + 1) / 2;
    for (int k = grp; k < kHalfRow * kRegY; k += kGroups) {
        const int ry = k / kHalfRow;
        const int rx = 2 * (k % kHalfRow) + ((rx0 + ry0 + ry) & 1);
        const int gx = rx0 + rx, gy = ry0 + ry;
        if (rx >= kRegX || gx < 0 || gx >= gw || gy < 0 || gy >= gh) continue;
        const int x = gx * n, y = gy * n;
        const size_t i = pix(V.w, x, y);            // image pixel: records, random stream
        const size_t si = (size_t)gy * gw + gx;      // compact state of the scale's grid
        const int ax = x - T.dx * n, by = y - T.dy * n;
        const bool has_a = ax >= 0 && ax < V.w, has_b = by >= 0 && by < V.h;
        const size_t ja = has_a ? si - T.dx : si, jb = has_b ? si - (size_t)(T.dy * gw) : si;
        int c, ca = kEmpty, cb = kEmpty;
        int so = 0, sa = 0, sb = 0;  // change stamps: own, predecessors
        uint2 wc, wa = make_uint2(0u, 0u), wb = make_uint2(0u, 0u);
        if (T.inherit) {
            c = inherited_state<kCg>(T, gx, gy, gw, wc);
        } else {
            c = ld_cost<kCg>(T.cin + si);
            wc = ld_vec<kCg>(T.fin + si);
            if (has_a) ca = ld_cost<kCg>(T.cin + ja);
            if (has_b) cb = ld_cost<kCg>(T.cin + jb);
            wa = ld_vec<kCg>(T.fin + ja);
            wb = ld_vec<kCg>(T.fin + jb);
            if (read_st) {
                so = ld_stamp<kCg>(T.stamp + si);
                sa = ld_stamp<kCg>(T.stamp + ja);
                sb = ld_stamp<kCg>(T.stamp + jb);
            }
        }
        Slice<L> a;
        ref_slice(i, ry * kRegX + rx, a);
        Vec4 cur = unpack_vec(wc);
        if (T.inherit && c != kEmpty) c = group_sum<L>(group_part<L>(V, a, q, x, y, cur), gmask);
        const bool changed =
            update_pixel<L>(V, a, q, gmask, n, T.s, A.key, A.mirror, x, y, (uint32_t)i, T.it - 1, -1, unpack_vec(wa),
                            ca, unpack_vec(wb), cb, cur, c, read_st && sa <= lim.h, read_st && sb <= lim.v);
        if (q == 0) {
            const uint2 wv = pack_vec(cur);
            const int st = changed ? 2 * T.it + 1 : so;
            s_vec[ry * kRegX + rx] = wv;
            s_cost[ry * kRegX + rx] = c;
            s_stamp[ry * kRegX + rx] = (uint8_t)st;
            if (gx >= tx0 && gx < tx0 + TX && gy >= ty0 && gy < ty0 + TY) {
                st_state<kCg>(T, si, wv, c);
                if (stamps && (changed || T.it == 0)) st_stamp<kCg>(T.stamp + si, st);
            }
        }
    }
    __syncthreads();

    // phase 2: colour-1 pixels of the tile
    constexpr int kTileHalfRow = TX / 2;
    for (int k = grp; k < kTileHalfRow * TY; k += kGroups) {
        const int ly = k / kTileHalfRow;
        const int gy = ty0 + ly;
        const int gx = tx0 + 2 * (k % kTileHalfRow) + ((tx0 + gy + 1) & 1);
        if (gx >= gw || gy >= gh) continue;
        const int x = gx * n, y = gy * n;
        const size_t i = pix(V.w, x, y);
        const size_t si = (size_t)gy * gw + gx;
        int c = kEmpty;  // a colour-1 pixel starts empty at an inheriting iteration
        Vec4 cur = {0, 0, 0, 0};
        if (!T.inherit) {
            c = ld_cost<kCg>(T.cin + si);
            cur = unpack_vec(ld_vec<kCg>(T.fin + si));
        }
        Slice<L> a;
        ref_slice(i, (gy - ry0) * kRegX + (gx - rx0), a);
        const int agx = gx - T.dx, bgy = gy - T.dy;  // predecessors (colour 0, in the region)
        int ca = kEmpty, cb = kEmpty, sa = 0, sb = 0;
        uint2 wa = make_uint2(0u, 0u), wb = make_uint2(0u, 0u);
        if (agx >= 0 && agx < gw) {
            const int r = (gy - ry0) * kRegX + (agx - rx0);
            ca = s_cost[r];
            wa = s_vec[r];
            sa = s_stamp[r];
        }
        if (bgy >= 0 && bgy < gh) {
            const int r = (bgy - ry0) * kRegX + (gx - rx0);
            cb = s_cost[r];
            wb = s_vec[r];
            sb = s_stamp[r];
        }
        const bool changed =
            update_pixel<L>(V, a, q, gmask, n, T.s, A.key, A.mirror, x, y, (uint32_t)i, -1, T.it, unpack_vec(wa), ca,
                            unpack_vec(wb), cb, cur, c, read_st && sa <= lim.h + 1, read_st && sb <= lim.v + 1);
        if (q == 0) {
            st_state<kCg>(T, si, pack_vec(cur), c);
            if (stamps && (changed || T.it == 0)) st_stamp<kCg>(T.stamp + si, changed ? 2 * T.it + 2 : 0);
        }
    }
    if (!T.last) return;

    // phase 3 (last iteration of the scale): the random search of this
    // iteration for the tile's colour-0 pixels, from their phase-1 results in
    // shared memory.  It reads only the pixel itself, so it may follow the
    // colour-1 half-step, which read the colour-0 values before the search.
    for (int k = grp; k < kTileHalfRow * TY; k += kGroups) {
        const int ly = k / kTileHalfRow;
        const int gy = ty0 + ly;
        const int gx = tx0 + 2 * (k % kTileHalfRow) + ((tx0 + gy) & 1);
        if (gx >= gw || gy >= gh) continue;
        const int r = (gy - ry0) * kRegX + (gx - rx0);
        int c = s_cost[r];
        if (c == kEmpty) continue;  // the whole group
        const int x = gx * n, y = gy * n;
        const size_t i = pix(V.w, x, y);
        Vec4 cur = unpack_vec(s_vec[r]);
        Slice<L> a;
        ref_slice(i, r, a);
        if (update_pixel<L>(V, a, q, gmask, n, T.s, A.key, A.mirror, x, y, (uint32_t)i, T.it, -1, cur, kEmpty, cur,
                            kEmpty, cur, c) &&
            q == 0)
            st_state<kCg>(T, (size_t)gy * gw + gx, pack_vec(cur), c);
    }
}

// MB > 0: compiled for at least MB resident CTAs per SM (a register budget
// of 64K / (MB x threads)), so that a launch of few CTAs per SM fits one wave.
template <int L, int TX, int TY, int MB>
__global__ void __launch_bounds__(iter_threads<L, TX, TY>(), MB) k_iteration(const __grid_constant__ Fields F,
                                                                              IterStep H) {
    __shared__ uint2 s_vec[(TX + 1) * (TY + 1)];
    __shared__ int s_cost[(TX + 1) * (TY + 1)];
    __shared__ uint8_t s_stamp[(TX + 1) * (TY + 1)];
    // programmatic dependent launch: wait for the previous launch (its state
    // and memory), then let the next one be scheduled; no-ops otherwise
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int3 blk = iter_block(H);
    const Field& A = F.f[iter_field(H, blk)];
    const TileStep T{A.field, A.cost, A.field_out, A.cost_out, H.n, H.s, H.dx, H.dy, H.it, H.last, H.inherit,
                     A.stamp};
    iter_tile<L, TX, TY, false>(A, T, iter_tile_x(H, blk) * TX, blk.y * TY, s_vec, s_cost, s_stamp);
}

// Tensor maps of the scale-0 reference records of every field of a launch:
// the three 16-byte chunk planes of an image as a 4D tensor {4 x u32, W, H, 3}.
struct RefMaps {
    CUtensorMap m[kMaxFields];
};

// Scale-0 throughput form with the reference records of the tile's region
// staged in shared memory by one tensor copy per CTA (TMA), issued before
// the state loads so that both are in flight together.  The candidates'
// records stay gathers: their addresses depend on the vectors, and the window
// they span is larger than the records read (the tile plus the spread of the
// vectors and the random search).
template <int L, int TX, int TY, int MB>
__global__ void __launch_bounds__(iter_threads<L, TX, TY>(), MB)
    k_iteration_tma(const __grid_constant__ Fields F, IterStep H, const __grid_constant__ RefMaps M) {
    __shared__ __align__(128) int4 s_ref[3 * (TX + 1) * (TY + 1)];
    __shared__ uint2 s_vec[(TX + 1) * (TY + 1)];
    __shared__ int s_cost[(TX + 1) * (TY + 1)];
    __shared__ uint8_t s_stamp[(TX + 1) * (TY + 1)];
    __shared__ __align__(8) uint64_t bar;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int3 blk = iter_block(H);
    const int f = iter_field(H, blk);
    const Field& A = F.f[f];
    const int tx0 = iter_tile_x(H, blk) * TX, ty0 = blk.y * TY;
    if (tx0 >= A.gw || ty0 >= A.gh) return;  // tile beyond this field's grid (whole CTA)
    const unsigned long long wait_ns = g_wait_limit_ns ? g_wait_limit_ns : kDefaultWaitNs;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        mbar_expect_tx(&bar, (unsigned)sizeof(s_ref));
        // box {4, TX + 1, TY + 1, 3} at the region origin; a negative origin
        // (the halo at the image border) reads zeros, never used
        tma_load_4d(s_ref, &M.m[f], 0, tx0 - (H.dx > 0 ? 1 : 0), ty0 - (H.dy > 0 ? 1 : 0), 0, &bar);
    }
    __syncthreads();
    const TileStep T{A.field, A.cost, A.field_out, A.cost_out, H.n, H.s, H.dx, H.dy, H.it, H.last, H.inherit,
                     A.stamp};
    iter_tile<L, TX, TY, false, true>(A, T, tx0, ty0, s_vec, s_cost, s_stamp, s_ref, &bar, wait_ns);
    // no CTA leaves with its copy in flight
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, kDrainFactor * wait_ns)) {
        atomicAdd(&g_drain_timeouts, 1u);
        note_timeout();
    }
}

// ---------------------------------------------------------------------------
// Latency-oriented form of the same iteration (identical results).  At the
// coarse scales an SM holds few grid pixels and a launch lasts about as long
// as one pixel's chain of dependent loads, so this form shortens the chain:
//   - the colour-1 pixel's own state and reference record are loaded at the
//     start, together with the colour-0 cell's, instead of after the barrier;
//   - the random draws, which depend only on pixel, iteration, scale and
//     field, are made while those loads are in flight;
//   - colour 1's random-search candidate around the pixel's own vector (the
//     candidate whenever propagation leaves the pixel unchanged) is scored
//     together with the two predecessors; with four slots so is the one
//     around the horizontal predecessor's vector.  Only when propagation took
//     a vector whose search candidate was not scored is it scored afterwards.
// The candidates of one update are spread over C slots of L lanes (C = 1:
// all lanes score all candidates; C = 4: slot k scores candidate k), and the
// comparisons always run in the plain kernel's order (random search before
// propagation for colour 0, horizontal before vertical, strict less-than).
// One region slot per L*C-lane group in each phase: a variant whose region
// needs more than 1024 threads does not exist.
struct RsOff {
    int u, v, d0, d1;
};

__device__ __forceinline__ RsOff rs_draw(int n, int s, uint2 key, int mirror, int it, uint32_t pixel) {
    const uint4 r = philox4x32_10(make_uint4(pixel, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u), key);
    return RsOff{rs_offset(r.x, n), rs_offset(r.y, n), rs_offset(r.z, n), rs_offset(r.w, n)};
}

// Random-search candidate around base vector b; false when it equals b.
__device__ __forceinline__ bool rs_from(const RsOff& o, const Vec4& b, Vec4& cand) {
    cand.u = (int)(int16_t)(b.u + o.u);
    cand.v = (int)(int16_t)(b.v + o.v);
    cand.d0 = (int)(int16_t)max(0, b.d0 + o.d0);
    cand.d1 = (int)(int16_t)max(0, b.d1 + o.d1);
    return !same_vec(cand, b);
}

// Costs of the candidates k < K with valid[k] (the others get 0), their loads
// in flight together.  Every lane of the group ends with every cost.
template <int L, int C, int K>
__device__ __forceinline__ void costs_of(const Views& V, const Slice<L>& a, int q, int slot, unsigned gmask, int x,
                                         int y, const Vec4 (&cand)[K], const bool (&valid)[K], int (&cc)[K]) {
    if constexpr (C == 1) {
        int p[K];
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = valid[k] ? group_part<L>(V, a, q, x, y, cand[k]) : 0;
#pragma unroll
        for (int k = 0; k < K; ++k) cc[k] = group_sum<L>(p[k], gmask);
    } else {
        static_assert(K <= C, "one candidate per slot");
        Vec4 mine = cand[0];
        bool ok = slot == 0 && valid[0];
#pragma unroll
        for (int k = 1; k < K; ++k)
            if (slot == k) {
                mine = cand[k];
                ok = valid[k];
            }
        const int p = group_sum<L>(ok ? group_part<L>(V, a, q, x, y, mine) : 0, gmask);
        const int base = (int)(threadIdx.x & 31) & ~(L * C - 1);
#pragma unroll
        for (int k = 0; k < K; ++k) cc[k] = __shfl_sync(gmask, p, base + k * L);
    }
}

// Threads of the latency form: one G-lane group per colour-0 slot of the
// region, (TX / 2 + 1) slots per region row (some of them beyond the row's
// end in rows of odd parity) times TY + 1 rows.
template <int G, int TX, int TY>
__host__ __device__ constexpr int lat_threads() {
    return (G * ((TX + 2) / 2) * (TY + 1) + 31) / 32 * 32;
}

template <int G, int TX, int TY>
__host__ __device__ constexpr bool lat_fits() {
    return lat_threads<G, TX, TY>() <= 1024;
}

// One iteration of the latency form over the tile at grid (tx0, ty0) of
// field A, with the shared-memory region s_vec / s_cost.  Every thread of
// the CTA calls it; it contains one __syncthreads.
template <int L, int C, int TX, int TY, bool kCg>
__device__ __forceinline__ void lat_tile(const Field& A, const TileStep& T, int tx0, int ty0, uint2* s_vec,
                                         int* s_cost, uint8_t* s_stamp) {
    constexpr int G = L * C;
    static_assert(G <= 16 && lat_fits<G, TX, TY>() && TX % 2 == 0, "one region slot per group");
    constexpr int kRegX = TX + 1, kRegY = TY + 1;
    constexpr int kHalfRow = (kRegX + 1) / 2, kTileHalfRow = TX / 2;
    const Views& V = A.V;
    const int g = threadIdx.x & (G - 1);
    const int q = g & (L - 1), slot = g / L;
    const unsigned gmask = group_mask<G>();
    const int grp = threadIdx.x / G;  // this group's cell in each phase
    const int gw = A.gw, gh = A.gh;
    if (tx0 >= gw || ty0 >= gh) return;  // tile beyond this field's grid (whole CTA)
    const int rx0 = tx0 - (T.dx > 0 ? 1 : 0), ry0 = ty0 - (T.dy > 0 ? 1 : 0);
    const int n = T.n;
    const bool stamps = T.stamp != nullptr, read_st = stamps && T.it >= 2;
    const StampLimits lim = stamp_limits(T.it, 0);  // colour 0; colour 1 is one higher

    // colour-1 pixel of the tile (phase 2): state, reference record, draw
    const int gy2 = ty0 + grp / kTileHalfRow;
    const int gx2 = tx0 + 2 * (grp % kTileHalfRow) + ((tx0 + gy2 + 1) & 1);
    const bool has2 = grp < kTileHalfRow * TY && gx2 < gw && gy2 < gh;
    int c2 = kEmpty;
    uint2 w2 = make_uint2(0u, 0u);
    Slice<L> a2;
    RsOff o2{0, 0, 0, 0};
    if (has2) {
        const size_t si = (size_t)gy2 * gw + gx2;
        const size_t i = pix(V.w, gx2 * n, gy2 * n);
        if (!T.inherit) {  // a colour-1 pixel starts empty at an inheriting iteration
            c2 = ld_cost<kCg>(T.cin + si);
            w2 = ld_vec<kCg>(T.fin + si);
        }
        load_slice<L>(V.ref, i, q, a2);
        o2 = rs_draw(n, T.s, A.key, A.mirror, T.it, (uint32_t)i);
    }

    // phase 1: this group's colour-0 cell of the region (tile + halo)
    {
        const int ry = grp / kHalfRow;
        const int rx = 2 * (grp % kHalfRow) + ((rx0 + ry0 + ry) & 1);
        const int gx = rx0 + rx, gy = ry0 + ry;
        if (ry < kRegY && rx < kRegX && gx >= 0 && gx < gw && gy >= 0 && gy < gh) {
            const int x = gx * n, y = gy * n;
            const size_t i = pix(V.w, x, y);
            const size_t si = (size_t)gy * gw + gx;
            const int ax = x - T.dx * n, by = y - T.dy * n;
            const bool has_a = ax >= 0 && ax < V.w, has_b = by >= 0 && by < V.h;
            const size_t ja = has_a ? si - T.dx : si, jb = has_b ? si - (size_t)(T.dy * gw) : si;
            int c, ca = kEmpty, cb = kEmpty;
            int so = 0, sa = 0, sb = 0;  // change stamps: own, predecessors
            uint2 wc, wa = make_uint2(0u, 0u), wb = make_uint2(0u, 0u);
            if (T.inherit) {
                c = inherited_state<kCg>(T, gx, gy, gw, wc);
            } else {
                c = ld_cost<kCg>(T.cin + si);
                wc = ld_vec<kCg>(T.fin + si);
                if (has_a) ca = ld_cost<kCg>(T.cin + ja);
                if (has_b) cb = ld_cost<kCg>(T.cin + jb);
                wa = ld_vec<kCg>(T.fin + ja);
                wb = ld_vec<kCg>(T.fin + jb);
                if (read_st) {
                    so = ld_stamp<kCg>(T.stamp + si);
                    sa = ld_stamp<kCg>(T.stamp + ja);
                    sb = ld_stamp<kCg>(T.stamp + jb);
                }
            }
            Slice<L> a;
            load_slice<L>(V.ref, i, q, a);
            const RsOff o = rs_draw(n, T.s, A.key, A.mirror, T.it - 1, (uint32_t)i);
            Vec4 cur = unpack_vec(wc);
            if (T.inherit && c != kEmpty) c = group_sum<L>(group_part<L>(V, a, q, x, y, cur), gmask);
            const Vec4 va = unpack_vec(wa), vb = unpack_vec(wb);
            const bool own_valid = c != kEmpty;
            Vec4 cr;
            const bool do_rs = T.it > 0 && own_valid && rs_from(o, cur, cr);
            const bool do_a = ca != kEmpty && !(read_st && sa <= lim.h) && !(own_valid && same_vec(va, cur));
            const bool do_b = cb != kEmpty && !(read_st && sb <= lim.v) && !(own_valid && same_vec(vb, cur)) &&
                              !(ca != kEmpty && same_vec(vb, va));
            const int c0 = c;
            const Vec4 cand[3] = {cr, va, vb};
            const bool valid[3] = {do_rs, do_a, do_b};
            int cc[3];
            costs_of<L, C, 3>(V, a, q, slot, gmask, x, y, cand, valid, cc);
            if (do_rs && cc[0] < c) {
                c = cc[0];
                cur = cr;
            }
            if (do_a && cc[1] < c) {
                c = cc[1];
                cur = va;
            }
            if (do_b && cc[2] < c) {
                c = cc[2];
                cur = vb;
            }
            if (g == 0) {
                const uint2 wv = pack_vec(cur);
                const bool changed = c != c0;  // an accepted candidate is strictly lower
                const int st = changed ? 2 * T.it + 1 : so;
                s_vec[ry * kRegX + rx] = wv;
                s_cost[ry * kRegX + rx] = c;
                s_stamp[ry * kRegX + rx] = (uint8_t)st;
                if (gx >= tx0 && gx < tx0 + TX && gy >= ty0 && gy < ty0 + TY) {
                    st_state<kCg>(T, si, wv, c);
                    if (stamps && (changed || T.it == 0)) st_stamp<kCg>(T.stamp + si, st);
                }
            }
        }
    }
    __syncthreads();

    // phase 2: the colour-1 pixel, propagation then random search
    if (has2) {
        const int x = gx2 * n, y = gy2 * n;
        int c = c2;
        Vec4 cur = unpack_vec(w2);
        const int agx = gx2 - T.dx, bgy = gy2 - T.dy;  // predecessors (colour 0, in the region)
        int ca = kEmpty, cb = kEmpty, sa = 0, sb = 0;
        uint2 wa = make_uint2(0u, 0u), wb = make_uint2(0u, 0u);
        if (agx >= 0 && agx < gw) {
            const int r = (gy2 - ry0) * kRegX + (agx - rx0);
            ca = s_cost[r];
            wa = s_vec[r];
            sa = s_stamp[r];
        }
        if (bgy >= 0 && bgy < gh) {
            const int r = (bgy - ry0) * kRegX + (gx2 - rx0);
            cb = s_cost[r];
            wb = s_vec[r];
            sb = s_stamp[r];
        }
        const Vec4 va = unpack_vec(wa), vb = unpack_vec(wb);
        const bool own_valid = c != kEmpty;
        const int c0 = c;
        const bool do_a = ca != kEmpty && !(read_st && sa <= lim.h + 1) && !(own_valid && same_vec(va, cur));
        const bool do_b = cb != kEmpty && !(read_st && sb <= lim.v + 1) && !(own_valid && same_vec(vb, cur)) &&
                          !(ca != kEmpty && same_vec(vb, va));
        Vec4 r0, r1 = cur;
        const bool do_r0 = own_valid && rs_from(o2, cur, r0);
        bool do_r1 = false;
        if constexpr (C == 4) do_r1 = do_a && rs_from(o2, va, r1);
        constexpr int K = C == 4 ? 4 : 3;
        Vec4 cand[K];
        bool valid[K];
        cand[0] = va;
        cand[1] = vb;
        cand[2] = r0;
        valid[0] = do_a;
        valid[1] = do_b;
        valid[2] = do_r0;
        if constexpr (K == 4) {
            cand[3] = r1;
            valid[3] = do_r1;
        }
        int cc[K];
        costs_of<L, C, K>(V, a2, q, slot, gmask, x, y, cand, valid, cc);
        int base = 0;  // 0: own vector kept, 1: horizontal, 2: vertical predecessor taken
        if (do_a && cc[0] < c) {
            c = cc[0];
            cur = va;
            base = 1;
        }
        if (do_b && cc[1] < c) {
            c = cc[1];
            cur = vb;
            base = 2;
        }
        if (c != kEmpty) {
            Vec4 cr;
            int crc = 0;
            bool have;
            if (base == 0) {
                have = do_r0;
                cr = r0;
                crc = cc[2];
            } else if (K == 4 && base == 1) {
                have = do_r1;
                cr = r1;
                crc = cc[K - 1];
            } else {
                have = rs_from(o2, cur, cr);
                if (have) crc = group_sum<L>(group_part<L>(V, a2, q, x, y, cr), gmask);
            }
            if (have && crc < c) {
                c = crc;
                cur = cr;
            }
        }
        if (g == 0) {
            st_state<kCg>(T, (size_t)gy2 * gw + gx2, pack_vec(cur), c);
            if (stamps && (c != c0 || T.it == 0))
                st_stamp<kCg>(T.stamp + (size_t)gy2 * gw + gx2, c != c0 ? 2 * T.it + 2 : 0);
        }
    }
    if (!T.last) return;

    // phase 3 (last iteration of the scale): the random search of this
    // iteration for the tile's colour-0 pixels, from their phase-1 results
    {
        const int gy = ty0 + grp / kTileHalfRow;
        const int gx = tx0 + 2 * (grp % kTileHalfRow) + ((tx0 + gy) & 1);
        if (grp >= kTileHalfRow * TY || gx >= gw || gy >= gh) return;
        const int r = (gy - ry0) * kRegX + (gx - rx0);
        const int c = s_cost[r];
        if (c == kEmpty) return;  // the whole group
        const int x = gx * n, y = gy * n;
        const size_t i = pix(V.w, x, y);
        const Vec4 cur = unpack_vec(s_vec[r]);
        const RsOff o = rs_draw(n, T.s, A.key, A.mirror, T.it, (uint32_t)i);
        Vec4 cr;
        if (!rs_from(o, cur, cr)) return;
        Slice<L> a;
        load_slice<L>(V.ref, i, q, a);
        const int cc = group_sum<L>(group_part<L>(V, a, q, x, y, cr), gmask);
        if (cc < c && g == 0) st_state<kCg>(T, (size_t)gy * gw + gx, pack_vec(cr), cc);
    }
}

template <int L, int C, int TX, int TY>
__global__ void __launch_bounds__(lat_threads<L * C, TX, TY>()) k_iteration_lat(const __grid_constant__ Fields F,
                                                                                 IterStep H) {
    __shared__ uint2 s_vec[(TX + 1) * (TY + 1)];
    __shared__ int s_cost[(TX + 1) * (TY + 1)];
    __shared__ uint8_t s_stamp[(TX + 1) * (TY + 1)];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int3 blk = iter_block(H);
    const Field& A = F.f[iter_field(H, blk)];
    const TileStep T{A.field, A.cost, A.field_out, A.cost_out, H.n, H.s, H.dx, H.dy, H.it, H.last, H.inherit,
                     A.stamp};
    lat_tile<L, C, TX, TY, false>(A, T, iter_tile_x(H, blk) * TX, blk.y * TY, s_vec, s_cost, s_stamp);
}

// ---------------------------------------------------------------------------
// Fused form of a coarse scale: all iterations of the scale in one
// cooperative launch (every CTA resident), a grid barrier between
// iterations instead of a launch boundary.  Each CTA takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... of every field in turn and runs
// the latency form's iteration on each; iteration `it` reads the buffers
// (field, cost) when even and (field_out, cost_out) when odd and writes the
// other pair, exactly as the separate launches do, so the results are the
// same.  At a coarse scale an SM holds a few hundred grid pixels and a
// launch lasts a few microseconds, about as long as the gap between two
// dependent launches that the barrier replaces.
struct FusedStep {
    int n, s, iters;
    int f0, nf;              // fields f0 .. f0 + nf - 1
    int tiles_x, tiles_y;    // tile grid of the largest field
    unsigned* sync;          // barrier counter, zero at launch
    int inherit;             // iteration 0 also inherits (TileStep::inherit)
};

// Failure injection for tests (sff_debug_barrier_withhold): CTA 0 of a fused
// launch leaves before arriving at this barrier (-1: never), so that the
// other CTAs' bounded waits run out.
__device__ int g_withhold_barrier = -1;

// Grid barrier number b (0, 1, ...) of a cooperative launch: the counter
// reaches (b + 1) * gridDim.x when every CTA has arrived.  Thread 0 arrives
// with a release reduction (after the CTA barrier, so the release covers
// the whole CTA's stores) and polls with acquire loads, which order the
// CTA's later loads after the other CTAs' stores; it gives up after
// limit_ns.  Measured on GB300: about 1.25 us per barrier at 120-150 CTAs,
// 1.8 us at 456, 3.4 us at 1064 (a fence after the poll added 0.3 us).
// Every thread of the CTA calls it; false when the wait gave up (the caller
// leaves).
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, int b, unsigned long long limit_ns) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned target = (unsigned)(b + 1) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
        const unsigned long long t0 = global_ns();
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (global_ns() - t0 > limit_ns) {
                ok = 0;
                break;
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

// Threads and resident CTAs per SM of a fused variant: C = 0 is the
// throughput form, C > 0 the latency form with C slots.  MB > 0 is the
// throughput form's register budget for MB resident CTAs; otherwise the
// budget is about 100 registers a thread (without one, the loop over
// iterations and tiles takes about 130 and the larger CTAs fit once per SM;
// at 80 every latency variant spills).
template <int L, int C, int TX, int TY>
__host__ __device__ constexpr int fused_threads() {
    return C == 0 ? iter_threads<L, TX, TY>() : lat_threads<L * C, TX, TY>();
}
template <int L, int C, int TX, int TY, int MB>
__host__ __device__ constexpr int fused_min_blocks() {
    return MB > 0 ? MB
                  : (65536 / (fused_threads<L, C, TX, TY>() * 100) > 1 ? 65536 / (fused_threads<L, C, TX, TY>() * 100)
                                                                        : 1);
}

template <int L, int C, int TX, int TY, int MB>
__global__ void __launch_bounds__(fused_threads<L, C, TX, TY>(), fused_min_blocks<L, C, TX, TY, MB>())
    k_iteration_fused(const __grid_constant__ Fields F, FusedStep H) {
    __shared__ uint2 s_vec[(TX + 1) * (TY + 1)];
    __shared__ int s_cost[(TX + 1) * (TY + 1)];
    __shared__ uint8_t s_stamp[(TX + 1) * (TY + 1)];
    const unsigned long long wait_ns = g_wait_limit_ns ? g_wait_limit_ns : kDefaultWaitNs;
    const int withhold = g_withhold_barrier;
    const int per = H.tiles_x * H.tiles_y, total = per * H.nf;
    for (int it = 0; it < H.iters; ++it) {
        // sweep directions of iteration it: (1,1), (-1,-1), (1,-1), (-1,1), ...
        const int m = it & 3;
        const int dx = (m == 0 || m == 2) ? 1 : -1, dy = (m == 0 || m == 3) ? 1 : -1;
        const bool odd = (it & 1) != 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const Field& A = F.f[H.f0 + t / per];
            const int r = t % per;
            const TileStep T{odd ? A.field_out : A.field, odd ? A.cost_out : A.cost, odd ? A.field : A.field_out,
                             odd ? A.cost : A.cost_out, H.n, H.s, dx, dy, it, it == H.iters - 1,
                             it == 0 ? H.inherit : 0, A.stamp};
            if constexpr (C == 0)
                iter_tile<L, TX, TY, true>(A, T, (r % H.tiles_x) * TX, (r / H.tiles_x) * TY, s_vec, s_cost,
                                           s_stamp);
            else
                lat_tile<L, C, TX, TY, true>(A, T, (r % H.tiles_x) * TX, (r / H.tiles_x) * TY, s_vec, s_cost,
                                             s_stamp);
            __syncthreads();  // the region arrays are reused by the next tile
        }
        if (it + 1 == H.iters) break;
        if (withhold == it && blockIdx.x == 0) return;  // injected: never arrives
        if (!grid_barrier(H.sync, it, wait_ns)) {
            if (threadIdx.x == 0) note_timeout();
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// The paper's own propagation order (departure D4 switched back): each
// iteration is one in-place raster sweep in the iteration's direction, a
// pixel taking its two predecessors' current vectors (horizontal first,
// replaced only on strictly lower cost), then the random search over every
// non-empty grid pixel.  In sweep coordinates (a, b) a pixel depends on
// (a - 1, b) and (a, b - 1) only, so the pixels of one anti-diagonal
// a + b = t are independent: one CTA per field walks the gw + gh - 1
// diagonals, a barrier between them.  The critical path is that many
// dependent cost evaluations per iteration, so this order is an order of
// magnitude slower per quad than the checkerboard; it exists to reproduce
// the sequential scan exactly.
constexpr int kSweepLanes = 2;
constexpr int kSweepThreads = 1024;

__global__ void __launch_bounds__(kSweepThreads) k_sweep(const __grid_constant__ Fields F, int n, int dx, int dy) {
    constexpr int L = kSweepLanes;
    constexpr int kGroups = kSweepThreads / L;
    const Field& A = pick(F);
    const Views& V = A.V;
    const int q = threadIdx.x & (L - 1);
    const unsigned gmask = group_mask<L>();
    const int grp = threadIdx.x / L;
    const int gw = A.gw, gh = A.gh;
    for (int t = 0; t < gw + gh - 1; ++t) {
        const int b0 = max(0, t - (gw - 1)), b1 = min(gh - 1, t);
        for (int b = b0 + grp; b <= b1; b += kGroups) {
            const int a = t - b;
            const int gx = dx > 0 ? a : gw - 1 - a, gy = dy > 0 ? b : gh - 1 - b;
            const int x = gx * n, y = gy * n;
            const size_t si = (size_t)gy * gw + gx;
            const bool has_a = gx - dx >= 0 && gx - dx < gw, has_b = gy - dy >= 0 && gy - dy < gh;
            // plain loads: the predecessors were written by this CTA on the
            // previous diagonal
            int c = A.cost[si];
            Vec4 cur = unpack_vec(A.field[si]);
            const int ca = has_a ? A.cost[si - dx] : kEmpty;
            const int cb = has_b ? A.cost[si - (size_t)(dy * gw)] : kEmpty;
            const uint2 wa = has_a ? A.field[si - dx] : make_uint2(0u, 0u);
            const uint2 wb = has_b ? A.field[si - (size_t)(dy * gw)] : make_uint2(0u, 0u);
            Slice<L> r;
            load_slice<L>(V.ref, pix(V.w, x, y), q, r);
            if (update_pixel<L>(V, r, q, gmask, n, 0, A.key, A.mirror, x, y, 0u, -1, -1, unpack_vec(wa), ca,
                                unpack_vec(wb), cb, cur, c) &&
                q == 0) {
                A.field[si] = pack_vec(cur);
                A.cost[si] = c;
            }
        }
        __syncthreads();
    }
}

// The random search of iteration `it` over every non-empty grid pixel, in
// place (it reads only the pixel itself).  L = 4 lanes per pixel.
__global__ void __launch_bounds__(256) k_random_search(const __grid_constant__ Fields F, int n, int s, int it) {
    constexpr int L = 4;
    const Field& A = pick(F);
    const Views& V = A.V;
    const int q = threadIdx.x & (L - 1);
    const unsigned gmask = group_mask<L>();
    const int gx = blockIdx.x * (256 / L) + (int)(threadIdx.x / L), gy = blockIdx.y;
    if (gx >= A.gw || gy >= A.gh) return;  // the whole group
    const size_t si = (size_t)gy * A.gw + gx;
    int c = A.cost[si];
    if (c == kEmpty) return;
    const int x = gx * n, y = gy * n;
    const size_t i = pix(V.w, x, y);
    Vec4 cur = unpack_vec(A.field[si]);
    Slice<L> r;
    load_slice<L>(V.ref, i, q, r);
    if (update_pixel<L>(V, r, q, gmask, n, s, A.key, A.mirror, x, y, (uint32_t)i, it, -1, cur, kEmpty, cur, kEmpty,
                        cur, c) &&
        q == 0) {
        A.field[si] = pack_vec(cur);
        A.cost[si] = c;
    }
}

// ---------------------------------------------------------------------------
// The paper's own cost (Eq. 1): the sum over a 7 x 7 window (stride n) of the
// Euclidean distances between the reference view's SIFT-PCA features phi
// and those of the three other views (sff_sift.cu computes phi).  Every
// float operation is written out in the definition's order, so a cost does
// not depend on the compiler or the machine; the non-negative float is kept as its bit
// pattern, which orders like the float, so the int32 cost state and its
// comparisons serve unchanged.  These kernels keep the state at full
// resolution ([y][x]) and update it in place: a half-step writes one colour
// and reads the other, the search and the inheritance only the pixel
// itself.  The initialisation's nearest neighbours are still those of the WHT
// features (Sec. 3.1 "Initialization"); its combinations are scored with
// this cost.
struct SiftViews {
    const float4 *ref, *tmp, *ste, *crs;  // phi of the scale, [y][x]
    int w, h, n, sigma;
};

__device__ __forceinline__ float sift_dist(float4 a, float4 b) {
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
}

__device__ int sift_cost(const SiftViews& S, int px, int py, const Vec4& a) {
    float c = 0.0f;
    for (int j = -3; j <= 3; ++j) {
        const int y = py + j * S.n;
        const size_t ry = (size_t)clampi(y, 0, S.h - 1) * S.w, ty = (size_t)clampi(y + a.v, 0, S.h - 1) * S.w;
        for (int i = -3; i <= 3; ++i) {
            const int x = px + i * S.n;
            const float4 r = __ldg(S.ref + ry + clampi(x, 0, S.w - 1));
            const float4 t = __ldg(S.tmp + ty + clampi(x + a.u, 0, S.w - 1));
            const float4 st = __ldg(S.ste + ry + clampi(x - S.sigma * a.d0, 0, S.w - 1));
            const float4 cr = __ldg(S.crs + ty + clampi(x + a.u - S.sigma * a.d1, 0, S.w - 1));
            c = __fadd_rn(c, sift_dist(r, t));
            c = __fadd_rn(c, sift_dist(r, st));
            c = __fadd_rn(c, sift_dist(r, cr));
        }
    }
    return __float_as_int(c);
}

__global__ void k_sift_clear(uint2* field, int* cost, size_t np) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    field[i] = make_uint2(0u, 0u);
    cost[i] = kEmpty;
}

// The K nearest epipolar points of one coarsest-grid row by WHT distance, in
// (distance, x) order, among the points with sigma (xlim - x) >= 0: K rounds,
// each taking the smallest pair after the previous one.  All lanes return
// the same list.
__device__ int warp_row_topk(const RefFeat& r, const int4* rec, const int* rec_n, int n, int gw, int gy, int xlim,
                             int sigma, int lane, int K, int* kd, int* kx) {
    const int4* row = rec + (size_t)gy * gw * 3;
    const int* row_n = rec_n + (size_t)gy * gw;
    int pd = -1, px = -1, cnt = 0;
    for (int k = 0; k < K; ++k) {
        int bd = 0x7fffffff, bx = 0x7fffffff;
        for (int g = lane; g < gw; g += 32) {
            const int x = g * n;
            if (sigma * (xlim - x) < 0) continue;
            const int4 q0 = __ldg(row + 3 * g), q1 = __ldg(row + 3 * g + 1), q2 = __ldg(row + 3 * g + 2);
            int dot = 0;
            dot = __dp4a(r.a[0], q0.x, dot); dot = __dp4a(r.a[1], q0.y, dot);
            dot = __dp4a(r.a[2], q0.z, dot); dot = __dp4a(r.a[3], q0.w, dot);
            dot = __dp4a(r.a[4], q1.x, dot); dot = __dp4a(r.a[5], q1.y, dot);
            dot = __dp4a(r.a[6], q1.z, dot); dot = __dp4a(r.a[7], q1.w, dot);
            dot = __dp4a(r.a[8], q2.x, dot); dot = __dp4a(r.a[9], q2.y, dot);
            dot = __dp4a(r.a[10], q2.z, dot); dot = __dp4a(r.a[11], q2.w, dot);
            const int d = r.n + __ldg(row_n + g) - 2 * dot;
            const bool after = d > pd || (d == pd && x > px);
            if (after && (d < bd || (d == bd && x < bx))) {
                bd = d;
                bx = x;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int od = __shfl_xor_sync(0xffffffffu, bd, o), ox = __shfl_xor_sync(0xffffffffu, bx, o);
            if (od < bd || (od == bd && ox < bx)) {
                bd = od;
                bx = ox;
            }
        }
        if (bx == 0x7fffffff) break;
        kd[k] = bd;
        kx[k] = bx;
        pd = bd;
        px = bx;
        ++cnt;
    }
    return cnt;
}

// One warp per coarsest-grid query: all K_T x K_E x K_E combinations, each
// scored by one lane; the first minimum in (temporal, stereo, cross) rank
// order wins, as in a sequential loop with a strict comparison.
__global__ void k_sift_init(const __grid_constant__ Fields F, SiftViews S, int n, int knn_t, int knn_e, uint2* field,
                            int* cost) {
    const Field& A = F.f[0];
    const Views& V = A.V;
    const int gw = A.gw;
    const int qi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qi >= A.gq) return;  // warp-uniform
    const int px = (qi % gw) * n, py = (qi / gw) * n;
    RefFeat r;
    load_ref(V.ref, pix(V.w, px, py), r);
    int sd[SFF_MAX_KNN], sx[SFF_MAX_KNN], xd[SFF_MAX_KNN], xx[SFF_MAX_KNN];
    const int ns = warp_row_topk(r, A.rec, A.rec_n, n, gw, qi / gw, px, V.sigma, lane, knn_e, sd, sx);
    int best = kEmpty;
    Vec4 bv = {0, 0, 0, 0};
    const int2* src = A.best8 + (size_t)qi * 8;
    for (int k = 0; k < knn_t && k < 8; ++k) {
        const int2 e = src[k];
        if (e.x == 0x7fffffff || e.y < 0 || e.y >= A.gq) break;
        const int tx = (e.y % gw) * n, ty = (e.y / gw) * n;
        const int nx = warp_row_topk(r, A.rec + (size_t)A.gq * 3, A.rec_n + A.gq, n, gw, e.y / gw, tx, V.sigma, lane,
                                     knn_e, xd, xx);
        // lane l scores combination (l / nx, l % nx)
        unsigned long long key = ~0ull;
        Vec4 cand = {tx - px, ty - py, 0, 0};
        for (int l0 = 0; l0 < ns * nx; l0 += 32) {
            const int l = l0 + lane;
            if (l < ns * nx) {
                int sxl = sx[0], cxl = xx[0];
#pragma unroll
                for (int t = 0; t < SFF_MAX_KNN; ++t) {
                    if (t == l / nx) sxl = sx[t];
                    if (t == l % nx) cxl = xx[t];
                }
                Vec4 u = {tx - px, ty - py, V.sigma * (px - sxl), V.sigma * (tx - cxl)};
                u.u = (int16_t)u.u;
                u.v = (int16_t)u.v;
                u.d0 = (int16_t)u.d0;
                u.d1 = (int16_t)u.d1;
                const int c = sift_cost(S, px, py, u);
                const unsigned long long kk = ((unsigned long long)(unsigned)c << 32) | (unsigned)l;
                if (kk < key) {
                    key = kk;
                    cand = u;
                }
            }
        }
        // the smallest (cost, combination) key of the warp and its lane
        unsigned long long m = key;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long om = __shfl_xor_sync(0xffffffffu, m, o);
            m = om < m ? om : m;
        }
        const int c = (int)(m >> 32);
        const int owner = __ffs(__ballot_sync(0xffffffffu, key == m && m != ~0ull)) - 1;
        if (owner >= 0 && c < best) {
            best = c;
            bv.u = __shfl_sync(0xffffffffu, cand.u, owner);
            bv.v = __shfl_sync(0xffffffffu, cand.v, owner);
            bv.d0 = __shfl_sync(0xffffffffu, cand.d0, owner);
            bv.d1 = __shfl_sync(0xffffffffu, cand.d1, owner);
        }
    }
    if (lane == 0) {
        field[pix(V.w, px, py)] = pack_vec(bv);
        cost[pix(V.w, px, py)] = best;
    }
}

__global__ void k_sift_inherit(SiftViews S, int gw, int gh, uint2* field, int* cost) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= gw || gy >= gh) return;
    const int x = gx * S.n, y = gy * S.n;
    const size_t i = pix(S.w, x, y);
    if (((gx | gy) & 1) == 0 && cost[i] != kEmpty) {
        cost[i] = sift_cost(S, x, y, unpack_vec(field[i]));
    } else {
        cost[i] = kEmpty;
        field[i] = make_uint2(0u, 0u);
    }
}

// Half-step of one colour: the pixel's own vector against its horizontal,
// then its vertical predecessor's (strictly lower cost wins).
__global__ void k_sift_half(SiftViews S, int gw, int gh, int colour, int dx, int dy, uint2* field, int* cost) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= gw || gy >= gh || ((gx + gy) & 1) != colour) return;
    const int x = gx * S.n, y = gy * S.n;
    const size_t i = pix(S.w, x, y);
    int bc = cost[i];
    uint2 bw = field[i];
    const int qx[2] = {x - dx * S.n, x}, qy[2] = {y, y - dy * S.n};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (qx[k] < 0 || qy[k] < 0 || qx[k] >= S.w || qy[k] >= S.h) continue;
        const size_t j = pix(S.w, qx[k], qy[k]);
        if (cost[j] == kEmpty) continue;
        const uint2 w = field[j];
        const int c = sift_cost(S, x, y, unpack_vec(w));
        if (c < bc) {
            bc = c;
            bw = w;
        }
    }
    field[i] = bw;
    cost[i] = bc;
}

__global__ void k_sift_search(SiftViews S, int gw, int gh, int s, int it, int mirror, uint2 key, uint2* field,
                              int* cost) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= gw || gy >= gh) return;
    const int x = gx * S.n, y = gy * S.n;
    const size_t i = pix(S.w, x, y);
    const int c0 = cost[i];
    if (c0 == kEmpty) return;
    const Vec4 a = unpack_vec(field[i]);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)it, (uint32_t)(s + 4 * mirror), 0u), key);
    Vec4 u = {a.u + rs_offset(r.x, S.n), a.v + rs_offset(r.y, S.n), a.d0 + rs_offset(r.z, S.n),
              a.d1 + rs_offset(r.w, S.n)};
    if (u.d0 < 0) u.d0 = 0;
    if (u.d1 < 0) u.d1 = 0;
    u.u = (int16_t)u.u;
    u.v = (int16_t)u.v;
    u.d0 = (int16_t)u.d0;
    u.d1 = (int16_t)u.d1;
    const int c = sift_cost(S, x, y, u);
    if (c < c0) {
        field[i] = pack_vec(u);
        cost[i] = c;
    }
}

// Instantiated variants of the iteration kernel; any of them gives identical
// results.  slots = 0: k_iteration with L lanes per pixel; slots = 1 or 4:
// k_iteration_lat with that many candidate slots of L lanes.
using IterKernel = void (*)(Fields, IterStep);
struct IterVariant {
    int lanes, slots, tx, ty, ctas;
    IterKernel k;
    int threads;
};
#define SFF_ITER_V(L, X, Y) {L, 0, X, Y, 0, k_iteration<L, X, Y, 0>, iter_threads<L, X, Y>()}
#define SFF_ITER_VB(L, X, Y, MB) {L, 0, X, Y, MB, k_iteration<L, X, Y, MB>, iter_threads<L, X, Y>()}
#define SFF_ITER_VARIANTS(L)                                                                        \
    SFF_ITER_V(L, 64, 16), SFF_ITER_V(L, 32, 16), SFF_ITER_V(L, 64, 8), SFF_ITER_V(L, 32, 8), \
        SFF_ITER_V(L, 16, 8), SFF_ITER_V(L, 8, 8)
#define SFF_LAT_V(L, C, X, Y) {L, C, X, Y, 0, k_iteration_lat<L, C, X, Y>, lat_threads<L * C, X, Y>()}
const IterVariant kIterVariants[] = {
    SFF_ITER_VARIANTS(1), SFF_ITER_VARIANTS(2), SFF_ITER_VARIANTS(4),
    // throughput form with a register budget for more resident CTAs per SM
    SFF_ITER_VB(1, 64, 16, 2), SFF_ITER_VB(1, 32, 16, 3), SFF_ITER_VB(1, 32, 16, 4), SFF_ITER_VB(1, 32, 8, 6),
    SFF_ITER_VB(1, 32, 8, 7), SFF_ITER_VB(1, 32, 8, 8), SFF_ITER_VB(1, 16, 8, 12),
    // latency form: every tile whose region fits one cell per group in 1024 threads
    SFF_LAT_V(1, 1, 64, 16), SFF_LAT_V(1, 1, 32, 16), SFF_LAT_V(1, 1, 64, 8), SFF_LAT_V(1, 1, 32, 8),
    SFF_LAT_V(1, 1, 16, 8), SFF_LAT_V(1, 1, 8, 8),
    SFF_LAT_V(2, 1, 32, 16), SFF_LAT_V(2, 1, 64, 8), SFF_LAT_V(2, 1, 32, 8), SFF_LAT_V(2, 1, 16, 8),
    SFF_LAT_V(2, 1, 8, 8),
    SFF_LAT_V(4, 1, 32, 8), SFF_LAT_V(4, 1, 16, 8), SFF_LAT_V(4, 1, 8, 8),
    SFF_LAT_V(1, 4, 32, 8), SFF_LAT_V(1, 4, 16, 8), SFF_LAT_V(1, 4, 8, 8),
    SFF_LAT_V(2, 4, 16, 8), SFF_LAT_V(2, 4, 8, 8),
    SFF_LAT_V(4, 4, 8, 8)};
#undef SFF_LAT_V
#undef SFF_ITER_VARIANTS
#undef SFF_ITER_VB
#undef SFF_ITER_V

const IterVariant* find_variant(int lanes, int slots, int tx, int ty, int ctas) {
    for (const auto& v : kIterVariants)
        if (v.lanes == lanes && v.slots == slots && v.tx == tx && v.ty == ty && v.ctas == ctas) return &v;
    return nullptr;
}

// Variants that also exist in the fused form (k_iteration_fused).
using FusedKernel = void (*)(Fields, FusedStep);
struct FusedVariant {
    int lanes, slots, tx, ty, ctas;
    FusedKernel k;
    int threads;
};
#define SFF_FUSED_V(L, C, X, Y, MB) {L, C, X, Y, MB, k_iteration_fused<L, C, X, Y, MB>, fused_threads<L, C, X, Y>()}
const FusedVariant kFusedVariants[] = {
    // throughput form
    SFF_FUSED_V(1, 0, 32, 16, 0), SFF_FUSED_V(1, 0, 32, 16, 4), SFF_FUSED_V(1, 0, 32, 8, 0),
    SFF_FUSED_V(1, 0, 32, 8, 7), SFF_FUSED_V(2, 0, 32, 8, 0),
    // latency form
    SFF_FUSED_V(1, 1, 32, 16, 0), SFF_FUSED_V(1, 1, 32, 8, 0), SFF_FUSED_V(1, 1, 16, 8, 0), SFF_FUSED_V(1, 1, 8, 8, 0),
    SFF_FUSED_V(2, 1, 32, 8, 0), SFF_FUSED_V(2, 1, 16, 8, 0), SFF_FUSED_V(2, 1, 8, 8, 0), SFF_FUSED_V(1, 4, 16, 8, 0),
    SFF_FUSED_V(1, 4, 8, 8, 0), SFF_FUSED_V(2, 4, 8, 8, 0)};
#undef SFF_FUSED_V
constexpr int kNumFused = (int)(sizeof kFusedVariants / sizeof kFusedVariants[0]);

const FusedVariant* find_fused(int lanes, int slots, int tx, int ty, int ctas) {
    for (const auto& v : kFusedVariants)
        if (v.lanes == lanes && v.slots == slots && v.tx == tx && v.ty == ty && v.ctas == ctas) return &v;
    return nullptr;
}

// Scale-0 throughput variants that also exist with TMA-staged reference
// records (k_iteration_tma, sff_tuning.tma).
using TmaKernel = void (*)(Fields, IterStep, RefMaps);
struct TmaVariant {
    int lanes, tx, ty, ctas;
    TmaKernel k;
    int threads;
};
#define SFF_TMA_V(L, X, Y, MB) {L, X, Y, MB, k_iteration_tma<L, X, Y, MB>, iter_threads<L, X, Y>()}
const TmaVariant kTmaVariants[] = {SFF_TMA_V(1, 32, 16, 0), SFF_TMA_V(1, 32, 16, 3), SFF_TMA_V(1, 32, 8, 0),
                                   SFF_TMA_V(1, 32, 8, 7)};
#undef SFF_TMA_V
static_assert(sizeof(Fields) + sizeof(IterStep) + sizeof(RefMaps) <= 32000, "kernel parameters of k_iteration_tma");

const TmaVariant* find_tma(int lanes, int slots, int tx, int ty, int ctas) {
    if (slots != 0) return nullptr;
    for (const auto& v : kTmaVariants)
        if (v.lanes == lanes && v.tx == tx && v.ty == ty && v.ctas == ctas) return &v;
    return nullptr;
}

// cuTensorMapEncodeTiled, resolved from the driver at run time (the library
// links only the runtime).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map of the scale-0 reference records of a w x h image (chunk planes
// of pyramid `pyr`, 16-byte aligned) with the box of one TX x TY tile's region.
bool encode_ref_map(CUtensorMap* m, const uint8_t* pyr, int w, int h, int S, int tx, int ty) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !chunk_planes(0)) return false;
    const Plane P = plane_of(pyr, 0, S, w, h);
    const cuuint64_t dim[4] = {4, (cuuint64_t)w, (cuuint64_t)h, 3};
    const cuuint64_t stride[3] = {16, (cuuint64_t)16 * w, (cuuint64_t)16 * w * h};
    const cuuint32_t box[4] = {4, (cuuint32_t)(tx + 1), (cuuint32_t)(ty + 1), 3};
    const cuuint32_t estride[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<int4*>(P.f), dim, stride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// CTAs of a fused variant that can be resident at once on this device (the
// largest grid of its cooperative launch); 0 on error.
int fused_capacity(const FusedVariant* v) {
    static std::mutex mu;
    static int cap[64][kNumFused] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int idx = (int)(v - kFusedVariants);
    std::lock_guard<std::mutex> lk(mu);
    if (cap[dev][idx] == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v->k, v->threads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        cap[dev][idx] = per_sm * sms;
    }
    return cap[dev][idx];
}

// A tuning is valid when its scale-0 variant exists and every coarse entry is
// either all zero (chosen from the grid size) or an existing variant.
bool tuning_valid(const sff_tuning& t) {
    if (!find_variant(t.lanes_per_pixel, t.slots, t.tile_x, t.tile_y, t.min_ctas)) return false;
    if (t.group_mb < 0 || t.group_mb > (1 << 20) || (t.pair_fields != 0 && t.pair_fields != 1) ||
        t.alternate_order < 0 || t.alternate_order > 15 || t.features_form < 0 || t.features_form > 2 ||
        t.pdl < 0 || t.pdl > 15 || t.fuse < 0 || t.fuse > 15 || (t.fuse & 1) ||
        (t.fuse & (t.pdl | t.alternate_order)) != 0 || (t.tma != 0 && t.tma != 1) ||
        (t.overlap != 0 && t.overlap != 1))
        return false;
    if (t.tma && !find_tma(t.lanes_per_pixel, t.slots, t.tile_x, t.tile_y, t.min_ctas)) return false;
    for (int k = 0; k < SFF_MAX_SCALES - 1; ++k) {
        const int32_t* c = t.coarse[k];
        if ((c[0] | c[1] | c[2] | c[3] | c[4]) != 0 && !find_variant(c[0], c[1], c[2], c[3], c[4])) return false;
        // a fused scale's variant has a fused form (both derived variants do)
        if (((t.fuse >> (k + 1)) & 1) && (c[0] | c[1] | c[2] | c[3] | c[4]) != 0 &&
            !find_fused(c[0], c[1], c[2], c[3], c[4]))
            return false;
    }
    return true;
}

// Variant of the iteration kernel at one scale.  Scale 0 takes the tuned
// variant, a coarser scale its tuning entry when one is given.  Otherwise it
// is chosen by the number of grid pixels per SM over all fields: a coarse
// scale is latency-bound (few grid pixels per SM, each a chain of dependent
// feature loads).  Measured per launch on the 1242x375 driving quad (both
// fields): at scale 1 (1536 pixels per SM) and scale 2 (385) one lane per
// pixel on 32 x 16 tiles was fastest of all 38 variants (23.2, 12.9 us), at
// scale 3 (96) the latency form with a slot per candidate on 16 x 8 tiles
// (8.9 us against 13.3).  Every variant gives the same result.
constexpr int kSmCount = 152;
constexpr long kPixPerSmSlots = 200;

const IterVariant* variant_for_scale(const sff_tuning& t, int s, const int* gw, const int* gh, int nf) {
    if (s == 0) return find_variant(t.lanes_per_pixel, t.slots, t.tile_x, t.tile_y, t.min_ctas);
    const int32_t* c = t.coarse[s - 1];
    if ((c[0] | c[1] | c[2] | c[3] | c[4]) != 0) return find_variant(c[0], c[1], c[2], c[3], c[4]);
    long px = 0;
    for (int k = 0; k < nf; ++k) px += (long)gw[k] * gh[k];
    return px / kSmCount < kPixPerSmSlots ? find_variant(1, 4, 16, 8, 0) : find_variant(1, 0, 32, 16, 0);
}

int coarse_gq(int w, int h, const sff_params& p) {
    const int n = 1 << (p.num_scales - 1);
    return ((w + n - 1) / n) * ((h + n - 1) / n);
}

// Scratch of one field: K-NN lists and the augmented coarsest-grid rows
// (whole 16 KB tiles, so every bulk copy starts and ends on 16 bytes), then
// a second state buffer (field + cost) for the double-buffered iterations,
// the grid-barrier counters and the change stamps (one byte per pixel,
// reused by every scale).
struct FieldScratch {
    size_t best8, tk, rec, rec_n, field, cost, sync, stamp, total;
};
FieldScratch field_scratch(int w, int h, const sff_params& p) {
    const int gq = coarse_gq(w, h, p);
    FieldScratch f;
    f.best8 = 0;
    f.tk = f.best8 + align256((size_t)gq * 8 * sizeof(int2));
    f.rec = f.tk + align256((size_t)2 * tc_rows(gq) * kTcK * 2);
    f.rec_n = f.rec + align256((size_t)2 * gq * kFeat);
    f.field = f.rec_n + align256((size_t)2 * gq * sizeof(int));
    f.cost = f.field + align256((size_t)w * h * 8);
    f.sync = f.cost + align256((size_t)w * h * 4);
    f.stamp = f.sync + 256;
    f.total = f.stamp + align256((size_t)w * h);
    return f;
}

}  // namespace

size_t field_ws_bytes(int w, int h, const sff_params& p) { return field_scratch(w, h, p).total; }

// Workspace of sff_match_views / sff_match_quad: the scratch of two fields.
size_t match_ws_bytes(int w, int h, const sff_params& p) { return 2 * field_ws_bytes(w, h, p); }

// Opts k_knn_tc into its dynamic shared memory, once per device.
bool knn_smem_ready() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(k_knn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes) != cudaSuccess)
            return false;
        done[dev] = true;
    }
    return true;
}

// The stage of Sec. 3.1 for nf <= kMaxFields fields (any sizes) sharing the
// launches.  spec[k].workspace holds field_ws_bytes() of scratch.
int run_fields(const FieldSpec* spec, int nf, const sff_params& P, const sff_tuning& T, cudaStream_t st,
               bool sequential, const cudaEvent_t* scale_ready, const ForkHook* fork_hook) {
    if (!tuning_valid(T) || nf < 1 || nf > kMaxFields) return SFF_ERR_ARG;
    const int S = P.num_scales, I = P.iterations;
    static const int kDirs[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    static Fields F;  // host staging of the kernel parameter (copied at each launch)
    static RefMaps RM;  // tensor maps of the TMA variant (scale 0)
    std::lock_guard<std::mutex> lk(g_fields_mu);
    memset(&F, 0, sizeof F);
    uint2* U[kMaxFields];
    int* Uc[kMaxFields];
    uint2* Tf[kMaxFields];
    int* Tc[kMaxFields];
    int gw[kMaxFields], gh[kMaxFields];
    for (int k = 0; k < nf; ++k) {
        const FieldSpec& fs = spec[k];
        const FieldScratch sc = field_scratch(fs.width, fs.height, P);
        char* ws = reinterpret_cast<char*>(fs.workspace);
        F.f[k].best8 = reinterpret_cast<int2*>(ws + sc.best8);
        F.f[k].tk = reinterpret_cast<uint8_t*>(ws + sc.tk);
        F.f[k].rec = reinterpret_cast<int4*>(ws + sc.rec);
        F.f[k].rec_n = reinterpret_cast<int*>(ws + sc.rec_n);
        F.f[k].sync = reinterpret_cast<unsigned*>(ws + sc.sync);
        F.f[k].stamp = reinterpret_cast<uint8_t*>(ws + sc.stamp);
        F.f[k].gq = coarse_gq(fs.width, fs.height, P);
        F.f[k].mirror = fs.mirror;
        F.f[k].key = make_uint2((uint32_t)fs.seed, (uint32_t)(fs.seed >> 32));
        U[k] = reinterpret_cast<uint2*>(fs.field);
        Uc[k] = fs.cost;
        Tf[k] = reinterpret_cast<uint2*>(ws + sc.field);
        Tc[k] = reinterpret_cast<int*>(ws + sc.cost);
    }
    // State buffers: 0 = the caller's (U), 1 = the workspace's (T).  Each
    // scale keeps its state compact (grid row-major; at scale 0 that is the
    // image).  The initialisation or inheritance writes buffer `cur`, the
    // iterations alternate from it, and the next finer scale inherits from
    // the final one into the other buffer; the start is chosen so that scale
    // 0 ends in U.
    uint2* Bf[2][kMaxFields];
    int* Bc[2][kMaxFields];
    for (int k = 0; k < nf; ++k) {
        Bf[0][k] = U[k];
        Bc[0][k] = Uc[k];
        Bf[1][k] = Tf[k];
        Bc[1][k] = Tc[k];
    }
    // With checkerboard iterations the first iteration of each finer scale
    // also does the inheritance (TileStep::inherit): it reads the coarser
    // scale's final buffer and writes the other one.  The sequential sweeps
    // (in place) and a run without iterations inherit with k_inherit into
    // the other buffer.
    const bool fused_inherit = !sequential && I > 0;
    const int flips = sequential ? 0 : (I & 1);  // the sweeps work in place
    auto final_of_scale0 = [&](int b) {
        for (int s = S - 1; s >= 0; --s) {
            if (s < S - 1 && !fused_inherit) b ^= 1;  // inherit into the other buffer
            b ^= flips;                                // after the iterations
        }
        return b;
    };
    int cur = final_of_scale0(0) == 0 ? 0 : 1, prev = 0;
    for (int s = S - 1; s >= 0; --s) {
        const int n = 1 << s;
        int mgw = 0, mgh = 0, mgq = 0;
        const bool inherit = s < S - 1 && fused_inherit;  // the first iteration inherits
        if (s < S - 1) cur = fused_inherit ? prev : prev ^ 1;
        for (int k = 0; k < nf; ++k) {
            const FieldSpec& fs = spec[k];
            const int w = fs.width, h = fs.height;
            F.f[k].V = Views{plane_of(fs.ref, s, S, w, h), plane_of(fs.tmp, s, S, w, h), plane_of(fs.ste, s, S, w, h),
                             plane_of(fs.crs, s, S, w, h), w, h, fs.mirror ? -1 : 1};
            if (s == S - 1) {  // k_init_select writes the state
                F.f[k].field = F.f[k].field_out = Bf[cur][k];
                F.f[k].cost = F.f[k].cost_out = Bc[cur][k];
            } else {  // k_inherit reads the coarser final state, writes this scale's (unless
                      // the first iteration inherits: it sets its own buffers)
                F.f[k].field = Bf[prev][k];
                F.f[k].cost = Bc[prev][k];
                F.f[k].field_out = Bf[cur][k];
                F.f[k].cost_out = Bc[cur][k];
            }
            gw[k] = F.f[k].gw = (w + n - 1) / n;
            gh[k] = F.f[k].gh = (h + n - 1) / n;
            mgw = std::max(mgw, gw[k]);
            mgh = std::max(mgh, gh[k]);
            mgq = std::max(mgq, F.f[k].gq);
        }
        if (s == S - 1) {
            dim3 g0((tc_rows(mgq) * 8 + 255) / 256, 4, nf);
            SFF_LAUNCH(k_gather_grid, g0, 256, 0, st, F, n);
            if (!knn_smem_ready()) return SFF_ERR_CUDA;
            if (fork_hook) {
                const int status = fork_hook->fn(fork_hook->ctx, st);
                if (status) return status;
            }
            dim3 g1((mgq + kTcRows - 1) / kTcRows, 1, nf);
            SFF_LAUNCH(k_knn_tc, g1, kTcThreads, kTcSmemBytes, st, F);
            dim3 g2((mgq + 7) / 8, 1, nf);
            SFF_LAUNCH(k_init_select, g2, 256, 0, st, F, n, P.knn_temporal);
        } else {
            // the features of this scale may still be in flight on another stream
            if (scale_ready && cudaStreamWaitEvent(st, scale_ready[s], 0) != cudaSuccess) return SFF_ERR_CUDA;
            if (!inherit) {
                dim3 g((mgw + 127) / 128, mgh, nf);
                SFF_LAUNCH(k_inherit, g, 128, 0, st, F, n);
            }
        }
        if (sequential) {
            for (int k = 0; k < nf; ++k) {
                F.f[k].field = F.f[k].field_out = Bf[cur][k];
                F.f[k].cost = F.f[k].cost_out = Bc[cur][k];
            }
            dim3 gr((mgw + 63) / 64, mgh, nf);
            for (int it = 0; it < I; ++it) {
                SFF_LAUNCH(k_sweep, dim3(1, 1, nf), kSweepThreads, 0, st, F, n, kDirs[it % 4][0], kDirs[it % 4][1]);
                SFF_LAUNCH(k_random_search, gr, 256, 0, st, F, n, s, it);
            }
            prev = cur;
            continue;
        }
        // profiled as one span per scale (and group), "k_iteration/s<scale>"
        static const char* const kIterNames[SFF_MAX_SCALES] = {"k_iteration/s0", "k_iteration/s1", "k_iteration/s2",
                                                               "k_iteration/s3"};
        // Scale 0 may run its iterations for consecutive groups of fields in
        // turn (T.group_mb): all iterations of one group, then the next, so
        // that a group's features and state stay in L2 across iterations.
        // Fields of one quad share their pyramids and are never split.
        for (int f0 = 0; f0 < nf;) {
            int f1 = nf;
            if (s == 0 && T.group_mb > 0) {
                const double budget = (double)T.group_mb * (1 << 20);
                double used = 0.0;
                f1 = f0;
                while (f1 < nf) {
                    const bool pair = f1 + 1 < nf && spec[f1 + 1].width == spec[f1].width &&
                                      spec[f1 + 1].height == spec[f1].height && spec[f1 + 1].ref == spec[f1].crs;
                    const int take = pair ? 2 : 1;
                    // four images' records + both fields' double-buffered state
                    const double ws = (double)spec[f1].width * spec[f1].height * (4.0 * kFeat + take * 24.0);
                    if (f1 > f0 && used + ws > budget) break;
                    used += ws;
                    f1 += take;
                }
            }
            int ggw = 0, ggh = 0;
            for (int k = f0; k < f1; ++k) {
                ggw = std::max(ggw, gw[k]);
                ggh = std::max(ggh, gh[k]);
            }
            const IterVariant* sv = variant_for_scale(T, s, gw + f0, gh + f0, f1 - f0);
            // pairs: every field f0 + 2j, f0 + 2j + 1 one quad's two fields
            bool pair = T.pair_fields != 0 && ((f1 - f0) & 1) == 0;
            for (int k = f0; pair && k < f1; k += 2)
                pair = spec[k + 1].width == spec[k].width && spec[k + 1].height == spec[k].height &&
                       spec[k + 1].ref == spec[k].crs;
            const unsigned tiles_x = (ggw + sv->tx - 1) / sv->tx;
            dim3 gi(pair ? 2 * tiles_x : tiles_x, (ggh + sv->ty - 1) / sv->ty, pair ? (f1 - f0) / 2 : f1 - f0);
            const bool fuse = ((T.fuse >> s) & 1) != 0 && I > 0;
            if (I > 0 && ::sff::profiling()) ::sff::profile_mark(kIterNames[s], st, false);
            if (fuse) {
                // one cooperative launch for all iterations (a variant with a
                // fused form: validated, or one of the derived ones)
                const FusedVariant* fv = find_fused(sv->lanes, sv->slots, sv->tx, sv->ty, sv->ctas);
                if (!fv) return SFF_ERR_ARG;
                const int cap = fused_capacity(fv);
                if (cap <= 0) return SFF_ERR_CUDA;
                const int tiles_x = (ggw + sv->tx - 1) / sv->tx, tiles_y = (ggh + sv->ty - 1) / sv->ty;
                const int total = tiles_x * tiles_y * (f1 - f0);
                for (int k = f0; k < f1; ++k) {
                    F.f[k].field = Bf[cur][k];
                    F.f[k].cost = Bc[cur][k];
                    F.f[k].field_out = Bf[cur ^ 1][k];
                    F.f[k].cost_out = Bc[cur ^ 1][k];
                }
                FusedStep FH{n, s, I, f0, f1 - f0, tiles_x, tiles_y, F.f[f0].sync + s, inherit ? 1 : 0};
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)std::min(total, cap));
                cfg.blockDim = dim3(fv->threads);
                cfg.dynamicSmemBytes = 0;
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                if (cudaLaunchKernelEx(&cfg, fv->k, F, FH) != cudaSuccess) return SFF_ERR_CUDA;
            }
            // scale 0 with TMA-staged reference records: one tensor map per field
            const TmaVariant* tv = nullptr;
            if (s == 0 && T.tma && !fuse && I > 0) {
                tv = find_tma(sv->lanes, sv->slots, sv->tx, sv->ty, sv->ctas);
                if (!tv) return SFF_ERR_ARG;
                for (int k = f0; k < f1; ++k)
                    if (!encode_ref_map(&RM.m[k], spec[k].ref, spec[k].width, spec[k].height, S, sv->tx, sv->ty))
                        return SFF_ERR_CUDA;
            }
            for (int it = 0; it < (fuse ? 0 : I); ++it) {
                const int in = cur ^ (it & 1);
                for (int k = f0; k < f1; ++k) {
                    F.f[k].field = Bf[in][k];
                    F.f[k].cost = Bc[in][k];
                    F.f[k].field_out = Bf[in ^ 1][k];
                    F.f[k].cost_out = Bc[in ^ 1][k];
                }
                IterStep H{n,      s,  kDirs[it % 4][0], kDirs[it % 4][1], it, it == I - 1, f0, pair ? 1 : 0,
                           ((T.alternate_order >> s) & 1) ? (it & 1) : 0, inherit && it == 0 ? 1 : 0};
                if (tv) {
                    // TMA-staged reference records (scale 0)
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = gi;
                    cfg.blockDim = dim3(tv->threads);
                    cfg.dynamicSmemBytes = 0;
                    cfg.stream = st;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = ((T.pdl >> s) & 1) ? 1 : 0;
                    if (cudaLaunchKernelEx(&cfg, tv->k, F, H, RM) != cudaSuccess) return SFF_ERR_CUDA;
                } else if ((T.pdl >> s) & 1) {
                    // scheduled while the previous iteration's last CTAs run;
                    // its CTAs wait in griddepcontrol.wait until it is done
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = gi;
                    cfg.blockDim = dim3(sv->threads);
                    cfg.dynamicSmemBytes = 0;
                    cfg.stream = st;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    if (cudaLaunchKernelEx(&cfg, sv->k, F, H) != cudaSuccess) return SFF_ERR_CUDA;
                } else {
                    sv->k<<<gi, sv->threads, 0, st>>>(F, H);
                }
            }
            if (I > 0 && ::sff::profiling()) ::sff::profile_mark(kIterNames[s], st, true, fuse ? 1 : I, I);
            f0 = f1;
        }
        prev = cur ^ (I & 1);
    }
    return launch_status();
}

// One field with the paper's own cost: the WHT K-NN of the coarsest scale as
// in run_fields, then initialisation, inheritance, half-steps and random
// search in the kernels above.  phi[4]: [S][H][W] float4 of the views in the
// field's roles (reference, temporal, stereo, cross).
int run_field_sift(const FieldSpec& fs, const float* const* phi, const sff_params& P, cudaStream_t st) {
    const int S = P.num_scales, I = P.iterations, w = fs.width, h = fs.height;
    static const int kDirs[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    static Fields F;
    std::lock_guard<std::mutex> lk(g_fields_mu);
    memset(&F, 0, sizeof F);
    const FieldScratch sc = field_scratch(w, h, P);
    char* ws = reinterpret_cast<char*>(fs.workspace);
    Field& A = F.f[0];
    A.best8 = reinterpret_cast<int2*>(ws + sc.best8);
    A.tk = reinterpret_cast<uint8_t*>(ws + sc.tk);
    A.rec = reinterpret_cast<int4*>(ws + sc.rec);
    A.rec_n = reinterpret_cast<int*>(ws + sc.rec_n);
    A.gq = coarse_gq(w, h, P);
    A.mirror = fs.mirror;
    A.key = make_uint2((uint32_t)fs.seed, (uint32_t)(fs.seed >> 32));
    uint2* field = reinterpret_cast<uint2*>(fs.field);
    int* cost = fs.cost;
    const size_t np = (size_t)w * h;
    SFF_LAUNCH(k_sift_clear, dim3((unsigned)((np + 255) / 256)), 256, 0, st, field, cost, np);
    for (int s = S - 1; s >= 0; --s) {
        const int n = 1 << s, gw = (w + n - 1) / n, gh = (h + n - 1) / n;
        const size_t off = (size_t)s * np;
        SiftViews SV{reinterpret_cast<const float4*>(phi[0]) + off, reinterpret_cast<const float4*>(phi[1]) + off,
                     reinterpret_cast<const float4*>(phi[2]) + off, reinterpret_cast<const float4*>(phi[3]) + off,
                     w, h, n, fs.mirror ? -1 : 1};
        const dim3 g((gw + 127) / 128, gh);
        if (s == S - 1) {
            A.V = Views{plane_of(fs.ref, s, S, w, h), plane_of(fs.tmp, s, S, w, h), plane_of(fs.ste, s, S, w, h),
                        plane_of(fs.crs, s, S, w, h), w, h, fs.mirror ? -1 : 1};
            A.gw = gw;
            A.gh = gh;
            dim3 g0((tc_rows(A.gq) * 8 + 255) / 256, 4, 1);
            SFF_LAUNCH(k_gather_grid, g0, 256, 0, st, F, n);
            if (!knn_smem_ready()) return SFF_ERR_CUDA;
            dim3 g1((A.gq + kTcRows - 1) / kTcRows, 1, 1);
            SFF_LAUNCH(k_knn_tc, g1, kTcThreads, kTcSmemBytes, st, F);
            SFF_LAUNCH(k_sift_init, dim3((A.gq + 7) / 8), 256, 0, st, F, SV, n, P.knn_temporal, P.knn_epipolar, field,
                       cost);
        } else {
            SFF_LAUNCH(k_sift_inherit, g, 128, 0, st, SV, gw, gh, field, cost);
        }
        for (int it = 0; it < I; ++it) {
            for (int colour = 0; colour < 2; ++colour)
                SFF_LAUNCH(k_sift_half, g, 128, 0, st, SV, gw, gh, colour, kDirs[it % 4][0], kDirs[it % 4][1], field,
                           cost);
            SFF_LAUNCH(k_sift_search, g, 128, 0, st, SV, gw, gh, s, it, fs.mirror, A.key, field, cost);
        }
    }
    return launch_status();
}

namespace {

bool misaligned_pyr(const uint8_t* p) { return ((uintptr_t)p & 15) != 0; }

}  // namespace

}  // namespace sff

extern "C" int sff_match_views(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                               const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev, int32_t width,
                               int32_t height, int32_t mirror, uint64_t seed, const sff_params* params,
                               int16_t* field_dev, int32_t* cost_dev, void* workspace, size_t workspace_bytes,
                               void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!pyr_ref_dev || !pyr_temporal_dev || !pyr_stereo_dev || !pyr_cross_dev || !field_dev || !cost_dev ||
        !workspace)
        return SFF_ERR_ARG;
    if (mirror != 0 && mirror != 1) return SFF_ERR_ARG;
    if (misaligned_pyr(pyr_ref_dev) || misaligned_pyr(pyr_temporal_dev) || misaligned_pyr(pyr_stereo_dev) ||
        misaligned_pyr(pyr_cross_dev))
        return SFF_ERR_ARG;
    if (((uintptr_t)field_dev & 7) || ((uintptr_t)cost_dev & 3) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < match_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    FieldSpec f{pyr_ref_dev, pyr_temporal_dev, pyr_stereo_dev, pyr_cross_dev, field_dev, cost_dev, mirror,
                width, height, seed, workspace};
    sff_tuning t;
    sff_default_tuning(&t);
    return run_fields(&f, 1, *params, t, (cudaStream_t)stream, false);
}

extern "C" int sff_match_views_sequential(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                                          const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev,
                                          int32_t width, int32_t height, int32_t mirror, uint64_t seed,
                                          const sff_params* params, int16_t* field_dev, int32_t* cost_dev,
                                          void* workspace, size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!pyr_ref_dev || !pyr_temporal_dev || !pyr_stereo_dev || !pyr_cross_dev || !field_dev || !cost_dev ||
        !workspace)
        return SFF_ERR_ARG;
    if (mirror != 0 && mirror != 1) return SFF_ERR_ARG;
    if (misaligned_pyr(pyr_ref_dev) || misaligned_pyr(pyr_temporal_dev) || misaligned_pyr(pyr_stereo_dev) ||
        misaligned_pyr(pyr_cross_dev))
        return SFF_ERR_ARG;
    if (((uintptr_t)field_dev & 7) || ((uintptr_t)cost_dev & 3) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < match_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    FieldSpec f{pyr_ref_dev, pyr_temporal_dev, pyr_stereo_dev, pyr_cross_dev, field_dev, cost_dev, mirror,
                width, height, seed, workspace};
    sff_tuning t;
    sff_default_tuning(&t);
    return run_fields(&f, 1, *params, t, (cudaStream_t)stream, true);
}

extern "C" int sff_default_tuning(sff_tuning* out) {
    if (!out) return SFF_ERR_ARG;
    memset(out, 0, sizeof *out);
    out->lanes_per_pixel = 1;
    out->tile_x = 32;
    out->tile_y = 16;
    out->overlap = 1;
    return SFF_OK;
}

extern "C" int sff_tuning_supported(const sff_tuning* t) {
    return t && sff::tuning_valid(*t) ? 1 : 0;
}

extern "C" int sff_match_quad_tuned(const uint8_t* pyr_l0_dev, const uint8_t* pyr_r0_dev, const uint8_t* pyr_l1_dev,
                                    const uint8_t* pyr_r1_dev, int32_t width, int32_t height, uint64_t seed,
                                    const sff_params* params, const sff_tuning* tuning, int16_t* fwd_dev,
                                    int32_t* fwd_cost_dev, int16_t* inv_dev, int32_t* inv_cost_dev, void* workspace,
                                    size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!tuning || !tuning_valid(*tuning)) return SFF_ERR_ARG;
    if (!pyr_l0_dev || !pyr_r0_dev || !pyr_l1_dev || !pyr_r1_dev || !fwd_dev || !fwd_cost_dev || !inv_dev ||
        !inv_cost_dev || !workspace)
        return SFF_ERR_ARG;
    if (misaligned_pyr(pyr_l0_dev) || misaligned_pyr(pyr_r0_dev) || misaligned_pyr(pyr_l1_dev) ||
        misaligned_pyr(pyr_r1_dev))
        return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)inv_dev & 7) || ((uintptr_t)fwd_cost_dev & 3) ||
        ((uintptr_t)inv_cost_dev & 3) || ((uintptr_t)workspace & 255))
        return SFF_ERR_ARG;
    if (workspace_bytes < match_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    char* ws = reinterpret_cast<char*>(workspace);
    const size_t half = field_ws_bytes(width, height, *params);
    FieldSpec f[2] = {{pyr_l0_dev, pyr_l1_dev, pyr_r0_dev, pyr_r1_dev, fwd_dev, fwd_cost_dev, 0, width, height, seed,
                       ws},
                      {pyr_r1_dev, pyr_r0_dev, pyr_l1_dev, pyr_l0_dev, inv_dev, inv_cost_dev, 1, width, height, seed,
                       ws + half}};
    return run_fields(f, 2, *params, *tuning, (cudaStream_t)stream, false);
}

extern "C" int sff_match_quad(const uint8_t* pyr_l0_dev, const uint8_t* pyr_r0_dev, const uint8_t* pyr_l1_dev,
                              const uint8_t* pyr_r1_dev, int32_t width, int32_t height, uint64_t seed,
                              const sff_params* params, int16_t* fwd_dev, int32_t* fwd_cost_dev, int16_t* inv_dev,
                              int32_t* inv_cost_dev, void* workspace, size_t workspace_bytes, void* stream) {
    sff_tuning t;
    sff_default_tuning(&t);
    return sff_match_quad_tuned(pyr_l0_dev, pyr_r0_dev, pyr_l1_dev, pyr_r1_dev, width, height, seed, params, &t,
                                fwd_dev, fwd_cost_dev, inv_dev, inv_cost_dev, workspace, workspace_bytes, stream);
}

namespace sff {
// Reads (and with reset clears) the condition bits of the matching kernels,
// in stream order; the caller synchronises the stream.
int match_status_read(cudaStream_t st, unsigned* out, bool reset) {
    static const unsigned zero = 0;
    if (cudaMemcpyFromSymbolAsync(out, g_match_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return SFF_ERR_CUDA;
    if (reset && cudaMemcpyToSymbolAsync(g_match_status, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st) !=
                     cudaSuccess)
        return SFF_ERR_CUDA;
    return SFF_OK;
}
}  // namespace sff

extern "C" int sff_debug_knn_withhold(int32_t step, int32_t wait_limit_us) {
    if (step < -1 || wait_limit_us < 0) return SFF_ERR_ARG;
    const int st = step;
    const unsigned long long ns = (unsigned long long)wait_limit_us * 1000ull;
    if (cudaMemcpyToSymbol(sff::g_withhold_step, &st, sizeof st) != cudaSuccess) return SFF_ERR_CUDA;
    if (cudaMemcpyToSymbol(sff::g_wait_limit_ns, &ns, sizeof ns) != cudaSuccess) return SFF_ERR_CUDA;
    return SFF_OK;
}

extern "C" int sff_debug_barrier_withhold(int32_t barrier, int32_t wait_limit_us) {
    if (barrier < -1 || wait_limit_us < 0) return SFF_ERR_ARG;
    const int b = barrier;
    const unsigned long long ns = (unsigned long long)wait_limit_us * 1000ull;
    if (cudaMemcpyToSymbol(sff::g_withhold_barrier, &b, sizeof b) != cudaSuccess) return SFF_ERR_CUDA;
    if (cudaMemcpyToSymbol(sff::g_wait_limit_ns, &ns, sizeof ns) != cudaSuccess) return SFF_ERR_CUDA;
    return SFF_OK;
}

extern "C" int sff_device_timeouts(uint32_t* out, int32_t reset) {
    if (!out) return SFF_ERR_ARG;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, sff::g_wait_timeouts, sizeof v) != cudaSuccess) return SFF_ERR_CUDA;
    *out = v;
    if (reset) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(sff::g_wait_timeouts, &z, sizeof z) != cudaSuccess) return SFF_ERR_CUDA;
        if (cudaMemcpyToSymbol(sff::g_drain_timeouts, &z, sizeof z) != cudaSuccess) return SFF_ERR_CUDA;
    }
    return SFF_OK;
}

extern "C" int sff_device_drain_timeouts(uint32_t* out) {
    if (!out) return SFF_ERR_ARG;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, sff::g_drain_timeouts, sizeof v) != cudaSuccess) return SFF_ERR_CUDA;
    *out = v;
    return SFF_OK;
}

extern "C" int sff_match_views_sift(const uint8_t* pyr_ref_dev, const uint8_t* pyr_temporal_dev,
                                    const uint8_t* pyr_stereo_dev, const uint8_t* pyr_cross_dev,
                                    const float* phi_ref_dev, const float* phi_temporal_dev,
                                    const float* phi_stereo_dev, const float* phi_cross_dev, int32_t width,
                                    int32_t height, int32_t mirror, uint64_t seed, const sff_params* params,
                                    int16_t* field_dev, int32_t* cost_dev, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!pyr_ref_dev || !pyr_temporal_dev || !pyr_stereo_dev || !pyr_cross_dev || !field_dev || !cost_dev ||
        !workspace || !phi_ref_dev || !phi_temporal_dev || !phi_stereo_dev || !phi_cross_dev)
        return SFF_ERR_ARG;
    if (mirror != 0 && mirror != 1) return SFF_ERR_ARG;
    if (misaligned_pyr(pyr_ref_dev) || misaligned_pyr(pyr_temporal_dev) || misaligned_pyr(pyr_stereo_dev) ||
        misaligned_pyr(pyr_cross_dev))
        return SFF_ERR_ARG;
    const float* phi[4] = {phi_ref_dev, phi_temporal_dev, phi_stereo_dev, phi_cross_dev};
    for (const float* p : phi)
        if ((uintptr_t)p & 15) return SFF_ERR_ARG;
    if (((uintptr_t)field_dev & 7) || ((uintptr_t)cost_dev & 3) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < match_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    FieldSpec f{pyr_ref_dev, pyr_temporal_dev, pyr_stereo_dev, pyr_cross_dev, field_dev, cost_dev, mirror,
                width, height, seed, workspace};
    return run_field_sift(f, phi, *params, (cudaStream_t)stream);
}
