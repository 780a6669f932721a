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
// k_gather_grid:  packs the coarsest-grid records of the reference and
//                 temporal images into contiguous arrays.
// k_knn_bound:    an exact upper bound of each query's 8th-nearest distance
//                 from a 5x5 window of coarsest-grid points around it.
// k_knn:          temporal K-NN, all-pairs over the coarsest grid, one warp
//                 per query; candidate tiles streamed into shared memory by
//                 TMA bulk copies on mbarriers (double-buffered); a sorted
//                 top-8 spread over lanes 0-7, entry capped by the bound.
// k_init_select:  one warp per query: takes the temporal top-K, finds
//                 the nearest epipolar stereo / cross points and keeps the
//                 best combination.  The cost is the sum of the three
//                 independent distances, so for a given temporal leaf the
//                 first-ranked epipolar leaves give the lowest cost and win
//                 every tie; the result equals scoring all K_T x K_E x K_E
//                 combinations in order.
// k_inherit:      grid points of the coarser scale keep their vector and are
//                 re-scored at this scale; the others start empty.
// k_half_step:    one colour of the checkerboard, four lanes per pixel.
//                 Fused with the random search of that colour: the search
//                 after iteration i of colour 1 runs at the end of its
//                 half-step of iteration i, the search of colour 0 at the
//                 start of its half-step of iteration i+1 (or in a final
//                 pass).  Both orders read the same values as the plain order
//                 "half-step 0, half-step 1, random search", because a
//                 half-step only reads the other colour and the search only
//                 reads the pixel itself.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "sff_internal.cuh"

namespace sff {
namespace {

std::mutex g_fields_mu;  // guards the host staging of the Fields parameter

constexpr int kKnnThreads = 256;
constexpr int kKnnWarps = kKnnThreads / 32;  // one query per warp
constexpr int kKnnTile = 256;                // candidates per shared-memory tile (12 KB of records)

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
    int gq, gq_pad;  // coarsest grid points and padded row count of the compact arrays
    int2* best8;  // [gq][8] temporal top-8 (distance, grid index)
    uint8_t* cf;  // [2 roles][gq_pad] 48-byte records: reference, temporal
    int* cn;  // [2 roles][gq_pad] norms
    int* bound;  // [gq] upper bound of each query's 8th-nearest temporal distance
    uint2 key;  // Philox key: the seed of the field's quad
};

// Up to kMaxFields fields of any sizes share every launch (blockIdx.z picks
// the field); passed by value as a __grid_constant__ kernel parameter.
constexpr int kMaxFields = kMaxBatchFields;
struct Fields {
    Field f[kMaxFields];
};

__device__ __forceinline__ const Field& pick(const Fields& F) { return F.f[blockIdx.z]; }

__device__ __forceinline__ bool less_di(int d, int i, int d2, int i2) { return d < d2 || (d == d2 && i < i2); }

__device__ __forceinline__ void top8_insert(int (&d)[8], int (&id)[8], int nd, int ni) {
    if (!less_di(nd, ni, d[7], id[7])) return;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        bool lt_prev = (k > 0) && less_di(nd, ni, d[k > 0 ? k - 1 : 0], id[k > 0 ? k - 1 : 0]);
        if (lt_prev) {
            d[k] = d[k - 1];
            id[k] = id[k - 1];
        } else if (less_di(nd, ni, d[k], id[k])) {
            d[k] = nd;
            id[k] = ni;
        }
    }
}

__device__ __forceinline__ int dot12(const int (&a)[12], const int4& p0, const int4& p1, const int4& p2) {
    int e = 0;
    e = __dp4a(a[0], p0.x, e); e = __dp4a(a[1], p0.y, e); e = __dp4a(a[2], p0.z, e); e = __dp4a(a[3], p0.w, e);
    e = __dp4a(a[4], p1.x, e); e = __dp4a(a[5], p1.y, e); e = __dp4a(a[6], p1.z, e); e = __dp4a(a[7], p1.w, e);
    e = __dp4a(a[8], p2.x, e); e = __dp4a(a[9], p2.y, e); e = __dp4a(a[10], p2.z, e); e = __dp4a(a[11], p2.w, e);
    return e;
}

// Copies the coarsest-grid records of the reference (role 0) and temporal
// (role 1) images of each field into contiguous arrays, so that the K-NN
// search streams them with bulk copies.  Layout per field: [2 roles][gq_pad]
// 48-byte records and int32 norms.
__global__ void k_gather_grid(const __grid_constant__ Fields F, int n) {
    const Field& A = pick(F);
    const int role = blockIdx.y;
    const Plane& P = role ? A.V.tmp : A.V.ref;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = t >> 2, part = t & 3;
    if (c >= A.gq) return;
    const size_t i = pix(A.V.w, (c % A.gw) * n, (c / A.gw) * n);
    const size_t slot = (size_t)role * A.gq_pad + c;
    if (part < 3)
        reinterpret_cast<int4*>(A.cf + slot * kFeat)[part] =
            __ldg(reinterpret_cast<const int4*>(P.f + i * kFeat) + part);
    else
        A.cn[slot] = __ldg(P.nrm + i);
}

// TMA (bulk-copy) helpers: 1-D global -> shared copies completing on an
// mbarrier.  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after kSpinLimit polls and reports false.
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (int k = 0; k < kSpinLimit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ unsigned int g_wait_timeouts;  // bounded waits that gave up (read by sff_device_timeouts)

// Upper bound of each query's 8th-nearest temporal distance: the 8th
// smallest distance among 25 distinct coarsest-grid points around the
// query's own position (a 5x5 window shifted inside the grid).  Eight real
// candidates lie at or below it, so the true 8th-nearest distance does too
// and k_knn can skip every candidate above it.  INT32_MAX (no bound) when
// the grid has fewer than 8 points in the window.  One warp per query.
__global__ void k_knn_bound(const __grid_constant__ Fields F, int n) {
    const Field& A = pick(F);
    const int qi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (qi >= A.gq) return;  // warp-uniform
    const int gw = A.gw, gh = A.gh;
    const int gx = qi % gw, gy = qi / gw;
    const int ww = min(5, gw), wh = min(5, gh);
    const int ox = clampi(gx - 2, 0, gw - ww), oy = clampi(gy - 2, 0, gh - wh);
    RefFeat r;
    load_ref(A.V.ref, pix(A.V.w, gx * n, gy * n), r);
    int d = 0x7fffffff;
    if (lane < ww * wh) d = ssd_at(r, A.V.tmp, pix(A.V.w, (ox + lane % ww) * n, (oy + lane / ww) * n));
    int t = 0x7fffffff;
    if (ww * wh >= 8) {
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {  // remove the smallest 7 times; the 8th minimum is the bound
            int m = d;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            t = m;
            const unsigned who = __ballot_sync(0xffffffffu, d == m);
            if (lane == __ffs(who) - 1) d = 0x7fffffff;
        }
    }
    if (lane == 0) A.bound[qi] = t;
}

// Temporal K-NN of one query per warp over all candidates.  The candidate
// records stream through two shared-memory tiles filled by bulk copies
// (thread 0 issues tile t+1 while tile t is scored); the 8 queries of a CTA
// share them.  Lane l scores candidate l of each batch of 32 (12 dp4a); a
// ballot against the query's current 8th-best distance, capped from the
// start by the bound of k_knn_bound, keeps the rare candidates that enter;
// each is inserted into the sorted top-8 held by lanes 0-7 with warp-uniform
// shuffles.  Candidates are visited in increasing index, so a strictly
// smaller distance is the only way in, exactly as in the (distance, index)
// order, and every candidate above the bound is provably not among the 8.
__global__ void __launch_bounds__(kKnnThreads) k_knn(const __grid_constant__ Fields F) {
    __shared__ __align__(128) int4 tile[2][kKnnTile][3];
    __shared__ __align__(16) int tnorm[2][kKnnTile];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_fail;
    const Field& A = pick(F);
    const int gq = A.gq;
    if ((int)blockIdx.x * kKnnWarps >= gq) return;  // CTA beyond this field's queries
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x * kKnnWarps + (threadIdx.x >> 5);
    const bool active = qi < gq;  // warp-uniform
    const uint8_t* tf = A.cf + (size_t)A.gq_pad * kFeat;  // role 1: candidates
    const int* tn = A.cn + A.gq_pad;
    RefFeat r;
    int lim = 0x7fffffff;
    if (active) {
        const int4* p = reinterpret_cast<const int4*>(A.cf + (size_t)qi * kFeat);  // role 0: queries
        const int4 q0 = __ldg(p), q1 = __ldg(p + 1), q2 = __ldg(p + 2);
        r.a[0] = q0.x; r.a[1] = q0.y; r.a[2] = q0.z; r.a[3] = q0.w;
        r.a[4] = q1.x; r.a[5] = q1.y; r.a[6] = q1.z; r.a[7] = q1.w;
        r.a[8] = q2.x; r.a[9] = q2.y; r.a[10] = q2.z; r.a[11] = q2.w;
        r.n = __ldg(A.cn + qi);
        const int b = A.bound[qi];
        lim = b == 0x7fffffff ? b : b + 1;  // distances <= bound may enter
    }
    const int ntiles = (gq + kKnnTile - 1) / kKnnTile;
    // copy sizes: whole records, rounded up to 4 records (16-byte multiples);
    // the arrays carry that padding
    auto issue = [&](int t) {
        const int base = t * kKnnTile;
        const int cnt4 = (min(kKnnTile, gq - base) + 3) & ~3;
        const unsigned fb = (unsigned)cnt4 * kFeat, nbytes = (unsigned)cnt4 * 4;
        mbar_expect_tx(&bar[t & 1], fb + nbytes);
        bulk_copy_g2s(&tile[t & 1][0][0], tf + (size_t)base * kFeat, fb, &bar[t & 1]);
        bulk_copy_g2s(&tnorm[t & 1][0], tn + base, nbytes, &bar[t & 1]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) issue(0);
    int ld = 0x7fffffff, li = 0x7fffffff;  // entry `lane` of the sorted top-8 (lanes 0-7)
    int thr = lim;
    for (int t = 0; t < ntiles; ++t) {
        const int buf = t & 1;
        // the other buffer was released by the __syncthreads that ended tile t-1
        if (threadIdx.x == 0 && t + 1 < ntiles) issue(t + 1);
        if (!mbar_wait(&bar[buf], (unsigned)(t >> 1) & 1u)) s_fail = 1;
        if (__syncthreads_or(s_fail)) {
            if (threadIdx.x == 0) {
                atomicAdd(&g_wait_timeouts, 1u);
                // let the copy issued for the next tile land (bounded) before the CTA exits
                if (t + 1 < ntiles) mbar_wait(&bar[buf ^ 1], (unsigned)((t + 1) >> 1) & 1u);
            }
            return;
        }
        const int base = t * kKnnTile;
        const int cnt = min(kKnnTile, gq - base);
        if (active) {
            const int4(*tl)[3] = tile[buf];
            const int* tnm = tnorm[buf];
#pragma unroll 2
            for (int b = 0; b < cnt; b += 32) {
                const int k = b + lane;
                const int d = k < cnt ? r.n + tnm[k] - 2 * dot12(r.a, tl[k][0], tl[k][1], tl[k][2]) : 0x7fffffff;
                unsigned enter = __ballot_sync(0xffffffffu, d < thr);
                while (enter) {
                    const int src = __ffs(enter) - 1;
                    enter &= enter - 1;
                    const int nd = __shfl_sync(0xffffffffu, d, src);
                    if (nd >= thr) continue;  // the threshold moved meanwhile
                    const int ni = base + b + src;
                    // entries are earlier candidates: (d, index) order is d order with ties kept
                    const int pos = __popc(__ballot_sync(0xffffffffu, lane < 8 && ld <= nd));
                    const int pd = __shfl_up_sync(0xffffffffu, ld, 1), pi = __shfl_up_sync(0xffffffffu, li, 1);
                    if (lane < 8) {
                        if (lane > pos) {
                            ld = pd;
                            li = pi;
                        } else if (lane == pos) {
                            ld = nd;
                            li = ni;
                        }
                    }
                    thr = min(lim, __shfl_sync(0xffffffffu, ld, 7));
                }
            }
        }
        __syncthreads();
    }
    if (active && lane < 8) A.best8[(size_t)qi * 8 + lane] = make_int2(ld, li);
}

// Nearest grid point of row y by (distance, x), constrained by sigma, found by
// one warp: lane l scans grid columns l, l+32, ...; then a warp argmin.
__device__ __forceinline__ void warp_row_nearest(const RefFeat& r, const Plane& img, int w, int n, int gw, int y,
                                                 int xlim, int sigma, int lane, int& best_d, int& best_x) {
    int bd = 0x7fffffff, bx = 0x7fffffff;
    for (int g = lane; g < gw; g += 32) {
        const int x = g * n;
        if (sigma * (xlim - x) < 0) continue;
        const int d = ssd_at(r, img, pix(w, x, y));
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
    const int gw = A.gw;
    const int qi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qi >= A.gq) return;  // warp-uniform
    const int px = (qi % gw) * n, py = (qi / gw) * n;
    RefFeat r;
    load_ref(V.ref, pix(V.w, px, py), r);
    // the query's temporal top-8 (every lane the same, reads broadcast)
    int bd[8], bi[8];
    const int2* src = A.best8 + (size_t)qi * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int2 e = src[k];
        bd[k] = e.x;
        bi[k] = e.y;
    }
    int ds, sx;
    warp_row_nearest(r, V.ste, V.w, n, gw, py, px, V.sigma, lane, ds, sx);
    int best_c = 0x7fffffff;
    Vec4 best = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k >= knn || bd[k] == 0x7fffffff) break;
        const int tx = (bi[k] % gw) * n, ty = (bi[k] / gw) * n;
        int dxc, cx;
        warp_row_nearest(r, V.crs, V.w, n, gw, ty, tx, V.sigma, lane, dxc, cx);
        const int c = bd[k] + ds + dxc;
        if (c < best_c) {
            best_c = c;
            best.u = tx - px;
            best.v = ty - py;
            best.d0 = V.sigma * (px - sx);
            best.d1 = V.sigma * (tx - cx);
        }
    }
    if (lane == 0) {
        const size_t i = pix(V.w, px, py);
        A.field[i] = pack_vec(best);
        A.cost[i] = best_c;
    }
}

__global__ void k_inherit(const __grid_constant__ Fields F, int n) {
    const Field& A = pick(F);
    const Views& V = A.V;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y;
    if (gx >= A.gw || gy >= A.gh) return;
    const int x = gx * n, y = gy * n;
    const size_t i = pix(V.w, x, y);
    const bool coarse = ((gx | gy) & 1) == 0;
    const int c = coarse ? A.cost[i] : kEmpty;
    if (c != kEmpty) {
        RefFeat r;
        load_ref(V.ref, i, r);
        const Vec4 a = unpack_vec(A.field[i]);
        A.cost[i] = cost_of(V, r, x, y, a.u, a.v, a.d0, a.d1);
    } else {
        A.cost[i] = kEmpty;
        A.field[i] = make_uint2(0u, 0u);
    }
}

struct HalfStep {
    int n, s, colour, dx, dy, prop, rs_before, rs_after;
};

// Pixels are processed by groups of L lanes (L = 1, 2 or 4, a tuning knob
// that never changes results).  Lane q of a group holds the 16-byte chunks j
// of a 48-byte record with j % L == q and, on lane 3 % L, the norm; every
// target record is loaded the same way, so with L = 4 one warp-wide load
// fetches eight whole records.  Partial sums |a|^2 + |b|^2 - 2 a.b of the
// three views are combined with log2(L) shuffles inside the group.
template <int L>
struct Slice {
    static constexpr int kChunks = (3 + L - 1) / L;
    int4 c[kChunks];
    int nrm;  // the norm on lane 3 % L, 0 on the others
};

template <int L>
__device__ __forceinline__ void load_slice(const Plane& P, size_t i, int q, Slice<L>& s) {
    const int4* p = reinterpret_cast<const int4*>(P.f + i * kFeat);
#pragma unroll
    for (int k = 0; k < Slice<L>::kChunks; ++k) {
        const int j = q + k * L;
        s.c[k] = j < 3 ? __ldg(p + j) : make_int4(0, 0, 0, 0);
    }
    s.nrm = q == 3 % L ? __ldg(P.nrm + i) : 0;
}

template <int L>
__device__ __forceinline__ int slice_part(const Slice<L>& a, const Plane& P, size_t i, int q) {
    Slice<L> t;
    load_slice<L>(P, i, q, t);
    int d = 0;
#pragma unroll
    for (int k = 0; k < Slice<L>::kChunks; ++k) {
        d = __dp4a(a.c[k].x, t.c[k].x, d);
        d = __dp4a(a.c[k].y, t.c[k].y, d);
        d = __dp4a(a.c[k].z, t.c[k].z, d);
        d = __dp4a(a.c[k].w, t.c[k].w, d);
    }
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

// One half-step of one pixel with own state (cur, c) and predecessor states
// (va, ca), (vb, cb) (ca/cb = kEmpty when absent).  The costs of the
// candidates that do not depend on each other -- the random-search candidate
// that precedes the propagation (colour 0) and the two predecessors -- are
// evaluated with all their loads in flight together; the
// strict-less-than comparisons then run in the order random search,
// horizontal, vertical, exactly as if evaluated one after the other.  The
// random search that follows the propagation (colour 1) depends on its
// result and comes last.  rs_before / rs_after < 0: no search.
template <int L>
__device__ __forceinline__ bool update_pixel(const Views& V, const Slice<L>& a, int q, unsigned gmask, int n, int s,
                                             uint2 key, int mirror, int x, int y, uint32_t pixel, int rs_before,
                                             int rs_after, const Vec4& va, int ca, const Vec4& vb, int cb, Vec4& cur,
                                             int& c) {
    bool changed = false;
    Vec4 cr;
    const bool do_rs = rs_before >= 0 && c != kEmpty && rs_candidate(n, s, key, mirror, rs_before, pixel, cur, cr);
    // A predecessor holding the pixel's own vector, or the same vector as the
    // other predecessor, has exactly that candidate's cost and can never be
    // strictly lower: it is not evaluated (the result is unchanged).
    const bool own_valid = c != kEmpty;
    const bool do_a = ca != kEmpty && !(own_valid && same_vec(va, cur));
    const bool do_b = cb != kEmpty && !(own_valid && same_vec(vb, cur)) && !(ca != kEmpty && same_vec(vb, va));
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

constexpr int kHalfLanes = 4;
constexpr int kHalfThreads = 256;
constexpr int kHalfPixels = kHalfThreads / kHalfLanes;

// One colour of the checkerboard over the whole grid, in place.  Used for
// the random search of colour 0 after the last iteration of a scale.
__global__ void __launch_bounds__(kHalfThreads) k_half_step(const __grid_constant__ Fields F, HalfStep H) {
    constexpr int L = kHalfLanes;
    const Field& A = pick(F);
    const Views& V = A.V;
    const int q = threadIdx.x & (L - 1);
    const unsigned gmask = group_mask<L>();
    const int gy = blockIdx.y;
    const int gx = 2 * (blockIdx.x * kHalfPixels + (int)(threadIdx.x / L)) + ((H.colour + gy) & 1);
    if (gx >= A.gw || gy >= A.gh) return;  // the whole group leaves together
    const int x = gx * H.n, y = gy * H.n;
    const size_t i = pix(V.w, x, y);
    const int ax = x - H.dx * H.n, by = y - H.dy * H.n;
    const bool has_a = H.prop && ax >= 0 && ax < V.w;
    const bool has_b = H.prop && by >= 0 && by < V.h;
    const size_t ja = has_a ? pix(V.w, ax, y) : i, jb = has_b ? pix(V.w, x, by) : i;
    int c = A.cost[i];
    const uint2 wc = A.field[i];
    const int ca = has_a ? A.cost[ja] : kEmpty, cb = has_b ? A.cost[jb] : kEmpty;
    const uint2 wa = A.field[ja], wb = A.field[jb];
    if (!H.prop && c == kEmpty) return;
    Slice<L> a;
    load_slice<L>(V.ref, i, q, a);
    Vec4 cur = unpack_vec(wc);
    if (update_pixel<L>(V, a, q, gmask, H.n, H.s, A.key, A.mirror, x, y, (uint32_t)i, H.rs_before, H.rs_after,
                        unpack_vec(wa), ca, unpack_vec(wb), cb, cur, c) &&
        q == 0) {
        A.field[i] = pack_vec(cur);
        A.cost[i] = c;
    }
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
};

template <int L, int TX, int TY>
__global__ void __launch_bounds__(iter_threads<L, TX, TY>()) k_iteration(const __grid_constant__ Fields F, IterStep H) {
    constexpr int kRegX = TX + 1, kRegY = TY + 1;
    constexpr int kGroups = iter_threads<L, TX, TY>() / L;
    __shared__ uint2 s_vec[kRegX * kRegY];
    __shared__ int s_cost[kRegX * kRegY];
    const Field& A = pick(F);
    const Views& V = A.V;
    const int q = threadIdx.x & (L - 1);
    const unsigned gmask = group_mask<L>();
    const int grp = threadIdx.x / L;
    const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * TY;
    const int gw = A.gw, gh = A.gh;
    if (tx0 >= gw || ty0 >= gh) return;  // tile beyond this field's grid (whole CTA)
    const int rx0 = tx0 - (H.dx > 0 ? 1 : 0), ry0 = ty0 - (H.dy > 0 ? 1 : 0);  // region origin
    const int n = H.n;

    // phase 1: colour-0 pixels of the region (tile + halo)
    constexpr int kHalfRow = (kRegX + 1) / 2;
    for (int k = grp; k < kHalfRow * kRegY; k += kGroups) {
        const int ry = k / kHalfRow;
        const int rx = 2 * (k % kHalfRow) + ((rx0 + ry0 + ry) & 1);
        const int gx = rx0 + rx, gy = ry0 + ry;
        if (rx >= kRegX || gx < 0 || gx >= gw || gy < 0 || gy >= gh) continue;
        const int x = gx * n, y = gy * n;
        const size_t i = pix(V.w, x, y);
        const int ax = x - H.dx * n, by = y - H.dy * n;
        const bool has_a = ax >= 0 && ax < V.w, has_b = by >= 0 && by < V.h;
        const size_t ja = has_a ? pix(V.w, ax, y) : i, jb = has_b ? pix(V.w, x, by) : i;
        int c = A.cost[i];
        const uint2 wc = A.field[i];
        const int ca = has_a ? A.cost[ja] : kEmpty, cb = has_b ? A.cost[jb] : kEmpty;
        const uint2 wa = A.field[ja], wb = A.field[jb];
        Slice<L> a;
        load_slice<L>(V.ref, i, q, a);
        Vec4 cur = unpack_vec(wc);
        update_pixel<L>(V, a, q, gmask, n, H.s, A.key, A.mirror, x, y, (uint32_t)i, H.it - 1, -1, unpack_vec(wa), ca,
                        unpack_vec(wb), cb, cur, c);
        if (q == 0) {
            const uint2 wv = pack_vec(cur);
            s_vec[ry * kRegX + rx] = wv;
            s_cost[ry * kRegX + rx] = c;
            if (gx >= tx0 && gx < tx0 + TX && gy >= ty0 && gy < ty0 + TY) {
                A.field_out[i] = wv;
                A.cost_out[i] = c;
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
        int c = A.cost[i];
        Vec4 cur = unpack_vec(A.field[i]);
        Slice<L> a;
        load_slice<L>(V.ref, i, q, a);
        const int agx = gx - H.dx, bgy = gy - H.dy;  // predecessors (colour 0, in the region)
        int ca = kEmpty, cb = kEmpty;
        uint2 wa = make_uint2(0u, 0u), wb = make_uint2(0u, 0u);
        if (agx >= 0 && agx < gw) {
            const int r = (gy - ry0) * kRegX + (agx - rx0);
            ca = s_cost[r];
            wa = s_vec[r];
        }
        if (bgy >= 0 && bgy < gh) {
            const int r = (bgy - ry0) * kRegX + (gx - rx0);
            cb = s_cost[r];
            wb = s_vec[r];
        }
        update_pixel<L>(V, a, q, gmask, n, H.s, A.key, A.mirror, x, y, (uint32_t)i, -1, H.it, unpack_vec(wa), ca,
                        unpack_vec(wb), cb, cur, c);
        if (q == 0) {
            A.field_out[i] = pack_vec(cur);
            A.cost_out[i] = c;
        }
    }
}

// Instantiated (lanes per pixel, tile) variants; any of them gives identical
// results.
using IterKernel = void (*)(Fields, IterStep);
struct IterVariant {
    int lanes, tx, ty;
    IterKernel k;
    int threads;
};
#define SFF_ITER_V(L, X, Y) {L, X, Y, k_iteration<L, X, Y>, iter_threads<L, X, Y>()}
#define SFF_ITER_VARIANTS(L)                                                                        \
    SFF_ITER_V(L, 64, 16), SFF_ITER_V(L, 32, 16), SFF_ITER_V(L, 64, 8), SFF_ITER_V(L, 32, 8), \
        SFF_ITER_V(L, 16, 8), SFF_ITER_V(L, 8, 8)
const IterVariant kIterVariants[] = {SFF_ITER_VARIANTS(1), SFF_ITER_VARIANTS(2), SFF_ITER_VARIANTS(4)};
#undef SFF_ITER_VARIANTS
#undef SFF_ITER_V

const IterVariant* find_variant(const sff_tuning& t) {
    for (const auto& v : kIterVariants)
        if (v.lanes == t.lanes_per_pixel && v.tx == t.tile_x && v.ty == t.tile_y) return &v;
    return nullptr;
}

// Tile of the iteration kernel at one scale: the tuned tile at scale 0; at
// coarser scales the tuned tile if it gives at least two CTAs per SM over
// all fields, else the largest smaller tile (same lanes per pixel) that
// does, else the smallest.  Any tile gives the same result.
long ctas_for(const IterVariant& v, const int* gw, const int* gh, int nf) {
    long c = 0;
    for (int k = 0; k < nf; ++k) c += (long)((gw[k] + v.tx - 1) / v.tx) * ((gh[k] + v.ty - 1) / v.ty);
    return c;
}

const IterVariant* tile_for_grid(const IterVariant* tuned, int s, const int* gw, const int* gh, int nf) {
    if (s == 0) return tuned;
    constexpr long kWantCtas = 2 * 152;
    const IterVariant* pick_v = nullptr;
    for (const auto& v : kIterVariants) {
        if (v.lanes != tuned->lanes || v.tx * v.ty > tuned->tx * tuned->ty) continue;
        if (ctas_for(v, gw, gh, nf) >= kWantCtas && (!pick_v || v.tx * v.ty > pick_v->tx * pick_v->ty)) pick_v = &v;
    }
    if (pick_v) return (tuned->tx * tuned->ty == pick_v->tx * pick_v->ty) ? tuned : pick_v;
    for (const auto& v : kIterVariants)  // none fills the GPU: the smallest tile
        if (v.lanes == tuned->lanes && (!pick_v || v.tx * v.ty < pick_v->tx * pick_v->ty)) pick_v = &v;
    return pick_v;
}

int coarse_gq(int w, int h, const sff_params& p) {
    const int n = 1 << (p.num_scales - 1);
    return ((w + n - 1) / n) * ((h + n - 1) / n);
}

// Scratch of one field: K-NN lists and compact coarsest-grid records, then a
// second state buffer (field + cost) for the double-buffered iterations.
// Compact rows are padded to a multiple of 4 records plus 4, so every bulk
// copy (whole groups of 4 records) starts and ends on 16 bytes.
int gq_padded(int gq) { return ((gq + 3) & ~3) + 4; }
struct FieldScratch {
    size_t best8, cf, cn, bound, field, cost, total;
};
FieldScratch field_scratch(int w, int h, const sff_params& p) {
    const int gq = coarse_gq(w, h, p), gp = gq_padded(gq);
    FieldScratch f;
    f.best8 = 0;
    f.cf = f.best8 + align256((size_t)gq * 8 * sizeof(int2));
    f.cn = f.cf + align256((size_t)2 * gp * kFeat);
    f.bound = f.cn + align256((size_t)2 * gp * sizeof(int));
    f.field = f.bound + align256((size_t)gq * sizeof(int));
    f.cost = f.field + align256((size_t)w * h * 8);
    f.total = f.cost + align256((size_t)w * h * 4);
    return f;
}

}  // namespace

size_t field_ws_bytes(int w, int h, const sff_params& p) { return field_scratch(w, h, p).total; }

// Workspace of sff_match_views / sff_match_quad: the scratch of two fields.
size_t match_ws_bytes(int w, int h, const sff_params& p) { return 2 * field_ws_bytes(w, h, p); }

// The stage of Sec. 3.1 for nf <= kMaxFields fields (any sizes) sharing the
// launches.  spec[k].workspace holds field_ws_bytes() of scratch.
int run_fields(const FieldSpec* spec, int nf, const sff_params& P, const sff_tuning& T, cudaStream_t st) {
    const IterVariant* var = find_variant(T);
    if (!var || nf < 1 || nf > kMaxFields) return SFF_ERR_ARG;
    const int S = P.num_scales, I = P.iterations;
    static const int kDirs[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    static Fields F;  // host staging of the kernel parameter (copied at each launch)
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
        F.f[k].cf = reinterpret_cast<uint8_t*>(ws + sc.cf);
        F.f[k].cn = reinterpret_cast<int*>(ws + sc.cn);
        F.f[k].bound = reinterpret_cast<int*>(ws + sc.bound);
        F.f[k].gq = coarse_gq(fs.width, fs.height, P);
        F.f[k].gq_pad = gq_padded(F.f[k].gq);
        F.f[k].mirror = fs.mirror;
        F.f[k].key = make_uint2((uint32_t)fs.seed, (uint32_t)(fs.seed >> 32));
        U[k] = reinterpret_cast<uint2*>(fs.field);
        Uc[k] = fs.cost;
        Tf[k] = reinterpret_cast<uint2*>(ws + sc.field);
        Tc[k] = reinterpret_cast<int*>(ws + sc.cost);
    }
    for (int s = S - 1; s >= 0; --s) {
        const int n = 1 << s;
        int mgw = 0, mgh = 0, mgq = 0;
        for (int k = 0; k < nf; ++k) {
            const FieldSpec& fs = spec[k];
            const int w = fs.width, h = fs.height;
            F.f[k].V = Views{plane_of(fs.ref, s, S, w, h), plane_of(fs.tmp, s, S, w, h), plane_of(fs.ste, s, S, w, h),
                             plane_of(fs.crs, s, S, w, h), w, h, fs.mirror ? -1 : 1};
            F.f[k].field = F.f[k].field_out = U[k];
            F.f[k].cost = F.f[k].cost_out = Uc[k];
            gw[k] = F.f[k].gw = (w + n - 1) / n;
            gh[k] = F.f[k].gh = (h + n - 1) / n;
            mgw = std::max(mgw, gw[k]);
            mgh = std::max(mgh, gh[k]);
            mgq = std::max(mgq, F.f[k].gq);
        }
        if (s == S - 1) {
            dim3 g0((mgq * 4 + 255) / 256, 2, nf);
            SFF_LAUNCH(k_gather_grid, g0, 256, 0, st, F, n);
            dim3 gb((mgq + 7) / 8, 1, nf);
            SFF_LAUNCH(k_knn_bound, gb, 256, 0, st, F, n);
            dim3 g1((mgq + kKnnWarps - 1) / kKnnWarps, 1, nf);
            SFF_LAUNCH(k_knn, g1, kKnnThreads, 0, st, F);
            dim3 g2((mgq + 7) / 8, 1, nf);
            SFF_LAUNCH(k_init_select, g2, 256, 0, st, F, n, P.knn_temporal);
        } else {
            dim3 g((mgw + 127) / 128, mgh, nf);
            SFF_LAUNCH(k_inherit, g, 128, 0, st, F, n);
        }
        // iterations alternate between the caller's buffers (U) and the
        // workspace buffers (T); with an odd count U is first copied to T so
        // that the last iteration writes U
        if (I & 1)
            for (int k = 0; k < nf; ++k) {
                const size_t np = (size_t)spec[k].width * spec[k].height;
                cudaMemcpyAsync(Tf[k], U[k], np * 8, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(Tc[k], Uc[k], np * 4, cudaMemcpyDeviceToDevice, st);
            }
        const IterVariant* sv = tile_for_grid(var, s, gw, gh, nf);
        dim3 gi((mgw + sv->tx - 1) / sv->tx, (mgh + sv->ty - 1) / sv->ty, nf);
        for (int it = 0; it < I; ++it) {
            const bool from_user = ((I - it) & 1) == 0;  // the last iteration reads T and writes U
            for (int k = 0; k < nf; ++k) {
                F.f[k].field = from_user ? U[k] : Tf[k];
                F.f[k].cost = from_user ? Uc[k] : Tc[k];
                F.f[k].field_out = from_user ? Tf[k] : U[k];
                F.f[k].cost_out = from_user ? Tc[k] : Uc[k];
            }
            IterStep H{n, s, kDirs[it % 4][0], kDirs[it % 4][1], it};
            if (::sff::profiling()) ::sff::profile_mark("k_iteration", st, false);
            sv->k<<<gi, sv->threads, 0, st>>>(F, H);
            if (::sff::profiling()) ::sff::profile_mark("k_iteration", st, true);
        }
        for (int k = 0; k < nf; ++k) {
            F.f[k].field = F.f[k].field_out = U[k];
            F.f[k].cost = F.f[k].cost_out = Uc[k];
        }
        if (I > 0) {
            const int half_w = (mgw + 1) / 2;
            dim3 g((half_w + kHalfPixels - 1) / kHalfPixels, mgh, nf);
            HalfStep H{n, s, 0, 0, 0, 0, I - 1, -1};
            SFF_LAUNCH(k_half_step, g, kHalfThreads, 0, st, F, H);
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
    return run_fields(&f, 1, *params, t, (cudaStream_t)stream);
}

extern "C" int sff_default_tuning(sff_tuning* out) {
    if (!out) return SFF_ERR_ARG;
    out->lanes_per_pixel = 1;
    out->tile_x = 32;
    out->tile_y = 16;
    return SFF_OK;
}

extern "C" int sff_tuning_supported(const sff_tuning* t) {
    return t && sff::find_variant(*t) ? 1 : 0;
}

extern "C" int sff_match_quad_tuned(const uint8_t* pyr_l0_dev, const uint8_t* pyr_r0_dev, const uint8_t* pyr_l1_dev,
                                    const uint8_t* pyr_r1_dev, int32_t width, int32_t height, uint64_t seed,
                                    const sff_params* params, const sff_tuning* tuning, int16_t* fwd_dev,
                                    int32_t* fwd_cost_dev, int16_t* inv_dev, int32_t* inv_cost_dev, void* workspace,
                                    size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!tuning || !find_variant(*tuning)) return SFF_ERR_ARG;
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
    return run_fields(f, 2, *params, *tuning, (cudaStream_t)stream);
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

extern "C" int sff_device_timeouts(uint32_t* out, int32_t reset) {
    if (!out) return SFF_ERR_ARG;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, sff::g_wait_timeouts, sizeof v) != cudaSuccess) return SFF_ERR_CUDA;
    *out = v;
    if (reset) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(sff::g_wait_timeouts, &z, sizeof z) != cudaSuccess) return SFF_ERR_CUDA;
    }
    return SFF_OK;
}
