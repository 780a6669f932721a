// Dense interpolation of the seeds (Sec. 3.2, "Interpolation Models" and
// "Edge-Aware Neighborhood"), with Euclidean distances in place of the
// geodesic ones (the trained boundary detector is not part of this stage).
//
// Every seed gets two local models, fitted by weighted least squares over
// its nearest seeds (weights exp(-alpha D / dist_unit), D the pixel
// distance):
//   a plane of the disparity d0 over the k_geo nearest seeds, in
//   coordinates centred at the seed;
//   an affine map x1 = A (x0 - c) + t of triangulated 3D points over the
//   k_motion nearest seeds with d0, d1 >= 1, c the weighted centroid.
// The linear parts get a ridge of 1e-9 * trace / dimension towards a flat
// plane and A = I.  Every pixel takes the models of its closest seed and
// evaluates them at its own position (d0, then reproject, transform,
// project back).  Ties in all distance orders go to the lower seed index.
//
// GB300 has little double-precision throughput, and the fits run in double
// precision, so the design spends double-precision instructions only on
// the sums and the solves:
//   - the seeds of sff_emit_seeds hold at most one seed per 3x3 block
//     (anchored at (0, 0)); a block map whose words pack the seed index, the
//     motion flag and the offset inside the block gives exact nearest-seed
//     searches by rings of blocks (ring r is at least 3r - 2 px away) with
//     no seed loads;
//   - the weight depends on the integer squared distance only: a table of
//     exp(-alpha sqrt(d2) / dist_unit) for d2 < 65536, the same expression
//     as inline, serves every fit;
//   - each seed's 3D points x0, x1 are triangulated once;
//   - the neighbourhoods are selected by counting (the k-th smallest
//     (d2, index) key by bisection), not by sorting;
//   - the selected neighbours are compacted into lists, so that the sums
//     run over them alone with every lane busy;
//   - the warp sums are a reduce-scatter (N - 1 additions for N values
//     instead of 5 N), and the plane and the three rows of the affine map
//     are solved by four lanes at once.
//
// k_interp_clear:  empty map, status, weight table.
// k_interp_prep:   map words and triangulated points of every seed.
// k_interp_models: one warp per seed: one pass over rings of blocks collects
//                  the candidates of both neighbourhoods, bisection selects
//                  them, the normal equations accumulate in double precision.
// k_interp_columns: per pixel column the closest seed in that column, for
//                  every row (a sweep down and up the block map).
// k_interp_pixels: per pixel the closest seed over the columns of its row,
//                  then its models evaluated in double precision.
#include "sff_internal.cuh"

namespace sff {
namespace {

constexpr int kBlock = 3;            // sparsification block of Sec. 3.2
constexpr int kModelWarps = 2;       // warps (seeds) per CTA of k_interp_models
constexpr int kMaxK = 1024;          // largest k_geo / k_motion
constexpr int kRegKeys = 16;         // candidate keys per lane held in registers during selection

// Candidate slots per seed: the rings up to the bound of the k-th nearest
// hold about 4/pi times k seeds plus a margin of whole rings; 6 k + 256
// leaves room for uneven seed density (with k = 160, a lone seed in the
// middle of a 480 x 480 px hole in a dense seed lattice takes 833).
__host__ __device__ __forceinline__ int candidate_slots(int kg, int km) {
    return ((6 * (kg > km ? kg : km) + 256) + 31) & ~31;
}
constexpr int kModelDoubles = 18;    // plane 3, [A | t] 12, centre 3
constexpr int kPointDoubles = 8;     // x0 3, x1 3, d0, pad
constexpr int kSumDoubles = 32;      // plane sums 9, motion N 10 and R 12, pad
constexpr int kWeightTable = 1 << 16;
constexpr unsigned kErrSeed = 1u, kErrOverflow = 2u;
constexpr unsigned kFull = 0xffffffffu;

// Map word of a block: (seed index << 5) | (motion << 4) | (ox << 2) | oy,
// (ox, oy) the seed's offset inside its block; -1 for an empty block.
__device__ __forceinline__ int word_index(int w) { return w >> 5; }
__device__ __forceinline__ bool word_motion(int w) { return (w >> 4) & 1; }

struct InterpJob {
    const sff_seed* seeds;
    const int32_t* count;
    int capacity, w, h, gbw, gbh;
    int* map;          // [gbh][gbw] words
    double* pts;       // [capacity][kPointDoubles]
    double* wt;        // [kWeightTable]
    double* models;    // [capacity][kModelDoubles]
    double* sums;      // [capacity][kSumDoubles] normal equations
    int* motion;       // [capacity] motion neighbours
    unsigned* status;  // error bits
    sff_interp_params p;
    double fb, inv_f;  // focal * baseline, 1 / focal
    int slots;         // candidate slots per warp of k_interp_models
};

__device__ __forceinline__ int seed_count(const InterpJob& J) { return min(*J.count, J.capacity); }

__device__ __forceinline__ double weight_of(const InterpJob& J, unsigned d2) {
    return d2 < (unsigned)kWeightTable ? J.wt[d2] : exp(-J.p.alpha * sqrt((double)d2) / J.p.dist_unit);
}

__global__ void k_interp_clear(InterpJob J) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < J.gbw * J.gbh) J.map[i] = -1;
    if (i < kWeightTable) J.wt[i] = exp(-J.p.alpha * sqrt((double)i) / J.p.dist_unit);
    if (i == 0) *J.status = 0u;
}

// Pinhole triangulation: Z = f B / d, X = (x - cx) Z / f, Y = (y - cy) Z / f.
__device__ __forceinline__ void triangulate(const InterpJob& J, double x, double y, double d, double* X) {
    const double Z = J.fb / d;
    X[0] = (x - J.p.cx) * Z / J.p.focal;
    X[1] = (y - J.p.cy) * Z / J.p.focal;
    X[2] = Z;
}

__global__ void k_interp_prep(InterpJob J) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= seed_count(J)) return;
    const sff_seed s = J.seeds[i];
    const bool motion = s.d0 >= 1 && s.d1 >= 1;
    // an index past the number of blocks implies a duplicate or an outside seed
    const bool inside = s.x >= 0 && s.y >= 0 && s.x < J.w && s.y < J.h && i < J.gbw * J.gbh;
    if (inside) {
        const int word = (i << 5) | ((int)motion << 4) | ((s.x % kBlock) << 2) | (s.y % kBlock);
        if (atomicCAS(J.map + (s.y / kBlock) * J.gbw + s.x / kBlock, -1, word) != -1) atomicOr(J.status, kErrSeed);
    } else {
        atomicOr(J.status, kErrSeed);
    }
    double X[kPointDoubles] = {0, 0, 0, 0, 0, 0, (double)s.d0, 0};
    if (motion) {
        triangulate(J, s.x, s.y, s.d0, X);
        triangulate(J, s.x + s.u, s.y + s.v, s.d1, X + 3);
    }
    double2* o = reinterpret_cast<double2*>(J.pts + (size_t)i * kPointDoubles);
#pragma unroll
    for (int k = 0; k < kPointDoubles / 2; ++k) o[k] = make_double2(X[2 * k], X[2 * k + 1]);
}

// Cell k of the Chebyshev ring r around a block: offsets (ox, oy).
__device__ __forceinline__ void ring_cell(int r, int k, int& ox, int& oy) {
    const int side = 2 * r + 1;
    if (r == 0) {
        ox = oy = 0;
    } else if (k < side) {  // top row
        ox = k - r;
        oy = -r;
    } else if (k < 2 * side) {  // bottom row
        ox = k - side - r;
        oy = r;
    } else {  // the two columns without their corners
        const int m = k - 2 * side;
        ox = (m & 1) ? r : -r;
        oy = (m >> 1) - r + 1;
    }
}

__device__ __forceinline__ int ring_cells(int r) { return r == 0 ? 1 : 8 * r; }

// Sums v[0 .. N) over the warp by recursive halving: on return lane l holds
// in v[0] the total of value l >> (5 - log2 N).
template <int N>
__device__ __forceinline__ void reduce_scatter(double (&v)[N], int lane) {
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "power of two up to 32");
#pragma unroll
    for (int h = N / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? v[i] : v[i + h];
            const double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    constexpr int kLog = N >= 32 ? 5 : N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : N >= 2 ? 1 : 0;
#pragma unroll
    for (int o = 16 >> kLog; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(kFull, v[0], o);
}

struct Candidates {
    const uint32_t* pos;  // (dy << 16) | (dx & 0xffff), offsets from the seed
    const int* word;
    int m;
};

__device__ __forceinline__ unsigned cand_d2(uint32_t p, int& dx, int& dy) {
    dx = (int)(int16_t)(p & 0xffffu);
    dy = (int)(int16_t)(p >> 16);
    return (unsigned)(dx * dx + dy * dy);
}

struct Threshold {
    unsigned D;  // a member has d2 < D, or d2 == D and index <= I
    int I;
};

// Warp sum of an int.
__device__ __forceinline__ int warp_sum_i(int c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    return c;
}

// The index threshold among the candidates tied at distance D: the need-th
// smallest index of the set's members with d2 == D (need < number tied).
// Up to 32 tied members are ranked in registers; more fall back to
// bisection over the index.
__device__ int tie_threshold(const Candidates& C, bool motion, unsigned D, int need, int tied, int n, int* scratch,
                             int lane) {
    if (tied <= 32) {
        int filled = 0;
        for (int base = 0; base < C.m; base += 32) {
            const int j = base + lane;
            bool t = false;
            int idx = 0;
            if (j < C.m) {
                const int w = C.word[j];
                int dx, dy;
                t = (!motion || word_motion(w)) && cand_d2(C.pos[j], dx, dy) == D;
                idx = word_index(w);
            }
            const unsigned bt = __ballot_sync(kFull, t);
            if (t) scratch[filled + __popc(bt & ((1u << lane) - 1u))] = idx;
            filled += __popc(bt);
        }
        __syncwarp();
        const int v = lane < tied ? scratch[lane] : 0x7fffffff;
        int rank = 0;
        for (int u = 0; u < tied; ++u) rank += __shfl_sync(kFull, v, u) < v;
        __syncwarp();
        const unsigned hit = __ballot_sync(kFull, lane < tied && rank == need - 1);
        return __shfl_sync(kFull, v, __ffs(hit) - 1);
    }
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        int c = 0;
        for (int j = lane; j < C.m; j += 32) {
            const int w = C.word[j];
            int dx, dy;
            c += (!motion || word_motion(w)) && cand_d2(C.pos[j], dx, dy) == D && word_index(w) <= mid;
        }
        if (warp_sum_i(c) >= need)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// The k-th smallest d2 of both neighbourhoods, all candidates (k_geo) and
// the motion seeds among them (k_motion), by bisections that share their
// passes over the candidates: the smallest D with at least k members
// within D.  hiA / hiM are distances that at least k members are within
// (0 skips that set).  each(f) calls f(d2, motion) for every candidate of
// the lane.
template <class Each>
__device__ void bisect_both(Each each, int kg, int km, unsigned hiA, unsigned hiM, unsigned& DA, unsigned& DM) {
    unsigned loA = 0, loM = 0;
    while (loA < hiA || loM < hiM) {
        const unsigned midA = loA + ((hiA - loA) >> 1), midM = loM + ((hiM - loM) >> 1);
        int ca = 0, cm = 0;
        each([&](unsigned d2, unsigned mot) {
            ca += d2 <= midA;
            cm += mot & (d2 <= midM);
        });
        ca = warp_sum_i(ca);
        cm = warp_sum_i(cm);
        if (loA < hiA) {
            if (ca >= kg)
                hiA = midA;
            else
                loA = midA + 1;
        }
        if (loM < hiM) {
            if (cm >= km)
                hiM = midM;
            else
                loM = midM + 1;
        }
    }
    DA = loA;
    DM = loM;
}

// Runs f(each) with each(g) calling g(d2, motion) for the lane's candidates:
// from keys held in registers when the candidates fit (bit 31 = motion; the
// filler 0x7fffffff is farther than any bound), else from shared memory.
template <class F>
__device__ __forceinline__ void with_keys(const Candidates& C, int lane, F f) {
    if (C.m <= 32 * kRegKeys) {
        unsigned key[kRegKeys];
#pragma unroll
        for (int t = 0; t < kRegKeys; ++t) {
            const int j = lane + 32 * t;
            key[t] = 0x7fffffffu;
            if (j < C.m) {
                int dx, dy;
                key[t] = cand_d2(C.pos[j], dx, dy) | ((unsigned)word_motion(C.word[j]) << 31);
            }
        }
        f([&](auto g) {
#pragma unroll
            for (int t = 0; t < kRegKeys; ++t) g(key[t] & 0x7fffffffu, key[t] >> 31);
        });
    } else {
        f([&](auto g) {
            for (int j = lane; j < C.m; j += 32) {
                int dx, dy;
                g(cand_d2(C.pos[j], dx, dy), (unsigned)word_motion(C.word[j]));
            }
        });
    }
}

// The k-th smallest distances DA, DM of both sets (hiA / hiM: bounds that
// at least k members are within; 0 skips a set) and the counts of members
// below and at them (warp-reduced).  One routine serves the tightening of
// the ring bound and the final selection, so that its code exists once.
__device__ __noinline__ void kth_and_counts(const Candidates& C, int kg, int km, unsigned hiA, unsigned hiM,
                                            int lane, unsigned& DA, unsigned& DM, int (&cnt)[4]) {
    int ba = 0, ea = 0, bm = 0, em = 0;
    with_keys(C, lane, [&](auto each) {
        bisect_both(each, kg, km, hiA, hiM, DA, DM);
        each([&](unsigned d2, unsigned mot) {
            ba += d2 < DA;
            ea += d2 == DA;
            bm += mot & (d2 < DM);
            em += mot & (d2 == DM);
        });
    });
    cnt[0] = warp_sum_i(ba);
    cnt[1] = warp_sum_i(ea);
    cnt[2] = warp_sum_i(bm);
    cnt[3] = warp_sum_i(em);
}

// Thresholds of the k smallest (d2, index) keys of both neighbourhoods.
// `fa`/`fm` are the sizes of the two sets, `far_a`/`far_m` distances that
// at least k of their members are within.
__device__ void select_both(const Candidates& C, int kg, int km, int fa, int fm, unsigned far_a, unsigned far_m,
                            int n, int* scratch, int lane, Threshold& A, Threshold& M) {
    A = Threshold{0xffffffffu, 0x7fffffff};
    M = Threshold{0xffffffffu, 0x7fffffff};
    const bool sa = fa > kg, sm = fm > km;
    if (!sa && !sm) return;
    unsigned DA, DM;
    int cnt[4];
    kth_and_counts(C, kg, km, sa ? far_a : 0, sm ? far_m : 0, lane, DA, DM, cnt);
    if (sa) {
        A.D = DA;
        if (kg - cnt[0] < cnt[1]) A.I = tie_threshold(C, false, DA, kg - cnt[0], cnt[1], n, scratch, lane);
    }
    if (sm) {
        M.D = DM;
        if (km - cnt[2] < cnt[3]) M.I = tie_threshold(C, true, DM, km - cnt[2], cnt[3], n, scratch, lane);
    }
}

__device__ __forceinline__ bool selected(unsigned d2, int idx, unsigned D, int I) {
    return d2 < D || (d2 == D && idx <= I);
}

// Cholesky solve of one 4x4 system per lane (upper triangle u[10] row by
// row, right-hand side b[4], solution into b); divisions by the diagonal
// are multiplications by its reciprocal.
__device__ __forceinline__ void solve4(const double (&u)[10], double (&b)[4]) {
    double L[4][4], inv[4];
    L[0][0] = u[0];
    L[1][0] = u[1];
    L[2][0] = u[2];
    L[3][0] = u[3];
    L[1][1] = u[4];
    L[2][1] = u[5];
    L[3][1] = u[6];
    L[2][2] = u[7];
    L[3][2] = u[8];
    L[3][3] = u[9];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double s = L[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        const double ljj = sqrt(s > 0.0 ? s : 1e-300);
        inv[j] = 1.0 / ljj;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            double t = L[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t * inv[j];
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * b[k];
        b[i] = t * inv[i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        double t = b[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) t -= L[k][i] * b[k];
        b[i] = t * inv[i];
    }
}

// Shared memory of one warp of k_interp_models: candidate positions and map
// words (J.slots each), the two neighbour lists (k_geo, k_motion slots of
// 16 bits), 32 ints of scratch.
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int slots, int kg, int km) {
    return (size_t)slots * 8 + (((size_t)(kg + km) * 2 + 15) & ~(size_t)15) + 128;
}

__global__ void __launch_bounds__(kModelWarps * 32) k_interp_models(InterpJob J) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int si = blockIdx.x * kModelWarps + wid;
    const int n = seed_count(J);
    if (si >= n) return;  // warp-uniform
    const int kg = J.p.k_geo, km = J.p.k_motion;
    unsigned char* mine = smem_raw + (size_t)wid * warp_smem_bytes(J.slots, kg, km);
    uint32_t* pos = reinterpret_cast<uint32_t*>(mine);
    int* word = reinterpret_cast<int*>(mine + (size_t)J.slots * 4);
    uint16_t* la = reinterpret_cast<uint16_t*>(mine + (size_t)J.slots * 8);
    uint16_t* lm = la + kg;
    int* scratch = reinterpret_cast<int*>(mine + warp_smem_bytes(J.slots, kg, km) - 128);
    const sff_seed s = J.seeds[si];
    const int bx = s.x / kBlock, by = s.y / kBlock;
    const int rmax = max(J.gbw, J.gbh);
    const unsigned lt = (1u << lane) - 1u;

    // Candidates by rings of blocks around the seed's block (ring q is at
    // least 3q - 2 px away).  First the rings until both neighbourhoods have
    // k members; a set's bound is the largest distance found when it got
    // them, and from then on a seed is kept only if it is within the bound
    // of a set it belongs to (so that sparse motion seeds do not drag every
    // seed in).  Then the k-th smallest distances of the candidates replace
    // the bounds, and the further rings that can still hold a member within
    // a bound are scanned.
    int fill = 0;                                          // candidates kept
    int fa = 0, fm = 0;                                    // ... of which motion seeds: fm
    unsigned far_a = 0, far_m = 0;                         // largest distance kept (all / motion)
    unsigned bound_a = 0xffffffffu, bound_m = 0xffffffffu;  // storage bounds, none yet
    // Compaction, when a batch would not fit the slots (motion seeds far
    // away behind many geometry-only seeds, e.g. the disparity fill's): the
    // k-th smallest distances of the candidates so far bound the final ones
    // from above (more candidates only lower them), so the candidates beyond
    // them are no members and are dropped, keeping the others in scan order.
    auto compact = [&]() {
        const Candidates Cc{pos, word, fill};
        unsigned DA = bound_a, DM = bound_m;
        if (fa >= kg || fm >= km) {
            int cnt[4];
            unsigned da, dm;
            kth_and_counts(Cc, kg, km, fa >= kg ? far_a : 0, fm >= km ? far_m : 0, lane, da, dm, cnt);
            if (fa >= kg) DA = min(DA, da);
            if (fm >= km) DM = min(DM, dm);
        }
        int kept = 0, kmot = 0;
        for (int base = 0; base < fill; base += 32) {
            const int j = base + lane;
            uint32_t pj = 0;
            int wj = -1;
            bool keep = false, mot = false;
            if (j < fill) {
                pj = pos[j];
                wj = word[j];
                int dx, dy;
                const unsigned d2 = cand_d2(pj, dx, dy);
                mot = word_motion(wj);
                keep = d2 <= DA || (mot && d2 <= DM);
            }
            const unsigned b = __ballot_sync(kFull, keep), bm = __ballot_sync(kFull, keep && mot);
            __syncwarp();  // the batch is read before any of it is overwritten
            if (keep) {
                const int slot = kept + __popc(b & lt);  // <= j
                pos[slot] = pj;
                word[slot] = wj;
            }
            __syncwarp();
            kept += __popc(b);
            kmot += __popc(bm);
        }
        fill = kept;
        fa = kept;
        fm = kmot;
        bound_a = DA;
        bound_m = DM;
    };
    auto scan = [&](int q) {
        unsigned ma = 0, mm = 0;
        for (int base = 0; base < ring_cells(q); base += 32) {
            const int k = base + lane;
            int w = -1, dx = 0, dy = 0;
            unsigned d2 = 0;
            if (k < ring_cells(q)) {
                int ox, oy;
                ring_cell(q, k, ox, oy);
                const int cx = bx + ox, cy = by + oy;
                if (cx >= 0 && cy >= 0 && cx < J.gbw && cy < J.gbh) w = J.map[cy * J.gbw + cx];
                if (w >= 0) {
                    dx = cx * kBlock + ((w >> 2) & 3) - s.x;
                    dy = cy * kBlock + (w & 3) - s.y;
                    d2 = (unsigned)(dx * dx + dy * dy);
                    if (!(d2 <= bound_a || (word_motion(w) && d2 <= bound_m))) w = -1;
                }
            }
            if (fill + __popc(__ballot_sync(kFull, w >= 0)) > J.slots) {
                compact();
                if (w >= 0 && !(d2 <= bound_a || (word_motion(w) && d2 <= bound_m))) w = -1;
            }
            const unsigned has = __ballot_sync(kFull, w >= 0), mot = __ballot_sync(kFull, w >= 0 && word_motion(w));
            if (w >= 0) {
                const int slot = fill + __popc(has & lt);
                if (slot < J.slots) {
                    pos[slot] = ((uint32_t)(dy & 0xffff) << 16) | (uint32_t)(dx & 0xffff);
                    word[slot] = w;
                }
                ma = max(ma, d2);
                if (word_motion(w)) mm = max(mm, d2);
            }
            fill += __popc(has);
            fa += __popc(has);
            fm += __popc(mot);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ma = max(ma, __shfl_xor_sync(kFull, ma, o));
            mm = max(mm, __shfl_xor_sync(kFull, mm, o));
        }
        far_a = max(far_a, ma);
        far_m = max(far_m, mm);
        if (bound_a == 0xffffffffu && fa >= kg) bound_a = far_a;
        if (bound_m == 0xffffffffu && fm >= km) bound_m = far_m;
    };
    int q = 0;
    for (; q <= rmax && (fa < kg || fm < km); ++q) scan(q);
    __syncwarp();
    if (fill > J.slots) {
        if (lane == 0) atomicOr(J.status, kErrOverflow);
        return;
    }
    if (fa >= kg && fm >= km) {
        const Candidates C1{pos, word, fill};
        int cnt[4];
        kth_and_counts(C1, kg, km, bound_a, bound_m, lane, bound_a, bound_m, cnt);
        for (; q <= rmax; ++q) {
            const long long b = 3 * q - 2;
            if (b * b > (long long)max(bound_a, bound_m)) break;
            scan(q);
        }
        __syncwarp();
    }
    const Candidates C{pos, word, fill};
    if (C.m > J.slots) {
        if (lane == 0) atomicOr(J.status, kErrOverflow);
        return;
    }
    Threshold TA, TM;
    select_both(C, kg, km, fa, fm, min(bound_a, far_a), min(bound_m, far_m), n, scratch, lane, TA, TM);

    // the members of both neighbourhoods, compacted into lists of slots
    int na = 0, nm = 0;
    for (int base = 0; base < C.m; base += 32) {
        const int j = base + lane;
        bool in_a = false, in_m = false;
        if (j < C.m) {
            const int w = C.word[j], idx = word_index(w);
            int dx, dy;
            const unsigned d2 = cand_d2(C.pos[j], dx, dy);
            in_a = selected(d2, idx, TA.D, TA.I);
            in_m = word_motion(w) && selected(d2, idx, TM.D, TM.I);
        }
        const unsigned ba = __ballot_sync(kFull, in_a), bm = __ballot_sync(kFull, in_m);
        const int qa = na + __popc(ba & lt), qm = nm + __popc(bm & lt);
        if (in_a && qa < kg) la[qa] = (uint16_t)j;
        if (in_m && qm < km) lm[qm] = (uint16_t)j;
        na += __popc(ba);
        nm += __popc(bm);
    }
    __syncwarp();
    if (na > kg || nm > km) {  // unreachable: at most k members are selected
        if (lane == 0) atomicOr(J.status, kErrOverflow);
        return;
    }

    // plane sums and the motion centroid: M00 M01 M02 M11 M12 M22 b0 b1 b2,
    // then W, W x0 (3)
    double g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.0;
    for (int t = lane; t < na; t += 32) {
        const int j = la[t];
        int dx, dy;
        const unsigned d2 = cand_d2(C.pos[j], dx, dy);
        const double wt = weight_of(J, d2);
        const double d = J.pts[(size_t)word_index(C.word[j]) * kPointDoubles + 6];
        const double r0 = dx, r1 = dy;
        const double w0 = wt * r0, w1 = wt * r1;
        g[0] += w0 * r0;
        g[1] += w0 * r1;
        g[2] += w0;
        g[3] += w1 * r1;
        g[4] += w1;
        g[5] += wt;
        g[6] += w0 * d;
        g[7] += w1 * d;
        g[8] += wt * d;
    }
    for (int t = lane; t < nm; t += 32) {
        const int j = lm[t];
        int dx, dy;
        const unsigned d2 = cand_d2(C.pos[j], dx, dy);
        const double wt = weight_of(J, d2);
        const double* X = J.pts + (size_t)word_index(C.word[j]) * kPointDoubles;
        g[9] += wt;
        g[10] += wt * X[0];
        g[11] += wt * X[1];
        g[12] += wt * X[2];
    }
    reduce_scatter(g, lane);  // value v on lanes 2v, 2v + 1
    double cen[3] = {0.0, 0.0, 0.0};
    {
        const double W = __shfl_sync(kFull, g[0], 18);
        const double c0 = __shfl_sync(kFull, g[0], 20), c1 = __shfl_sync(kFull, g[0], 22),
                     c2 = __shfl_sync(kFull, g[0], 24);
        if (nm > 0) {
            const double iw = 1.0 / W;
            cen[0] = c0 * iw;
            cen[1] = c1 * iw;
            cen[2] = c2 * iw;
        }
    }
    // centred motion sums: N (upper triangle of [r 1][r 1]^T, 10) and
    // R[j][a] = sum w r_a x1_j (12), r = x0 - c
    double a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = 0.0;
    for (int t = lane; t < nm; t += 32) {
        const int j = lm[t];
        int dx, dy;
        const unsigned d2 = cand_d2(C.pos[j], dx, dy);
        const double wt = weight_of(J, d2);
        const double* X = J.pts + (size_t)word_index(C.word[j]) * kPointDoubles;
        const double r[4] = {X[0] - cen[0], X[1] - cen[1], X[2] - cen[2], 1.0};
        const double wr[4] = {wt * r[0], wt * r[1], wt * r[2], wt};
        int e = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = p; q < 4; ++q) a[e++] += wr[p] * r[q];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
#pragma unroll
            for (int p = 0; p < 4; ++p) a[10 + jj * 4 + p] += wr[p] * X[3 + jj];
    }
    reduce_scatter(a, lane);  // value v on lane v

    // the sums go to k_interp_solve: plane sums first, then N and R
    double* sums = J.sums + (size_t)si * kSumDoubles;
    if (!(lane & 1) && lane < 18) sums[lane >> 1] = g[0];
    if (lane < 22) sums[9 + lane] = a[0];
    if (lane < 3) J.models[(size_t)si * kModelDoubles + 15 + lane] = lane == 0 ? cen[0] : lane == 1 ? cen[1] : cen[2];
    if (lane == 0) J.motion[si] = nm;
}

// The least-squares systems of every seed, one thread per system: the
// plane (a 3x3 system, padded to 4x4 with an identity row, which leaves its
// solution unchanged) and the three rows of [A | t] (4x4 each, one matrix).
__global__ void k_interp_solve(InterpJob J) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int si = t >> 2, row = t & 3;
    if (si >= seed_count(J)) return;
    const double* S = J.sums + (size_t)si * kSumDoubles;
    double* out = J.models + (size_t)si * kModelDoubles;
    double u[10], b[4];
    if (row == 3) {
        // M00 M01 M02 M11 M12 M22 into the padded upper triangle, b0 b1 b2
        u[0] = S[0];
        u[1] = S[1];
        u[2] = S[2];
        u[3] = 0.0;
        u[4] = S[3];
        u[5] = S[4];
        u[6] = 0.0;
        u[7] = S[5];
        u[8] = 0.0;
        u[9] = 1.0;
        const double lam = 1e-9 * (u[0] + u[4] + u[7]) / 3 + 1e-300;  // trace of the 3x3 system
        u[0] += lam;
        u[4] += lam;
        b[0] = S[6];
        b[1] = S[7];
        b[2] = S[8];
        b[3] = 0.0;
        solve4(u, b);
        out[0] = b[0];
        out[1] = b[1];
        out[2] = b[2];
        return;
    }
    if (J.motion[si] == 0) {
#pragma unroll
        for (int p = 0; p < 4; ++p) out[3 + 4 * row + p] = 0.0;
        return;
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) u[k] = S[9 + k];
#pragma unroll
    for (int p = 0; p < 4; ++p) b[p] = S[19 + 4 * row + p];
    const double lam = 1e-9 * (u[0] + u[4] + u[7] + u[9]) / 4 + 1e-300;
    u[0] += lam;
    u[4] += lam;
    u[7] += lam;
#pragma unroll
    for (int p = 0; p < 3; ++p)
        if (p == row) b[p] += lam;  // towards A = I
    solve4(u, b);
#pragma unroll
    for (int p = 0; p < 4; ++p) out[3 + 4 * row + p] = b[p];
}

// Closest seed of every pixel, exactly, in two separable passes: the
// squared distance to a seed is (x - xs)^2 + (y - ys)^2, so the closest seed
// minimises (x - x')^2 + g(x', y)^2 over the columns x', g(x', y) being the
// distance from row y to the closest seed in column x'.  A tie inside a
// column is a tie of the total distance at every pixel of the row, so each
// pass keeps the lower seed index on ties and the result is the closest
// seed with the lowest index.
//
// k_interp_columns: col[y][x] = (g, index) of the closest seed in column x,
// or (0, -1) when the column holds no seed.  A CTA takes 32 columns, each
// cut into kColSegments runs of block rows, one thread per column and run:
// every thread records the first and last seed of its run, then sweeps its
// run down and up starting from the nearest seeds of the runs above and
// below.
constexpr int kColSegments = 16;

__global__ void __launch_bounds__(32 * kColSegments) k_interp_columns(InterpJob J, int2* col) {
    __shared__ int2 first_s[kColSegments][32], last_s[kColSegments][32];  // (row, index), index -1: none
    const int lane = threadIdx.x, seg = threadIdx.y;
    const int x = blockIdx.x * 32 + lane;
    if (seed_count(J) == 0 || *J.status) return;  // uniform over the CTA
    const bool live = x < J.w;
    const int bx = x / kBlock, ox = x % kBlock;
    const int per = (J.gbh + kColSegments - 1) / kColSegments;
    const int b0 = min(J.gbh, seg * per), b1 = min(J.gbh, b0 + per);
    // the seed of block row by in this column, or -1
    auto seed_row = [&](int by, int& idx) {
        const int w = J.map[by * J.gbw + bx];
        idx = word_index(w);
        return (w >= 0 && ((w >> 2) & 3) == ox) ? by * kBlock + (w & 3) : -1;
    };
    int2 f = make_int2(0, -1), l = make_int2(0, -1);
    if (live)
        for (int by = b0; by < b1; ++by) {
            int idx;
            const int sy = seed_row(by, idx);
            if (sy < 0) continue;
            if (f.y < 0) f = make_int2(sy, idx);
            l = make_int2(sy, idx);
        }
    first_s[seg][lane] = f;
    last_s[seg][lane] = l;
    __syncthreads();
    if (!live) return;
    int2 up = make_int2(0, -1), dn = make_int2(0, -1);  // nearest seeds above / below the run
    for (int q = seg - 1; q >= 0 && up.y < 0; --q) up = last_s[q][lane];
    for (int q = seg + 1; q < kColSegments && dn.y < 0; ++q) dn = first_s[q][lane];
    int ly = up.x, li = up.y;
    for (int by = b0; by < b1; ++by) {
        int idx;
        const int sy = seed_row(by, idx);
        const int y0 = by * kBlock;
        for (int y = y0; y < min(y0 + kBlock, J.h); ++y) {
            if (y == sy) {
                ly = sy;
                li = idx;
            }
            col[(size_t)y * J.w + x] = make_int2(y - ly, li);
        }
    }
    int ny = dn.x, ni = dn.y;
    for (int by = b1 - 1; by >= b0; --by) {
        int idx;
        const int sy = seed_row(by, idx);
        const int y0 = by * kBlock;
        for (int y = min(y0 + kBlock, J.h) - 1; y >= y0; --y) {
            if (y == sy) {
                ny = sy;
                ni = idx;
            }
            if (ni < 0) continue;
            const size_t pi = (size_t)y * J.w + x;
            const int2 a = col[pi];
            const int g = ny - y;
            if (a.y < 0 || g < a.x || (g == a.x && ni < a.y)) col[pi] = make_int2(g, ni);
        }
    }
}

// k_interp_pixels: per pixel the closest seed along its row of col (scanning
// outwards until the horizontal distance alone exceeds the best), then its
// models evaluated at the pixel: d0 from the plane, x0 from
// (x, y, max(d0, 1)), x1 = A (x0 - c) + t projected back.
__global__ void k_interp_pixels(InterpJob J, const int2* col, float4* field) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= J.w || y >= J.h) return;
    const size_t pi = (size_t)y * J.w + x;
    if (seed_count(J) == 0 || *J.status) {
        field[pi] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int2* row = col + (size_t)y * J.w;
    long long bd = 0x7fffffffffffffffll;
    int best = 0x7fffffff;
    for (int dx = 0; dx < J.w; ++dx) {
        if ((long long)dx * dx > bd) break;
        const int xa = x - dx, xb = x + dx;
        if (xa >= 0) {
            const int2 c = row[xa];
            const long long d = (long long)dx * dx + (long long)c.x * c.x;
            if (c.y >= 0 && (d < bd || (d == bd && c.y < best))) {
                bd = d;
                best = c.y;
            }
        }
        if (dx > 0 && xb < J.w) {
            const int2 c = row[xb];
            const long long d = (long long)dx * dx + (long long)c.x * c.x;
            if (c.y >= 0 && (d < bd || (d == bd && c.y < best))) {
                bd = d;
                best = c.y;
            }
        }
    }
    if (best == 0x7fffffff) {  // unreachable while every seed is in the map
        field[pi] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const sff_seed s = J.seeds[best];
    const double* m = J.models + (size_t)best * kModelDoubles;
    const double d0 = m[0] * (x - s.x) + m[1] * (y - s.y) + m[2];
    float4 r = make_float4(0.f, 0.f, (float)d0, (float)d0);
    if (J.motion[best] > 0) {
        const double Z = J.fb / (d0 > 1.0 ? d0 : 1.0);
        const double X0[3] = {(x - J.p.cx) * Z * J.inv_f, (y - J.p.cy) * Z * J.inv_f, Z};
        const double* A = m + 3;
        const double* c = m + 15;
        double X1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            X1[j] = A[4 * j] * (X0[0] - c[0]) + A[4 * j + 1] * (X0[1] - c[1]) + A[4 * j + 2] * (X0[2] - c[2]) +
                    A[4 * j + 3];
        if (X1[2] > 0.0) {
            const double iz = 1.0 / X1[2];
            r.x = (float)(J.p.focal * X1[0] * iz + J.p.cx - x);
            r.y = (float)(J.p.focal * X1[1] * iz + J.p.cy - y);
            r.w = (float)(J.fb * iz);
        }
    }
    field[pi] = r;
}

struct InterpLayout {
    size_t map, pts, wt, models, sums, motion, nearest, status, total;
};

InterpLayout interp_layout(int w, int h, int capacity) {
    const int gbw = (w + kBlock - 1) / kBlock, gbh = (h + kBlock - 1) / kBlock;
    InterpLayout L;
    L.map = 0;
    L.pts = L.map + align256((size_t)gbw * gbh * sizeof(int));
    L.wt = L.pts + align256((size_t)capacity * kPointDoubles * sizeof(double));
    L.models = L.wt + align256((size_t)kWeightTable * sizeof(double));
    L.sums = L.models + align256((size_t)capacity * kModelDoubles * sizeof(double));
    L.motion = L.sums + align256((size_t)capacity * kSumDoubles * sizeof(double));
    L.nearest = L.motion + align256((size_t)capacity * sizeof(int));
    L.status = L.nearest + align256((size_t)w * h * sizeof(int2));
    L.total = L.status + 256;
    return L;
}

}  // namespace
}  // namespace sff

extern "C" int sff_default_interp_params(int32_t width, int32_t height, double focal, double baseline,
                                         sff_interp_params* out) {
    if (!out || width < 1 || height < 1 || !(focal > 0.0) || !(baseline > 0.0)) return SFF_ERR_ARG;
    out->k_geo = 160;
    out->k_motion = 80;
    out->alpha = 2.2;
    out->dist_unit = 20.0;
    out->focal = focal;
    out->baseline = baseline;
    out->cx = (width - 1) / 2.0;
    out->cy = (height - 1) / 2.0;
    return SFF_OK;
}

extern "C" size_t sff_interp_workspace_bytes(int32_t width, int32_t height, int32_t capacity) {
    if (sff::check_size(width, height) || capacity < 0) return 0;
    return sff::interp_layout(width, height, capacity).total;
}

extern "C" int sff_interpolate(const sff_seed* seeds_dev, const int32_t* count_dev, int32_t capacity, int32_t width,
                               int32_t height, const sff_interp_params* params, float* field_dev, void* workspace,
                               size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || !params || capacity < 0) return SFF_ERR_ARG;
    if (!seeds_dev || !count_dev || !field_dev || !workspace) return SFF_ERR_ARG;
    if (params->k_geo < 1 || params->k_geo > kMaxK || params->k_motion < 1 || params->k_motion > kMaxK ||
        !(params->alpha >= 0.0) || !(params->dist_unit > 0.0) || !(params->focal > 0.0) || !(params->baseline > 0.0))
        return SFF_ERR_ARG;
    if (((uintptr_t)field_dev & 15) || ((uintptr_t)workspace & 255) || ((uintptr_t)seeds_dev & 3)) return SFF_ERR_ARG;
    const InterpLayout L = interp_layout(width, height, capacity);
    if (workspace_bytes < L.total) return SFF_ERR_WORKSPACE;
    char* ws = reinterpret_cast<char*>(workspace);
    InterpJob J;
    J.seeds = seeds_dev;
    J.count = count_dev;
    J.capacity = capacity;
    J.w = width;
    J.h = height;
    J.gbw = (width + kBlock - 1) / kBlock;
    J.gbh = (height + kBlock - 1) / kBlock;
    J.map = reinterpret_cast<int*>(ws + L.map);
    J.pts = reinterpret_cast<double*>(ws + L.pts);
    J.wt = reinterpret_cast<double*>(ws + L.wt);
    J.models = reinterpret_cast<double*>(ws + L.models);
    J.sums = reinterpret_cast<double*>(ws + L.sums);
    J.motion = reinterpret_cast<int*>(ws + L.motion);
    J.status = reinterpret_cast<unsigned*>(ws + L.status);
    J.p = *params;
    J.fb = params->focal * params->baseline;
    J.inv_f = 1.0 / params->focal;
    J.slots = candidate_slots(params->k_geo, params->k_motion);
    cudaStream_t st = (cudaStream_t)stream;
    const int clear = max(J.gbw * J.gbh, kWeightTable);
    SFF_LAUNCH(k_interp_clear, dim3((clear + 255) / 256), 256, 0, st, J);
    if (capacity > 0) {
        SFF_LAUNCH(k_interp_prep, dim3((capacity + 255) / 256), 256, 0, st, J);
        const size_t smem = kModelWarps * warp_smem_bytes(J.slots, J.p.k_geo, J.p.k_motion);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k_interp_models, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SFF_ERR_CUDA;
        SFF_LAUNCH(k_interp_models, dim3((capacity + kModelWarps - 1) / kModelWarps), kModelWarps * 32, smem, st, J);
        SFF_LAUNCH(k_interp_solve, dim3((capacity + 31) / 32), 128, 0, st, J);
    }
    int2* col = reinterpret_cast<int2*>(ws + L.nearest);
    SFF_LAUNCH(k_interp_columns, dim3((width + 31) / 32), dim3(32, kColSegments), 0, st, J, col);
    SFF_LAUNCH(k_interp_pixels, dim3((width + 127) / 128, height), 128, 0, st, J, col,
               reinterpret_cast<float4*>(field_dev));
    return launch_status();
}

extern "C" int sff_interp_status(const void* workspace, int32_t width, int32_t height, int32_t capacity,
                                 uint32_t* status_out) {
    using namespace sff;
    if (!workspace || !status_out || check_size(width, height) || capacity < 0) return SFF_ERR_ARG;
    const InterpLayout L = interp_layout(width, height, capacity);
    if (cudaMemcpy(status_out, reinterpret_cast<const char*>(workspace) + L.status, sizeof(uint32_t),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return SFF_ERR_CUDA;
    return SFF_OK;
}
