// Consistency check and region filter (Sec. 3.1, "Consistency Check").
//
// Consistency: per L0 pixel, gather the inverse vector at its cross match
//                in R1 and compare the round trip of all three
//                correspondences (consistency_at, run by k_cc_local for the
//                pixels of its tile).
// Region filter: connected components of kept pixels (4-neighbours whose
//                vectors differ by at most tau_r) by union-find, first inside
//                32x32 tiles in shared memory (k_cc_local), then across tile
//                borders in global memory (k_cc_border).  Unions always hang
//                the larger root under the smaller one with atomicMin, so
//                every component ends with its minimum raster index as root,
//                independent of scheduling.  Then the size of each component
//                and whether a rejected neighbour could join it are
//                accumulated on the root (k_cc_stats), and small joinable
//                components are removed (k_cc_remove).
// Scratch (workspace): parent[H*W], size[H*W], joinable[H*W] int32.
#include <mutex>

#include "sff_internal.cuh"

namespace sff {
namespace {

struct FilterJobs {
    FilterJob q[kMaxQuads];
};

// Consistency of pixel (x, y): writes keep and cerr, returns keep.
__device__ __forceinline__ bool consistency_at(const FilterJob& Q, int x, int y, int tau_c) {
    const int w = Q.w, h = Q.h;
    const size_t i = (size_t)y * w + x;
    uint8_t k = 0, e = 255;
    if (Q.fcost[i] != kEmpty) {
        const Vec4 a = unpack_vec(Q.fwd[i]);
        const int qx = x + a.u - a.d1, qy = y + a.v;
        if (qx >= 0 && qx < w && qy >= 0 && qy < h) {
            const size_t j = (size_t)qy * w + qx;
            if (Q.icost[j] != kEmpty) {
                const Vec4 b = unpack_vec(Q.inv[j]);
                const int d0 = abs(b.u + a.u - a.d1 + a.d0), d1 = abs(b.v + a.v);
                const int d2 = abs(b.d0 - a.d1), d3 = abs(b.d1 - a.d0);
                const int mx = max(max(d0, d1), max(d2, d3)), sum = d0 + d1 + d2 + d3;
                k = mx <= tau_c;
                e = (uint8_t)min(sum, 255);
            }
        }
    }
    Q.keep[i] = k;
    Q.cerr[i] = e;
    return k != 0;
}

__device__ __forceinline__ bool close_vec(uint2 a, uint2 b, int tau) {
    const Vec4 p = unpack_vec(a), q = unpack_vec(b);
    return abs(p.u - q.u) <= tau && abs(p.v - q.v) <= tau && abs(p.d0 - q.d0) <= tau && abs(p.d1 - q.d1) <= tau;
}

__device__ __forceinline__ int find_root(const int* parent, int x) {
    int p = __ldcg(parent + x);
    while (p != x) {
        x = p;
        p = __ldcg(parent + x);
    }
    return x;
}

// Each round either finishes or moves a root to a strictly smaller index, so
// the loop ends after a few steps per element.
__device__ void unite(int* parent, int a, int b) {
    while (true) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
}

constexpr int kTile = 32;  // union-find tile: 32 x 32 pixels

// Root of k with path halving: every visited node is re-pointed to its
// grandparent.  Parents only ever point to smaller indices of the same
// component, so a concurrent halving write or link leaves every pointer on an
// ancestor: the races are benign and pointers only decrease.
__device__ __forceinline__ int find_local(volatile int* lp, int k) {
    while (true) {
        const int p = lp[k];
        if (p == k) return k;
        const int gp = lp[p];
        if (gp == p) return p;
        lp[k] = gp;
        k = gp;
    }
}

__device__ void unite_local(int* lp, int a, int b) {
    while (true) {
        a = find_local(lp, a);
        b = find_local(lp, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(lp + a, b);
        if (old == a) return;
        a = old;
    }
}

// Components inside one tile in shared memory.  Local indices follow raster
// order.  Each kept pixel starts linked to its connected upper neighbour, else
// its connected left one (both smaller indices), else to itself; a pixel
// connected both ways then unites the two; finds halve paths.  The minimum
// raster index of a local component has no connected upper or left
// neighbour, starts as a root and stays one, since links always go to the
// smaller root: every kept pixel's parent becomes that minimum.  Also clears
// size and joinable for the tile's pixels.  The tile's keep and cerr are
// computed first, by the consistency check of each of its pixels.
constexpr int kLocalThreads = 512;
constexpr int kPerThread = kTile * kTile / kLocalThreads;

__global__ void __launch_bounds__(kLocalThreads) k_cc_local(const __grid_constant__ FilterJobs J, int tau_r,
                                                            int tau_c) {
    __shared__ int lp[kTile * kTile];
    __shared__ uint2 lf[kTile * kTile];
    __shared__ uint8_t lk[kTile * kTile];
    const FilterJob& Q = J.q[blockIdx.z];
    const int w = Q.w, h = Q.h;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    if (x0 >= w || y0 >= h) return;  // whole CTA beyond this quad
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + j * kLocalThreads;
        const int x = x0 + (k % kTile), y = y0 + (k / kTile);
        const bool inside = x < w && y < h;
        const size_t i = (size_t)y * w + x;
        const bool kk = inside && consistency_at(Q, x, y, tau_c);
        lk[k] = kk;
        lf[k] = kk ? Q.fwd[i] : make_uint2(0u, 0u);
        if (inside) {
            Q.size[i] = 0;
            Q.joinable[i] = 0;
        }
    }
    __syncthreads();
    bool both[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + j * kLocalThreads;
        const int lx = k % kTile, ly = k / kTile;
        both[j] = false;
        if (!lk[k]) {
            lp[k] = -1;
            continue;
        }
        const bool up = ly > 0 && lk[k - kTile] && close_vec(lf[k], lf[k - kTile], tau_r);
        const bool left = lx > 0 && lk[k - 1] && close_vec(lf[k], lf[k - 1], tau_r);
        lp[k] = up ? k - kTile : left ? k - 1 : k;
        both[j] = up && left;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + j * kLocalThreads;
        if (both[j]) unite_local(lp, k - 1, k);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int k = threadIdx.x + j * kLocalThreads;
        if (!lk[k]) continue;
        const int r = find_local(lp, k);
        const int x = x0 + k % kTile, y = y0 + k / kTile;
        if (x < w && y < h) Q.parent[(size_t)y * w + x] = (y0 + r / kTile) * w + x0 + r % kTile;
    }
}

// Unions across tile borders only: one thread per pixel pair that a tile
// border separates, first the (x, x + 1) pairs of every vertical border
// (x = 31, 63, ...; all rows), then the (y, y + 1) pairs of every
// horizontal border (all columns).  The unions are the same whatever their
// order, and so is every root (the minimum raster index).
__global__ void k_cc_border(const __grid_constant__ FilterJobs J, int tau_r) {
    const FilterJob& Q = J.q[blockIdx.z];
    const int w = Q.w, h = Q.h;
    const int nv = (w - 1) / kTile, nh = (h - 1) / kTile;  // borders with a pixel on both sides
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i, j;
    if (t < (long long)nv * h) {
        const int y = (int)(t / nv), x = ((int)(t % nv) + 1) * kTile - 1;
        i = y * w + x;
        j = i + 1;
    } else if (t < (long long)nv * h + (long long)nh * w) {
        const long long u = t - (long long)nv * h;
        const int y = ((int)(u / w) + 1) * kTile - 1, x = (int)(u % w);
        i = y * w + x;
        j = i + w;
    } else {
        return;
    }
    if (Q.keep[i] && Q.keep[j] && close_vec(Q.fwd[i], Q.fwd[j], tau_r)) unite(Q.parent, i, j);
}

// Root of every kept pixel (written back to parent), component sizes with
// one atomic per distinct root per warp, and the "a rejected neighbour
// could join" flag.
__global__ void k_cc_stats(const __grid_constant__ FilterJobs J, int tau_r) {
    const FilterJob& Q = J.q[blockIdx.z];
    const int w = Q.w, h = Q.h;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int i = y * w + x;
    const bool kept = x < w && y < h && Q.keep[i];
    int root = -1;
    bool join = false;
    if (kept) {
        root = find_root(Q.parent, i);
        Q.parent[i] = root;
        const uint2 a = Q.fwd[i];
        const uint8_t* keep = Q.keep;
        const int* fcost = Q.fcost;
        const uint2* fwd = Q.fwd;
        if (x + 1 < w && !keep[i + 1] && fcost[i + 1] != kEmpty && close_vec(a, fwd[i + 1], tau_r)) join = true;
        if (x > 0 && !keep[i - 1] && fcost[i - 1] != kEmpty && close_vec(a, fwd[i - 1], tau_r)) join = true;
        if (y + 1 < h && !keep[i + w] && fcost[i + w] != kEmpty && close_vec(a, fwd[i + w], tau_r)) join = true;
        if (y > 0 && !keep[i - w] && fcost[i - w] != kEmpty && close_vec(a, fwd[i - w], tau_r)) join = true;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, root);
    const int lane = threadIdx.x & 31;
    if (kept && lane == __ffs(peers) - 1) atomicAdd(Q.size + root, __popc(peers));
    if (join) atomicOr(Q.joinable + root, 1);
}

__global__ void k_cc_remove(const __grid_constant__ FilterJobs J, int region_min) {
    const FilterJob& Q = J.q[blockIdx.z];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= Q.w || y >= Q.h) return;
    const int i = y * Q.w + x;
    if (!Q.keep[i]) return;
    const int root = Q.parent[i];
    if (Q.joinable[root] && Q.size[root] < region_min) Q.keep[i] = 0;
}

}  // namespace

size_t filter_ws_bytes(int w, int h) { return 3 * align256((size_t)w * h * sizeof(int)); }

void filter_carve(void* workspace, int w, int h, int** parent, int** size, int** joinable) {
    const size_t slab = align256((size_t)w * h * sizeof(int));
    *parent = reinterpret_cast<int*>(workspace);
    *size = reinterpret_cast<int*>((char*)workspace + slab);
    *joinable = reinterpret_cast<int*>((char*)workspace + 2 * slab);
}

int run_filter(const FilterJob* jobs, int n, const sff_params& P, cudaStream_t st, bool remove) {
    if (n < 1 || n > kMaxQuads) return SFF_ERR_ARG;
    static FilterJobs J;  // host staging of the kernel parameter (copied at each launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int mw = 0, mh = 0;
    for (int k = 0; k < n; ++k) {
        J.q[k] = jobs[k];
        mw = mw > jobs[k].w ? mw : jobs[k].w;
        mh = mh > jobs[k].h ? mh : jobs[k].h;
    }
    dim3 b2(128), g2((mw + 127) / 128, mh, n);
    dim3 gt((mw + kTile - 1) / kTile, (mh + kTile - 1) / kTile, n);
    // border pairs of the largest quad
    long long pairs = 0;
    for (int k = 0; k < n; ++k) {
        const long long p = (long long)((jobs[k].w - 1) / kTile) * jobs[k].h + (long long)((jobs[k].h - 1) / kTile) * jobs[k].w;
        pairs = pairs > p ? pairs : p;
    }
    SFF_LAUNCH(k_cc_local, gt, kLocalThreads, 0, st, J, P.tau_r, P.tau_c);
    if (pairs > 0) SFF_LAUNCH(k_cc_border, dim3((unsigned)((pairs + 127) / 128), 1, n), b2, 0, st, J, P.tau_r);
    SFF_LAUNCH(k_cc_stats, g2, b2, 0, st, J, P.tau_r);
    if (remove) SFF_LAUNCH(k_cc_remove, g2, b2, 0, st, J, P.region_min);
    return launch_status();
}

}  // namespace sff

extern "C" int sff_consistency_filter(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const int16_t* inv_dev,
                                      const int32_t* inv_cost_dev, int32_t width, int32_t height,
                                      const sff_params* params, uint8_t* keep_dev, uint8_t* cerr_dev,
                                      void* workspace, size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!fwd_dev || !fwd_cost_dev || !inv_dev || !inv_cost_dev || !keep_dev || !cerr_dev || !workspace)
        return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)inv_dev & 7) || ((uintptr_t)fwd_cost_dev & 3) ||
        ((uintptr_t)inv_cost_dev & 3) || ((uintptr_t)workspace & 255))
        return SFF_ERR_ARG;
    if (workspace_bytes < filter_ws_bytes(width, height)) return SFF_ERR_WORKSPACE;
    FilterJob job{reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev, reinterpret_cast<const uint2*>(inv_dev),
                  inv_cost_dev, width, height, keep_dev, cerr_dev, nullptr, nullptr, nullptr};
    filter_carve(workspace, width, height, &job.parent, &job.size, &job.joinable);
    return run_filter(&job, 1, *params, (cudaStream_t)stream);
}
