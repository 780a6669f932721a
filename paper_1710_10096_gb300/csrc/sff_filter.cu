// Consistency check and region filter (Sec. 3.1, "Consistency Check").
//
// k_consistency: per L0 pixel, gather the inverse vector at its cross match
//                in R1 and compare the round trip of all three
//                correspondences.
// Region filter: connected components of kept pixels (4-neighbours whose
//                vectors differ by at most tau_r) by union-find.  Unions
//                always hang the larger root under the smaller one with
//                atomicMin, so every component ends with its minimum raster
//                index as root, independent of scheduling.  Then the size of
//                each component and whether a rejected neighbour could join
//                it are accumulated on the root, and small joinable
//                components are removed.
// Scratch (workspace): parent[H*W], size[H*W], joinable[H*W] int32.
#include "sff_internal.cuh"

namespace sff {
namespace {

__global__ void k_consistency(const uint2* __restrict__ fwd, const int* __restrict__ fcost,
                              const uint2* __restrict__ inv, const int* __restrict__ icost, int w, int h, int tau_c,
                              uint8_t* __restrict__ keep, uint8_t* __restrict__ cerr) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= w) return;
    const size_t i = (size_t)y * w + x;
    uint8_t k = 0, e = 255;
    if (fcost[i] != kEmpty) {
        const Vec4 a = unpack_vec(fwd[i]);
        const int qx = x + a.u - a.d1, qy = y + a.v;
        if (qx >= 0 && qx < w && qy >= 0 && qy < h) {
            const size_t j = (size_t)qy * w + qx;
            if (icost[j] != kEmpty) {
                const Vec4 b = unpack_vec(inv[j]);
                const int d0 = abs(b.u + a.u - a.d1 + a.d0), d1 = abs(b.v + a.v);
                const int d2 = abs(b.d0 - a.d1), d3 = abs(b.d1 - a.d0);
                const int mx = max(max(d0, d1), max(d2, d3)), sum = d0 + d1 + d2 + d3;
                k = mx <= tau_c;
                e = (uint8_t)min(sum, 255);
            }
        }
    }
    keep[i] = k;
    cerr[i] = e;
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
// the loop ends after at most a few steps per element.
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

__global__ void k_cc_init(const uint8_t* __restrict__ keep, int np, int* __restrict__ parent, int* __restrict__ size,
                          int* __restrict__ joinable) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    parent[i] = keep[i] ? i : -1;
    size[i] = 0;
    joinable[i] = 0;
}

__global__ void k_cc_union(const uint2* __restrict__ fwd, const uint8_t* __restrict__ keep, int w, int h, int tau_r,
                           int* parent) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= w) return;
    const int i = y * w + x;
    if (!keep[i]) return;
    const uint2 a = fwd[i];
    if (x + 1 < w && keep[i + 1] && close_vec(a, fwd[i + 1], tau_r)) unite(parent, i, i + 1);
    if (y + 1 < h && keep[i + w] && close_vec(a, fwd[i + w], tau_r)) unite(parent, i, i + w);
}

__global__ void k_cc_stats(const uint2* __restrict__ fwd, const int* __restrict__ fcost,
                           const uint8_t* __restrict__ keep, int w, int h, int tau_r, int* parent, int* size,
                           int* joinable) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= w) return;
    const int i = y * w + x;
    if (!keep[i]) return;
    const int root = find_root(parent, i);
    atomicAdd(size + root, 1);
    const uint2 a = fwd[i];
    const int nx[4] = {x + 1, x - 1, x, x};
    const int ny[4] = {y, y, y + 1, y - 1};
    bool join = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (nx[k] < 0 || nx[k] >= w || ny[k] < 0 || ny[k] >= h) continue;
        const int j = ny[k] * w + nx[k];
        if (!keep[j] && fcost[j] != kEmpty && close_vec(a, fwd[j], tau_r)) join = true;
    }
    if (join) atomicOr(joinable + root, 1);
}

__global__ void k_cc_remove(uint8_t* __restrict__ keep, int np, const int* parent, const int* __restrict__ size,
                            const int* __restrict__ joinable, int region_min) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np || !keep[i]) return;
    const int root = find_root(parent, i);
    if (joinable[root] && size[root] < region_min) keep[i] = 0;
}

}  // namespace

size_t filter_ws_bytes(int w, int h) { return 3 * align256((size_t)w * h * sizeof(int)); }

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
    cudaStream_t st = (cudaStream_t)stream;
    const uint2* fwd = reinterpret_cast<const uint2*>(fwd_dev);
    const uint2* inv = reinterpret_cast<const uint2*>(inv_dev);
    const int np = width * height;
    const size_t slab = align256((size_t)np * sizeof(int));
    int* parent = reinterpret_cast<int*>(workspace);
    int* size = reinterpret_cast<int*>((char*)workspace + slab);
    int* joinable = reinterpret_cast<int*>((char*)workspace + 2 * slab);
    dim3 b2(128), g2((width + 127) / 128, height);
    const int g1 = (np + 255) / 256;
    SFF_LAUNCH(k_consistency, g2, b2, 0, st, fwd, fwd_cost_dev, inv, inv_cost_dev, width, height, params->tau_c, keep_dev,
                                     cerr_dev);
    SFF_LAUNCH(k_cc_init, g1, 256, 0, st, keep_dev, np, parent, size, joinable);
    SFF_LAUNCH(k_cc_union, g2, b2, 0, st, fwd, keep_dev, width, height, params->tau_r, parent);
    SFF_LAUNCH(k_cc_stats, g2, b2, 0, st, fwd, fwd_cost_dev, keep_dev, width, height, params->tau_r, parent, size,
                                  joinable);
    SFF_LAUNCH(k_cc_remove, g1, 256, 0, st, keep_dev, np, parent, size, joinable, params->region_min);
    return launch_status();
}
