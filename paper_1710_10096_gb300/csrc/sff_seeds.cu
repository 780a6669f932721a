// Sparsification into seeds (Sec. 3.2): per non-overlapping 3x3 block the
// kept match with the lowest consistency error (then cost, then raster
// index), compacted in block raster order.
//
// k_block_best: one thread per block -> raster index of its best pixel or -1.
// k_compact:    one CTA of 1024 threads: each thread counts the seeds of a
//               contiguous run of blocks, a CTA-wide exclusive scan gives the
//               run's output offset, then each thread writes its run in order.
// Scratch (workspace): best[ceil(W/3) * ceil(H/3)] int32.
#include <mutex>

#include "sff_internal.cuh"

namespace sff {
namespace {

constexpr int kScanThreads = 1024;

// Scratch of sff_emit_seeds_noalloc: one int32 per 3x3 block, in a static
// device array so that the call needs no allocation.  Every device that
// loads the library holds these 2 MiB until the process exits.
constexpr int kNoAllocMaxBlocks = SFF_NOALLOC_MAX_BLOCKS;
__device__ __align__(256) int g_noalloc_best[kNoAllocMaxBlocks];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int* g_noalloc_ptr[kMaxDevices] = {};

__global__ void k_block_best(const int* __restrict__ fcost, const uint8_t* __restrict__ keep,
                             const uint8_t* __restrict__ cerr, int w, int h, int bw, int nb, int* __restrict__ best) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int bx = (b % bw) * 3, by = (b / bw) * 3;
    int bi = -1, be = 0, bc = 0;
    for (int y = by; y < min(by + 3, h); ++y)
        for (int x = bx; x < min(bx + 3, w); ++x) {
            const int i = y * w + x;
            if (!keep[i]) continue;
            const int e = cerr[i], c = fcost[i];
            if (bi < 0 || e < be || (e == be && c < bc)) {  // raster order: ties keep the earlier pixel
                bi = i;
                be = e;
                bc = c;
            }
        }
    best[b] = bi;
}

__global__ void __launch_bounds__(kScanThreads) k_compact(const int* __restrict__ best, int nb, const uint2* __restrict__ fwd,
                                                         const int* __restrict__ fcost, const uint8_t* __restrict__ cerr,
                                                         int w, sff_seed* __restrict__ out, int capacity,
                                                         int* __restrict__ count) {
    __shared__ int warp_sums[kScanThreads / 32];
    const int t = threadIdx.x;
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    int mine = 0;
    for (int b = b0; b < b1; ++b) mine += best[b] >= 0;
    // inclusive scan within the warp, then across warps
    int v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if ((t & 31) >= o) v += u;
    }
    if ((t & 31) == 31) warp_sums[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        int s = warp_sums[t];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, s, o);
            if (t >= o) s += u;
        }
        warp_sums[t] = s;  // inclusive over warps
    }
    __syncthreads();
    int pos = v - mine + ((t >> 5) ? warp_sums[(t >> 5) - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const int i = best[b];
        if (i < 0) continue;
        if (pos < capacity) {
            const Vec4 a = unpack_vec(fwd[i]);
            sff_seed sd;
            sd.x = (int16_t)(i % w);
            sd.y = (int16_t)(i / w);
            sd.u = (int16_t)a.u;
            sd.v = (int16_t)a.v;
            sd.d0 = (int16_t)a.d0;
            sd.d1 = (int16_t)a.d1;
            sd.cost = fcost[i];
            sd.cerr = cerr[i];
            sd.pad[0] = sd.pad[1] = sd.pad[2] = 0;
            out[pos] = sd;
        }
        ++pos;
    }
    if (t == kScanThreads - 1) *count = pos;
}

}  // namespace

size_t seeds_ws_bytes(int w, int h) { return align256((size_t)((w + 2) / 3) * ((h + 2) / 3) * sizeof(int)); }

}  // namespace sff

extern "C" int sff_emit_seeds(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const uint8_t* keep_dev,
                              const uint8_t* cerr_dev, int32_t width, int32_t height, sff_seed* seeds_dev,
                              int32_t capacity, int32_t* count_dev, void* workspace, size_t workspace_bytes,
                              void* stream) {
    using namespace sff;
    if (check_size(width, height)) return SFF_ERR_ARG;
    if (!fwd_dev || !fwd_cost_dev || !keep_dev || !cerr_dev || !count_dev || !workspace || capacity < 0)
        return SFF_ERR_ARG;
    if (capacity > 0 && !seeds_dev) return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)seeds_dev & 3) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < seeds_ws_bytes(width, height)) return SFF_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int bw = (width + 2) / 3, nb = bw * ((height + 2) / 3);
    int* best = reinterpret_cast<int*>(workspace);
    SFF_LAUNCH(k_block_best, (nb + 255) / 256, 256, 0, st, fwd_cost_dev, keep_dev, cerr_dev, width, height, bw, nb, best);
    SFF_LAUNCH(k_compact, 1, kScanThreads, 0, st, best, nb, reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev, cerr_dev,
                                          width, seeds_dev, capacity, count_dev);
    return launch_status();
}

extern "C" int sff_emit_seeds_noalloc(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const uint8_t* keep_dev,
                                      const uint8_t* cerr_dev, int32_t width, int32_t height, sff_seed* seeds_dev,
                                      int32_t capacity, int32_t* count_dev, void* stream) {
    using namespace sff;
    if (check_size(width, height)) return SFF_ERR_ARG;
    if (!fwd_dev || !fwd_cost_dev || !keep_dev || !cerr_dev || !count_dev || capacity < 0) return SFF_ERR_ARG;
    if (capacity > 0 && !seeds_dev) return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)seeds_dev & 3)) return SFF_ERR_ARG;
    const int bw = (width + 2) / 3, nb = bw * ((height + 2) / 3);
    if (nb > kNoAllocMaxBlocks) return SFF_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SFF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SFF_ERR_ARG;
    int* best = nullptr;
    {
        // Host code cannot use the array's name as a device address: look the
        // address up once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_best) != cudaSuccess || !p) return SFF_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<int*>(p);
        }
        best = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // k_block_best writes every one of the nb entries before k_compact reads
    // them, so the array needs no clearing between calls.
    SFF_LAUNCH(k_block_best, (nb + 255) / 256, 256, 0, st, fwd_cost_dev, keep_dev, cerr_dev, width, height, bw, nb,
               best);
    SFF_LAUNCH(k_compact, 1, kScanThreads, 0, st, best, nb, reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev,
               cerr_dev, width, seeds_dev, capacity, count_dev);
    return launch_status();
}
