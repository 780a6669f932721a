// Sparsification into seeds (Sec. 3.2): per non-overlapping 3x3 block the
// kept match with the lowest consistency error (then cost, then raster
// index), compacted in block raster order.  With the disparity fill (Sec.
// 3.1, last paragraph) a block without a kept match takes its pixel whose
// d0 agrees best with the SGM map (|d0 - sgm| <= tau_c; then cost, then
// raster index) as a disparity-only seed (kind 1, u = v = d1 = 0).
//
// k_block_best:  one thread per block -> raster index i of its best kept
//                pixel, -(i + 2) for a disparity-only seed, or -1; and the
//                number of seeds of each chunk of 256 blocks.
// k_write_seeds: rank inside the chunk by warp ballots + chunk offset (the
//                sum of the earlier chunks' counts, which each CTA adds up
//                itself: at most a few thousand values); the last chunk's
//                CTA writes the total count.
// Scratch (workspace): best[ceil(W/3) * ceil(H/3)] and one int32 per chunk.
#include <mutex>

#include "sff_internal.cuh"

namespace sff {
namespace {

constexpr int kChunk = 256;        // 3x3 blocks per CTA of k_block_best / k_write_seeds

// Scratch of sff_emit_seeds_noalloc, in a static device array so that the
// call needs no allocation: one int32 per 3x3 block plus one per chunk of
// 256 blocks.  Every device that loads the library holds it until exit.
constexpr int kNoAllocMaxBlocks = SFF_NOALLOC_MAX_BLOCKS;
constexpr int kNoAllocInts = kNoAllocMaxBlocks + kNoAllocMaxBlocks / kChunk;
__device__ __align__(256) int g_noalloc_scratch[kNoAllocInts];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int* g_noalloc_ptr[kMaxDevices] = {};

struct SeedJobs {
    SeedJob q[kMaxQuads];
};

// Conditions raised since the last reset (read by sff_device_status): bit 1
// a seed buffer was smaller than the number of seeds (its count still holds
// the number needed).
constexpr unsigned kStatusCapacity = 2u;
__device__ unsigned int g_seed_status;

// One thread per block: raster index of its best kept pixel or -1; one count
// of found seeds per CTA.
__global__ void __launch_bounds__(kChunk) k_block_best(const __grid_constant__ SeedJobs J) {
    const SeedJob& Q = J.q[blockIdx.z];
    const int w = Q.w, h = Q.h, bw = (w + 2) / 3, nb = bw * ((h + 2) / 3);
    if ((int)blockIdx.x * kChunk >= nb) return;  // whole CTA beyond this quad's blocks
    const int b = blockIdx.x * kChunk + threadIdx.x;
    int bi = -1;
    if (b < nb) {
        const int bx = (b % bw) * 3, by = (b / bw) * 3;
        int be = 0, bc = 0;
        // the block's up to 9 pixels in raster order, each step's loads issued
        // for all of them together: kept?, then (with the removal) their
        // components, then their consistency errors and costs
        int pi[9];
        bool kk[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int y = by + k / 3, x = bx + k % 3;
            pi[k] = y * w + x;
            kk[k] = y < h && x < w && Q.keep[pi[k]];
        }
        if (Q.parent) {  // the region filter's removal (k_cc_remove's rule)
            int root[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) root[k] = kk[k] ? Q.parent[pi[k]] : 0;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (kk[k] && Q.joinable[root[k]] && Q.size[root[k]] < Q.region_min) {
                    Q.keep_rw[pi[k]] = 0;
                    kk[k] = false;
                }
        }
        int ek[9], ck[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            ek[k] = kk[k] ? Q.cerr[pi[k]] : 0;
            ck[k] = kk[k] ? Q.fcost[pi[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (kk[k] && (bi < 0 || ek[k] < be || (ek[k] == be && ck[k] < bc))) {  // ties keep the earlier pixel
                bi = pi[k];
                be = ek[k];
                bc = ck[k];
            }
        if (bi < 0 && Q.sgm) {
            int ge = 0, gc = 0;
            for (int y = by; y < min(by + 3, h); ++y)
                for (int x = bx; x < min(bx + 3, w); ++x) {
                    const int i = y * w + x;
                    const int c = Q.fcost[i];
                    if (c == kEmpty) continue;
                    const int e = abs(unpack_vec(Q.fwd[i]).d0 - Q.sgm[i]);
                    if (e <= Q.tau_c && (bi == -1 || e < ge || (e == ge && c < gc))) {
                        bi = -(i + 2);
                        ge = e;
                        gc = c;
                    }
                }
        }
        Q.best[b] = bi;
    }
    const int n = __syncthreads_count(bi != -1);
    if (threadIdx.x == 0) Q.chunk[blockIdx.x] = n;
}

// Same grid as k_block_best: rank of each found seed inside its CTA (warp
// ballots + warp offsets) plus the chunk offset gives its output slot.
__global__ void __launch_bounds__(kChunk) k_write_seeds(const __grid_constant__ SeedJobs J) {
    __shared__ int warp_base[kChunk / 32];
    __shared__ int warp_prior[kChunk / 32];
    __shared__ int chunk_base;
    const SeedJob& Q = J.q[blockIdx.z];
    const int w = Q.w, nb = ((Q.w + 2) / 3) * ((Q.h + 2) / 3);
    const int nchunks = (nb + kChunk - 1) / kChunk;
    if ((int)blockIdx.x >= nchunks) return;  // whole CTA beyond this quad's blocks
    // seeds of the chunks before this one
    int prior = 0;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += kChunk) prior += Q.chunk[c];
    prior = __reduce_add_sync(0xffffffffu, prior);
    const int b = blockIdx.x * kChunk + threadIdx.x;
    const int i = b < nb ? Q.best[b] : -1;
    const unsigned ballot = __ballot_sync(0xffffffffu, i != -1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        warp_base[wid] = __popc(ballot);
        warp_prior[wid] = prior;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0, base = 0;
        for (int k = 0; k < kChunk / 32; ++k) {
            const int n = warp_base[k];
            warp_base[k] = acc;
            acc += n;
            base += warp_prior[k];
        }
        chunk_base = base;
        if ((int)blockIdx.x == nchunks - 1) {  // the total
            *Q.count = base + acc;
            if (base + acc > Q.capacity) atomicOr(&g_seed_status, kStatusCapacity);
        }
    }
    __syncthreads();
    if (i == -1) return;
    const int pos = chunk_base + warp_base[wid] + __popc(ballot & ((1u << lane) - 1u));
    if (pos >= Q.capacity) return;
    const bool geo = i < -1;
    const int pi = geo ? -(i + 2) : i;
    const Vec4 a = unpack_vec(Q.fwd[pi]);
    sff_seed sd;
    sd.x = (int16_t)(pi % w);
    sd.y = (int16_t)(pi / w);
    sd.u = geo ? 0 : (int16_t)a.u;
    sd.v = geo ? 0 : (int16_t)a.v;
    sd.d0 = (int16_t)a.d0;
    sd.d1 = geo ? 0 : (int16_t)a.d1;
    sd.cost = Q.fcost[pi];
    sd.cerr = geo ? (uint8_t)abs(a.d0 - Q.sgm[pi]) : Q.cerr[pi];
    sd.kind = geo ? 1 : 0;
    sd.pad[0] = sd.pad[1] = 0;
    Q.out[pos] = sd;
}

}  // namespace

size_t seeds_ws_bytes(int w, int h) {
    const size_t nb = (size_t)((w + 2) / 3) * ((h + 2) / 3);
    return align256(nb * sizeof(int)) + align256((nb + kChunk - 1) / kChunk * sizeof(int));
}

void seeds_carve(void* workspace, int w, int h, int** best, int** chunk) {
    const size_t nb = (size_t)((w + 2) / 3) * ((h + 2) / 3);
    *best = reinterpret_cast<int*>(workspace);
    *chunk = reinterpret_cast<int*>((char*)workspace + align256(nb * sizeof(int)));
}

// Reads (and with reset clears) the condition bits of the seed kernels, in
// stream order; the caller synchronises the stream.
int seeds_status_read(cudaStream_t st, unsigned* out, bool reset) {
    static const unsigned zero = 0;
    if (cudaMemcpyFromSymbolAsync(out, g_seed_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SFF_ERR_CUDA;
    if (reset && cudaMemcpyToSymbolAsync(g_seed_status, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st) !=
                     cudaSuccess)
        return SFF_ERR_CUDA;
    return SFF_OK;
}

int run_seeds(const SeedJob* jobs, int n, cudaStream_t st) {
    if (n < 1 || n > kMaxQuads) return SFF_ERR_ARG;
    static SeedJobs J;  // host staging of the kernel parameter (copied at each launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int mchunks = 0;
    for (int k = 0; k < n; ++k) {
        J.q[k] = jobs[k];
        const int nb = ((jobs[k].w + 2) / 3) * ((jobs[k].h + 2) / 3);
        mchunks = mchunks > (nb + kChunk - 1) / kChunk ? mchunks : (nb + kChunk - 1) / kChunk;
    }
    SFF_LAUNCH(k_block_best, dim3(mchunks, 1, n), kChunk, 0, st, J);
    SFF_LAUNCH(k_write_seeds, dim3(mchunks, 1, n), kChunk, 0, st, J);
    return launch_status();
}

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
    SeedJob job{reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev, keep_dev, cerr_dev, width, height, nullptr,
                nullptr, seeds_dev, capacity, count_dev};
    seeds_carve(workspace, width, height, &job.best, &job.chunk);
    return run_seeds(&job, 1, (cudaStream_t)stream);
}

extern "C" int sff_emit_seeds_noalloc(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const uint8_t* keep_dev,
                                      const uint8_t* cerr_dev, int32_t width, int32_t height, sff_seed* seeds_dev,
                                      int32_t capacity, int32_t* count_dev, void* stream) {
    using namespace sff;
    if (check_size(width, height)) return SFF_ERR_ARG;
    if (!fwd_dev || !fwd_cost_dev || !keep_dev || !cerr_dev || !count_dev || capacity < 0) return SFF_ERR_ARG;
    if (capacity > 0 && !seeds_dev) return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)seeds_dev & 3)) return SFF_ERR_ARG;
    const int nb = ((width + 2) / 3) * ((height + 2) / 3);
    if (nb > kNoAllocMaxBlocks) return SFF_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SFF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SFF_ERR_ARG;
    int* scratch = nullptr;
    {
        // Host code cannot use the array's name as a device address: look the
        // address up once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SFF_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<int*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // Every scratch entry a call reads is written earlier in the same call
    // (block bests and chunk counts by k_block_best), so nothing is cleared.
    SeedJob job{reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev, keep_dev, cerr_dev, width, height, scratch,
                scratch + kNoAllocMaxBlocks, seeds_dev, capacity, count_dev};
    return run_seeds(&job, 1, (cudaStream_t)stream);
}

extern "C" int sff_emit_seeds_geo(const int16_t* fwd_dev, const int32_t* fwd_cost_dev, const uint8_t* keep_dev,
                                  const uint8_t* cerr_dev, const int16_t* sgm_dev, int32_t width, int32_t height,
                                  const sff_params* params, sff_seed* seeds_dev, int32_t capacity, int32_t* count_dev,
                                  void* workspace, size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!fwd_dev || !fwd_cost_dev || !keep_dev || !cerr_dev || !sgm_dev || !count_dev || !workspace || capacity < 0)
        return SFF_ERR_ARG;
    if (capacity > 0 && !seeds_dev) return SFF_ERR_ARG;
    if (((uintptr_t)fwd_dev & 7) || ((uintptr_t)seeds_dev & 3) || ((uintptr_t)workspace & 255) ||
        ((uintptr_t)sgm_dev & 1))
        return SFF_ERR_ARG;
    if (workspace_bytes < seeds_ws_bytes(width, height)) return SFF_ERR_WORKSPACE;
    SeedJob job{reinterpret_cast<const uint2*>(fwd_dev), fwd_cost_dev, keep_dev, cerr_dev, width, height, nullptr,
                nullptr, seeds_dev, capacity, count_dev, sgm_dev, params->tau_c};
    seeds_carve(workspace, width, height, &job.best, &job.chunk);
    return run_seeds(&job, 1, (cudaStream_t)stream);
}
