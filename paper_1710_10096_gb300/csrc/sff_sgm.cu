// Disparity fill (Sec. 3.1, last paragraph): a second disparity map of L0/R0
// by semi-global matching, which verifies the matching's own d0 where the
// joint consistency check removed the pixel (the disparity-only seeds are
// chosen in sff_seeds.cu).
//
// SGM as this library reads it (the paper gives no details):
//   grey = (R + 2G + B + 2) >> 2; census over a 9 x 7 window, bit k (row-major
//   window order, centre skipped) set when the neighbour is darker than the
//   centre, coordinates clamped; cost C(p, d) = popcount(census_L(x, y) ^
//   census_R(max(x - d, 0), y)); 8 directions r (4 axes, 4 diagonals)
//     L_r(p, d) = C(p, d) + min(L_r(p-r, d), L_r(p-r, d+-1) + P1,
//                               min_k L_r(p-r, k) + P2) - min_k L_r(p-r, k),
//   L_r(p, d) = C(p, d) at the first pixel of a path; disparity = argmin_d of
//   sum_r L_r(p, d), ties to the lowest d.
//
// L_r(p, d) lies in [0, 62 + P2], so with P2 <= 193 it is stored exactly in
// one byte.
//
// k_sgm_census: grey and census of both images from a shared-memory tile.
// k_sgm_cost:   the cost volume, one byte per pixel and disparity (a path
//               step then reads D bytes instead of D census words).
// k_sgm_paths:  one warp per path line of one direction (blockIdx.z), the
//               lanes holding D / 32 consecutive disparities each; one step
//               per pixel, the costs of the next 32 pixels of the line in
//               flight into a shared-memory ring (cp.async): the
//               neighbours' d +- 1 values by shuffles, the minimum over d
//               by one redux; L_r to [dir][y][x][d].
// k_sgm_wta:    one warp per pixel: the 8 directions summed per disparity,
//               the (sum, d) minimum by a warp reduction.
#include "sff_internal.cuh"

namespace sff {
namespace {

constexpr int kDirs = 8;
constexpr int kPathWarps = 4;  // warps (lines) per CTA of k_sgm_paths
constexpr int kRing = 32;      // pixels whose costs a path warp has in flight (shared-memory ring)
constexpr int kWtaWarps = 8;   // warps (pixels) per CTA of k_sgm_wta
constexpr int kCensusW = 9, kCensusH = 7;
constexpr int kTileX = 32, kTileY = 8;
constexpr int kInf = 1 << 20;
constexpr unsigned kFull = 0xffffffffu;

struct SgmJob {
    const uint8_t* img[2];  // L0, R0
    int pitch, w, h, D, p1, p2;
    uint64_t* census[2];    // [y][x]
    uint8_t* cost;          // [y][x][D] matching costs
    uint8_t* paths;         // [dir][y][x][D]
    int16_t* disp;          // [y][x]
};

__constant__ int c_dir[kDirs][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

__global__ void __launch_bounds__(kTileX * kTileY) k_sgm_census(SgmJob S) {
    constexpr int TW = kTileX + kCensusW - 1, TH = kTileY + kCensusH - 1;
    __shared__ uint8_t tile[TH][TW];
    const uint8_t* img = blockIdx.z ? S.img[1] : S.img[0];  // no dynamic index into the parameter
    const int x0 = blockIdx.x * kTileX - kCensusW / 2, y0 = blockIdx.y * kTileY - kCensusH / 2;
    for (int k = threadIdx.y * kTileX + threadIdx.x; k < TW * TH; k += kTileX * kTileY) {
        const int tx = k % TW, ty = k / TW;
        const int gx = clampi(x0 + tx, 0, S.w - 1), gy = clampi(y0 + ty, 0, S.h - 1);
        const uint8_t* p = img + (size_t)gy * S.pitch + 3 * gx;
        tile[ty][tx] = (uint8_t)((p[0] + 2 * p[1] + p[2] + 2) >> 2);
    }
    __syncthreads();
    const int x = blockIdx.x * kTileX + threadIdx.x, y = blockIdx.y * kTileY + threadIdx.y;
    if (x >= S.w || y >= S.h) return;
    const int c = tile[threadIdx.y + kCensusH / 2][threadIdx.x + kCensusW / 2];
    uint64_t bits = 0;
    int k = 0;
#pragma unroll
    for (int j = 0; j < kCensusH; ++j)
#pragma unroll
        for (int i = 0; i < kCensusW; ++i) {
            if (i == kCensusW / 2 && j == kCensusH / 2) continue;
            bits |= (uint64_t)(tile[threadIdx.y + j][threadIdx.x + i] < c) << k;
            ++k;
        }
    (blockIdx.z ? S.census[1] : S.census[0])[(size_t)y * S.w + x] = bits;
}

template <int J>
__device__ __forceinline__ void store_bytes(uint8_t* p, const int (&v)[J]) {
    if constexpr (J == 1) {
        *p = (uint8_t)v[0];
    } else if constexpr (J == 2) {
        *reinterpret_cast<uint16_t*>(p) = (uint16_t)(v[0] | (v[1] << 8));
    } else if constexpr (J == 4) {
        *reinterpret_cast<uint32_t*>(p) = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) |
                                          ((uint32_t)v[3] << 24);
    } else {
        static_assert(J == 8, "D = 32, 64, 128 or 256");
        uint2 w;
        w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
        w.y = (uint32_t)v[4] | ((uint32_t)v[5] << 8) | ((uint32_t)v[6] << 16) | ((uint32_t)v[7] << 24);
        *reinterpret_cast<uint2*>(p) = w;
    }
}

// J bytes as one machine word (kept packed while loads are in flight).
template <int J>
struct RawOf;
template <>
struct RawOf<1> { using T = uint8_t; };
template <>
struct RawOf<2> { using T = uint16_t; };
template <>
struct RawOf<4> { using T = uint32_t; };
template <>
struct RawOf<8> { using T = uint2; };

template <int J>
__device__ __forceinline__ typename RawOf<J>::T load_raw(const uint8_t* q) {
    return *reinterpret_cast<const typename RawOf<J>::T*>(q);
}

template <int J>
__device__ __forceinline__ void unpack(typename RawOf<J>::T t, int (&v)[J]) {
    if constexpr (J == 8) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (t.x >> (8 * j)) & 0xff;
            v[4 + j] = (t.y >> (8 * j)) & 0xff;
        }
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j) v[j] = ((uint32_t)t >> (8 * j)) & 0xff;
    }
}

template <int J>
__device__ __forceinline__ void load_bytes(const uint8_t* q, int (&v)[J]) {
    if constexpr (J == 1) {
        v[0] = q[0];
    } else if constexpr (J == 2) {
        const uint16_t t = *reinterpret_cast<const uint16_t*>(q);
        v[0] = t & 0xff;
        v[1] = t >> 8;
    } else if constexpr (J == 4) {
        const uint32_t t = *reinterpret_cast<const uint32_t*>(q);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (t >> (8 * j)) & 0xff;
    } else {
        const uint2 t = *reinterpret_cast<const uint2*>(q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (t.x >> (8 * j)) & 0xff;
            v[4 + j] = (t.y >> (8 * j)) & 0xff;
        }
    }
}

// C(p, d) for every pixel.  One CTA per segment of kCostSeg pixels of a row:
// the right image's census words the segment needs (x - D + 1 .. the
// segment's end, positions clamped at 0) are staged in shared memory once;
// each warp then takes pixels of the segment, J disparities per lane, the
// J costs of a lane packed into J bytes of [y][x][d].
constexpr int kCostSeg = 64;
constexpr int kCostThreads = 256;

template <int J>
__global__ void __launch_bounds__(kCostThreads) k_sgm_cost(SgmJob S) {
    constexpr int D = 32 * J;
    __shared__ uint64_t right[kCostSeg + D - 1];
    const int y = blockIdx.y, x0 = blockIdx.x * kCostSeg;
    const uint64_t* rrow = S.census[1] + (size_t)y * S.w;
    const int base = x0 - (D - 1);  // census position of right[0]
    for (int i = threadIdx.x; i < kCostSeg + D - 1; i += kCostThreads)
        right[i] = rrow[min(max(base + i, 0), S.w - 1)];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < kCostSeg; k += kCostThreads / 32) {
        const int x = x0 + k;
        if (x >= S.w) break;  // uniform over the warp
        const size_t p = (size_t)y * S.w + x;
        const uint64_t c = S.census[0][p];
        int v[J];
#pragma unroll
        for (int j = 0; j < J; ++j) v[j] = __popcll(c ^ right[max(x - (lane * J + j), 0) - base]);
        store_bytes<J>(S.cost + p * D + lane * J, v);
    }
}

template <int J>
__global__ void __launch_bounds__(kPathWarps * 32) k_sgm_paths(SgmJob S) {
    const int dir = blockIdx.z;
    const int rx = c_dir[dir][0], ry = c_dir[dir][1];
    const int lane = threadIdx.x & 31;
    const int line = blockIdx.x * kPathWarps + (threadIdx.x >> 5);
    const int W = S.w, H = S.h, D = S.D;
    // the line's first pixel: the pixels whose predecessor is outside the image
    int x, y, nlines;
    if (ry == 0) {
        nlines = H;
        y = line;
        x = rx > 0 ? 0 : W - 1;
    } else if (rx == 0) {
        nlines = W;
        x = line;
        y = ry > 0 ? 0 : H - 1;
    } else {
        nlines = W + H - 1;
        if (line < W) {
            x = line;
            y = ry > 0 ? 0 : H - 1;
        } else {
            x = rx > 0 ? 0 : W - 1;
            y = ry > 0 ? 1 + (line - W) : H - 2 - (line - W);
        }
    }
    if (line >= nlines) return;  // warp-uniform
    uint8_t* out = S.paths + (size_t)dir * W * H * D + lane * J;
    // steps until the line leaves the image
    const int n = min(rx > 0 ? W - x : rx < 0 ? x + 1 : 1 << 30, ry > 0 ? H - y : ry < 0 ? y + 1 : 1 << 30);
    const ptrdiff_t step = (ptrdiff_t)ry * W + rx;  // pixel index increment along the line
    const size_t p0 = (size_t)y * W + x;
    // The costs of the next kRing pixels of the line stream into a ring in
    // shared memory with cp.async (one commit group per pixel, so a step
    // waits only for its own pixel's group); the copy is spread over the
    // lanes in 4-byte pieces.
    extern __shared__ __align__(16) uint8_t ring_all[];
    uint8_t* ring = ring_all + (size_t)(threadIdx.x >> 5) * kRing * D;
    const uint8_t* line_cost = S.cost;
    auto fetch = [&](int t) {  // pixel t of the line into its ring slot
        if (t < n) {
            const uint8_t* src = line_cost + (p0 + (ptrdiff_t)t * step) * D;
            uint8_t* dst = ring + (t % kRing) * D;
            for (int b = 4 * lane; b < D; b += 128) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + b);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src + b) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int t = 0; t < kRing; ++t) fetch(t);
    auto take = [&](int t) {  // pixel t's costs, this lane's J bytes
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 1) : "memory");
        __syncwarp();
        const typename RawOf<J>::T r = load_raw<J>(ring + (t % kRing) * D + lane * J);
        __syncwarp();  // every lane has read the slot before it is refilled
        fetch(t + kRing);
        return r;
    };
    if constexpr (J == 1) {
        int prev = 0, m = 0;
        for (int t = 0; t < n; ++t) {
            {
                {
                    const size_t p = p0 + (ptrdiff_t)t * step;
                    int cur[1];
                    unpack<1>(take(t), cur);
                    if (t > 0) {
                        const int lo = __shfl_up_sync(kFull, prev, 1), hi = __shfl_down_sync(kFull, prev, 1);
                        const int pl = lane > 0 ? lo : kInf, pr = lane < 31 ? hi : kInf;
                        cur[0] += min(min(prev, min(pl, pr) + S.p1), m + S.p2) - m;
                    }
                    store_bytes<1>(out + p * D, cur);
                    m = __reduce_min_sync(kFull, cur[0]);
                    prev = cur[0];
                }
            }
        }
    } else {
        // Two disparities per 32-bit word (16-bit halves; every value stays
        // below 2^16 and every difference taken is >= 0, so plain 32-bit
        // adds and subtracts act on both halves) and the recurrence on the
        // DPX add-min instructions:
        //   min(P, Lm + P1, Rp + P1, m + P2) = min(min(Lm + P1, m + P2),
        //                                          min(Rp + P1, P)).
        // Lm / Rp: the pair of each half's d - 1 / d + 1 values, from byte
        // permutes of neighbouring pairs (the outer ones from the
        // neighbouring lanes); beyond the disparity range 0x7fff.
        constexpr int NP = J / 2;
        const uint32_t p1x2 = (uint32_t)S.p1 * 0x00010001u;
        uint32_t prev[NP];
        uint32_t m = 0;
        for (int t = 0; t < n; ++t) {
            {
                {
                    const size_t p = p0 + (ptrdiff_t)t * step;
                    const typename RawOf<J>::T raw = take(t);
                    uint32_t c2[NP];  // costs as 16-bit pairs
                    if constexpr (J == 2) {
                        c2[0] = __byte_perm((uint32_t)raw, 0u, 0x4140);
                    } else if constexpr (J == 4) {
                        c2[0] = __byte_perm((uint32_t)raw, 0u, 0x4140);
                        c2[1] = __byte_perm((uint32_t)raw, 0u, 0x4342);
                    } else {
                        c2[0] = __byte_perm(raw.x, 0u, 0x4140);
                        c2[1] = __byte_perm(raw.x, 0u, 0x4342);
                        c2[2] = __byte_perm(raw.y, 0u, 0x4140);
                        c2[3] = __byte_perm(raw.y, 0u, 0x4342);
                    }
                    uint32_t cur[NP];
                    if (t > 0) {
                        const uint32_t lo = __shfl_up_sync(kFull, prev[NP - 1], 1);  // its high half: d = lane J - 1
                        const uint32_t hi = __shfl_down_sync(kFull, prev[0], 1);     // its low half: d = lane J + J
                        const uint32_t left = lane > 0 ? lo : 0x7fff0000u, right = lane < 31 ? hi : 0x00007fffu;
                        const uint32_t mp2 = (m + (uint32_t)S.p2) * 0x00010001u, m2 = m * 0x00010001u;
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            const uint32_t lm = __byte_perm(j > 0 ? prev[j - 1] : left, prev[j], 0x5432);
                            const uint32_t rp = __byte_perm(prev[j], j < NP - 1 ? prev[j + 1] : right, 0x5432);
                            const uint32_t b = __vminu2(__viaddmin_u16x2(lm, p1x2, mp2),
                                                             __viaddmin_u16x2(rp, p1x2, prev[j]));
                            cur[j] = b + c2[j] - m2;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NP; ++j) cur[j] = c2[j];
                    }
                    // back to bytes (every value < 256)
                    if constexpr (J == 2) {
                        *reinterpret_cast<uint16_t*>(out + p * D) = (uint16_t)__byte_perm(cur[0], 0u, 0x4420);
                    } else if constexpr (J == 4) {
                        *reinterpret_cast<uint32_t*>(out + p * D) = __byte_perm(cur[0], cur[1], 0x6420);
                    } else {
                        *reinterpret_cast<uint2*>(out + p * D) =
                            make_uint2(__byte_perm(cur[0], cur[1], 0x6420), __byte_perm(cur[2], cur[3], 0x6420));
                    }
                    uint32_t mm = cur[0];
#pragma unroll
                    for (int j = 1; j < NP; ++j) mm = __vminu2(mm, cur[j]);
                    m = __reduce_min_sync(kFull, min(mm & 0xffffu, mm >> 16));
#pragma unroll
                    for (int j = 0; j < NP; ++j) prev[j] = cur[j];
                }
            }
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int J>
__global__ void __launch_bounds__(kWtaWarps * 32) k_sgm_wta(SgmJob S) {
    const int lane = threadIdx.x & 31;
    const size_t p = (size_t)blockIdx.x * kWtaWarps + (threadIdx.x >> 5);
    const size_t np = (size_t)S.w * S.h;
    if (p >= np) return;  // warp-uniform
    int sum[J];
#pragma unroll
    for (int j = 0; j < J; ++j) sum[j] = 0;
#pragma unroll
    for (int r = 0; r < kDirs; ++r) {
        int v[J];
        load_bytes<J>(S.paths + ((size_t)r * np + p) * S.D + lane * J, v);
#pragma unroll
        for (int j = 0; j < J; ++j) sum[j] += v[j];
    }
    // key = sum << 8 | d: the smallest key is the lowest sum, then the lowest d
    unsigned key = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < J; ++j) key = min(key, ((unsigned)sum[j] << 8) | (unsigned)(lane * J + j));
    key = __reduce_min_sync(kFull, key);
    if (lane == 0) S.disp[p] = (int16_t)(key & 0xff);
}

int check_sgm(const sff_sgm_params* P) {
    if (!P) return SFF_ERR_ARG;
    if (P->max_disp != 32 && P->max_disp != 64 && P->max_disp != 128 && P->max_disp != 256) return SFF_ERR_ARG;
    if (P->p1 < 0 || P->p2 < P->p1 || P->p2 > 193) return SFF_ERR_ARG;
    return SFF_OK;
}

struct SgmLayout {
    size_t census0, census1, cost, paths, total;
};

SgmLayout sgm_layout(int w, int h, int D) {
    const size_t np = (size_t)w * h;
    SgmLayout L;
    L.census0 = 0;
    L.census1 = align256(np * 8);
    L.cost = L.census1 + align256(np * 8);
    L.paths = L.cost + align256(np * D);
    L.total = L.paths + align256(np * kDirs * D);
    return L;
}

template <int J>
int launch_sgm(const SgmJob& S, cudaStream_t st) {
    const size_t np = (size_t)S.w * S.h;
    SFF_LAUNCH(k_sgm_cost<J>, dim3((S.w + kCostSeg - 1) / kCostSeg, S.h), kCostThreads, 0, st, S);
    const int lines = S.w + S.h - 1;  // the diagonals have the most lines
    const size_t ring = (size_t)kPathWarps * kRing * S.D;
    if (ring > 48 * 1024 &&
        cudaFuncSetAttribute(k_sgm_paths<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring) != cudaSuccess)
        return SFF_ERR_CUDA;
    SFF_LAUNCH(k_sgm_paths<J>, dim3((lines + kPathWarps - 1) / kPathWarps, 1, kDirs), kPathWarps * 32, ring, st, S);
    SFF_LAUNCH(k_sgm_wta<J>, dim3((unsigned)((np + kWtaWarps - 1) / kWtaWarps)), kWtaWarps * 32, 0, st, S);
    return SFF_OK;
}

}  // namespace
}  // namespace sff

extern "C" int sff_default_sgm_params(sff_sgm_params* out) {
    if (!out) return SFF_ERR_ARG;
    out->max_disp = 128;
    out->p1 = 10;
    out->p2 = 120;
    return SFF_OK;
}

extern "C" size_t sff_sgm_workspace_bytes(int32_t width, int32_t height, const sff_sgm_params* params) {
    if (sff::check_size(width, height) || sff::check_sgm(params)) return 0;
    return sff::sgm_layout(width, height, params->max_disp).total;
}

extern "C" int sff_sgm(const uint8_t* left_dev, const uint8_t* right_dev, int32_t pitch_bytes, int32_t width,
                       int32_t height, const sff_sgm_params* params, int16_t* disp_dev, void* workspace,
                       size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_sgm(params)) return SFF_ERR_ARG;
    if (!left_dev || !right_dev || !disp_dev || !workspace || pitch_bytes < 3 * width) return SFF_ERR_ARG;
    if (((uintptr_t)disp_dev & 1) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    const SgmLayout L = sgm_layout(width, height, params->max_disp);
    if (workspace_bytes < L.total) return SFF_ERR_WORKSPACE;
    char* ws = reinterpret_cast<char*>(workspace);
    SgmJob S;
    S.img[0] = left_dev;
    S.img[1] = right_dev;
    S.pitch = pitch_bytes;
    S.w = width;
    S.h = height;
    S.D = params->max_disp;
    S.p1 = params->p1;
    S.p2 = params->p2;
    S.census[0] = reinterpret_cast<uint64_t*>(ws + L.census0);
    S.census[1] = reinterpret_cast<uint64_t*>(ws + L.census1);
    S.cost = reinterpret_cast<uint8_t*>(ws + L.cost);
    S.paths = reinterpret_cast<uint8_t*>(ws + L.paths);
    S.disp = disp_dev;
    cudaStream_t st = (cudaStream_t)stream;
    SFF_LAUNCH(k_sgm_census, dim3((width + kTileX - 1) / kTileX, (height + kTileY - 1) / kTileY, 2),
               dim3(kTileX, kTileY), 0, st, S);
    const int rc = S.D == 32 ? launch_sgm<1>(S, st) : S.D == 64 ? launch_sgm<2>(S, st)
                   : S.D == 128 ? launch_sgm<4>(S, st) : launch_sgm<8>(S, st);
    return rc != SFF_OK ? rc : launch_status();
}
