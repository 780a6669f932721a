// Internal definitions shared by the CUDA translation units of libsff.
//
// Data layout in HBM (one quad of W x H images, S scales):
//   pyramid  [scale][y][x] 48-byte feature records (int8, channel-major),
//            then [scale][y][x] int32 norms (sum of squared features).
//            Three 16-byte loads fetch a record; the norms of neighbouring
//            pixels share cache lines.
//   field    [y][x] int16x4 (u, v, d0, d1): one 8-byte load per pixel.
//   cost     [y][x] int32, SFF_EMPTY_COST where no vector is held yet.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sff.h"

namespace sff {

constexpr int kFeat = SFF_FEATURE_BYTES;
constexpr int kEmpty = SFF_EMPTY_COST;

__host__ __device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

__host__ __device__ __forceinline__ size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// One image at one scale: its feature records and norms.
// One scale of one image's pyramid: the 48-byte record of pixel i as three
// 16-byte chunks, chunk j at f[j * cs + i * rs].  Scale 0 (grid stride 1)
// keeps three chunk planes (cs = W*H, rs = 1): a warp loading one chunk of 32
// nearby pixels' records touches a third of the cache lines, and the other
// colour of the checkerboard uses the rest of every sector.  Coarser scales
// keep whole records side by side (cs = 1, rs = 3): their grid pixels are
// n apart, so half or more of a chunk-plane sector would be a non-grid
// pixel's, and a whole record costs two sectors instead of three.  Measured
// on the 1242x375 quad / the 32-quad batch (M px/s): planes at stride 1 only
// 288.7 / 350.9, at strides 1-2 290.1 / 338.8, at 1-4 288.9 / 316.7, whole
// records everywhere 276.7 / 345.
constexpr int kWholeRecordStride = 2;

__host__ __device__ __forceinline__ bool chunk_planes(int s) { return (1 << s) < kWholeRecordStride; }

struct Plane {
    const int4* f;
    const int* nrm;
    size_t cs;    // chunk stride (int4)
    uint32_t rs;  // record stride (int4)
};

__host__ __device__ __forceinline__ Plane plane_of(const uint8_t* pyr, int s, int S, int w, int h) {
    const size_t np = (size_t)w * h;
    Plane P;
    P.f = reinterpret_cast<const int4*>(pyr + (size_t)s * np * kFeat);
    P.nrm = reinterpret_cast<const int*>(pyr + (size_t)S * np * kFeat) + (size_t)s * np;
    P.cs = chunk_planes(s) ? np : 1;
    P.rs = chunk_planes(s) ? 1 : 3;
    return P;
}

__device__ __forceinline__ const int4* chunk_ptr(const Plane& P, size_t i, int j) { return P.f + j * P.cs + i * P.rs; }
__device__ __forceinline__ int4 chunk_of(const Plane& P, size_t i, int j) { return __ldg(chunk_ptr(P, i, j)); }

// Reference feature held in registers: 12 packed int8x4 words and the norm.
struct RefFeat {
    int a[12];
    int n;
};

__device__ __forceinline__ void load_ref(const Plane& P, size_t i, RefFeat& r) {
    const int4 q0 = chunk_of(P, i, 0), q1 = chunk_of(P, i, 1), q2 = chunk_of(P, i, 2);
    r.a[0] = q0.x; r.a[1] = q0.y; r.a[2] = q0.z; r.a[3] = q0.w;
    r.a[4] = q1.x; r.a[5] = q1.y; r.a[6] = q1.z; r.a[7] = q1.w;
    r.a[8] = q2.x; r.a[9] = q2.y; r.a[10] = q2.z; r.a[11] = q2.w;
    r.n = __ldg(P.nrm + i);
}

// Sum of squared differences of two int8 feature vectors, as
// |a|^2 + |b|^2 - 2 a.b with the dot product on dp4a (exact in int32).
__device__ __forceinline__ int ssd_at(const RefFeat& r, const Plane& P, size_t i) {
    const int4 q0 = chunk_of(P, i, 0), q1 = chunk_of(P, i, 1), q2 = chunk_of(P, i, 2);
    // |b|^2 from the record itself (dp4a, exact): one sector less than
    // loading it from the norm plane
    int nb = 0, d = 0;
    nb = __dp4a(q0.x, q0.x, nb); nb = __dp4a(q0.y, q0.y, nb); nb = __dp4a(q0.z, q0.z, nb); nb = __dp4a(q0.w, q0.w, nb);
    nb = __dp4a(q1.x, q1.x, nb); nb = __dp4a(q1.y, q1.y, nb); nb = __dp4a(q1.z, q1.z, nb); nb = __dp4a(q1.w, q1.w, nb);
    nb = __dp4a(q2.x, q2.x, nb); nb = __dp4a(q2.y, q2.y, nb); nb = __dp4a(q2.z, q2.z, nb); nb = __dp4a(q2.w, q2.w, nb);
    d = __dp4a(r.a[0], q0.x, d); d = __dp4a(r.a[1], q0.y, d);
    d = __dp4a(r.a[2], q0.z, d); d = __dp4a(r.a[3], q0.w, d);
    d = __dp4a(r.a[4], q1.x, d); d = __dp4a(r.a[5], q1.y, d);
    d = __dp4a(r.a[6], q1.z, d); d = __dp4a(r.a[7], q1.w, d);
    d = __dp4a(r.a[8], q2.x, d); d = __dp4a(r.a[9], q2.y, d);
    d = __dp4a(r.a[10], q2.z, d); d = __dp4a(r.a[11], q2.w, d);
    return r.n + nb - 2 * d;
}

// The four views of one field at one scale.
struct Views {
    Plane ref, tmp, ste, crs;
    int w, h, sigma;
};

__device__ __forceinline__ size_t pix(int w, int x, int y) { return (size_t)y * w + x; }

// Eq. 1 with WHT-feature SSD: temporal p+(u,v), stereo p+(-sigma d0, 0),
// cross p+(u - sigma d1, v), positions clamped to the image.
__device__ __forceinline__ int cost_of(const Views& V, const RefFeat& r, int px, int py, int u, int v, int d0,
                                       int d1) {
    int tx = clampi(px + u, 0, V.w - 1);
    int ty = clampi(py + v, 0, V.h - 1);
    int sx = clampi(px - V.sigma * d0, 0, V.w - 1);
    int cx = clampi(px + u - V.sigma * d1, 0, V.w - 1);
    return ssd_at(r, V.tmp, pix(V.w, tx, ty)) + ssd_at(r, V.ste, pix(V.w, sx, py)) +
           ssd_at(r, V.crs, pix(V.w, cx, ty));
}

// Field element pack/unpack: int16x4 in one 64-bit word.
struct Vec4 {
    int u, v, d0, d1;
};

__device__ __forceinline__ Vec4 unpack_vec(uint2 w) {
    Vec4 r;
    r.u = (int)(int16_t)(w.x & 0xffffu);
    r.v = (int)(int16_t)(w.x >> 16);
    r.d0 = (int)(int16_t)(w.y & 0xffffu);
    r.d1 = (int)(int16_t)(w.y >> 16);
    return r;
}

__device__ __forceinline__ uint2 pack_vec(const Vec4& a) {
    uint2 w;
    w.x = ((uint32_t)(uint16_t)a.u) | ((uint32_t)(uint16_t)a.v << 16);
    w.y = ((uint32_t)(uint16_t)a.d0) | ((uint32_t)(uint16_t)a.d1 << 16);
    return w;
}

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplies with xor/permute, key advanced by
// the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Offset of the random search: nearest integer to a uniform value on ]-n, n[,
// from r as floor((floor(r * 4n / 2^32) + 1) / 2) - n.
__device__ __forceinline__ int rs_offset(uint32_t r, int n) {
    uint32_t j = __umulhi(r, (uint32_t)(4 * n));
    return (int)((j + 1) >> 1) - n;
}

// ---------------------------------------------------------------------------
// host-side helpers

// One field to match (Sec. 3.1): its four views' pyramids, its output and
// its scratch (field_ws_bytes).  Fields of any sizes and seeds can share a
// run_fields call.
struct FieldSpec {
    const uint8_t *ref, *tmp, *ste, *crs;
    int16_t* field;
    int32_t* cost;
    int mirror;
    int width, height;
    uint64_t seed;
    void* workspace;
};
// Capacity of the per-launch job tables (kernel parameters): quads per
// shared launch, and the fields and images of that many quads.
#ifndef SFF_TABLE_QUADS
#define SFF_TABLE_QUADS 32
#endif
constexpr int kMaxBatchFields = 2 * SFF_TABLE_QUADS;

// One image of a features launch: input, smoothed scale space (workspace,
// features_ws_bytes) and pyramid.  Up to kMaxImages share a launch.
struct ImageJob {
    const uint8_t* rgb;
    int pitch, w, h;
    uint32_t* sm;
    uint8_t* pyr;
};
constexpr int kMaxImages = 4 * SFF_TABLE_QUADS;
struct ImageJobs {
    ImageJob im[kMaxImages];
};
// Forms of the feature transform (sff_tuning.features_form): separable
// butterflies with each row transform computed once per CTA in shared memory
// (the default), the kept coefficients as a matrix product on the tensor
// cores, or butterflies per pair of vertically adjacent pixels.
constexpr int kFeaturesSeparable = 0, kFeaturesTensor = 1, kFeaturesPairs = 2;
// With smooth = true, smooths the images at scales smooth_lo..smooth_hi
// (< 0: s_lo and s_hi; the range must cover s_lo..s_hi); then computes the
// records of scales s_lo..s_hi (s_hi < 0: the last scale).
int run_features(const ImageJob* jobs, int n, const sff_params& P, cudaStream_t st, int form = kFeaturesSeparable,
                 bool smooth = true, int s_lo = 0, int s_hi = -1, int smooth_lo = -1, int smooth_hi = -1);

// One quad of a consistency-filter / seeds launch (up to kMaxQuads).
struct FilterJob {
    const uint2* fwd;
    const int* fcost;
    const uint2* inv;
    const int* icost;
    int w, h;
    uint8_t* keep;
    uint8_t* cerr;
    int* parent;
    int* size;
    int* joinable;
};
struct SeedJob {
    const uint2* fwd;
    const int* fcost;
    const uint8_t* keep;
    const uint8_t* cerr;
    int w, h;
    int* best;
    int* chunk;
    sff_seed* out;
    int capacity;
    int* count;
    const int16_t* sgm;  // disparity map of the fill (nullptr: joint seeds only)
    int tau_c;           // agreement of d0 with sgm for a disparity-only seed
    // The region filter's last step done by the seed kernels (nullptr: keep is
    // final): a kept pixel whose component (root parent[i]) is joinable and
    // smaller than region_min is removed, in keep_rw (the same mask as keep),
    // before its block is searched.
    const int* parent;
    const int* size;
    const int* joinable;
    int region_min;
    uint8_t* keep_rw;
};
constexpr int kMaxQuads = SFF_TABLE_QUADS;
// remove = false: the filter leaves the removal of small joinable regions to
// the seed kernels (SeedJob::parent ...), which then run on its results.
int run_filter(const FilterJob* jobs, int n, const sff_params& P, cudaStream_t st, bool remove = true);
int run_seeds(const SeedJob* jobs, int n, cudaStream_t st);
void filter_carve(void* workspace, int w, int h, int** parent, int** size, int** joinable);
void seeds_carve(void* workspace, int w, int h, int** best, int** chunk);
size_t field_ws_bytes(int w, int h, const sff_params& p);
// Work issued by the caller of run_fields once the coarsest grid is
// gathered, right before the K-NN launch (fn(ctx, stream); a nonzero status
// ends run_fields with it).
struct ForkHook {
    int (*fn)(void* ctx, cudaStream_t st);
    void* ctx;
};

// scale_ready (optional): per scale s < num_scales - 1, an event that the
// stream waits on before the first launch that reads scale s's records.
int run_fields(const FieldSpec* spec, int nf, const sff_params& P, const sff_tuning& T, cudaStream_t st,
               bool sequential, const cudaEvent_t* scale_ready = nullptr, const ForkHook* fork_hook = nullptr);

// Optional per-kernel event timing (sff_profile_enable).  SFF_LAUNCH wraps
// every kernel launch of the library; a mark pair may also span `launches`
// back-to-back launches of one kernel.
bool profiling();
// units: the work units the span covers (iterations of the iteration kernel);
// -1 = one per launch.
void profile_mark(const char* name, cudaStream_t st, bool after, int launches = 1, int units = -1);

#define SFF_LAUNCH(kernel, grid, block, smem, stream, ...)                       \
    do {                                                                         \
        if (::sff::profiling()) ::sff::profile_mark(#kernel, stream, false);     \
        kernel<<<grid, block, smem, stream>>>(__VA_ARGS__);                      \
        if (::sff::profiling()) ::sff::profile_mark(#kernel, stream, true);      \
    } while (0)

// Device-side condition words (sff_device_status): read and optionally
// cleared in stream order.
int match_status_read(cudaStream_t st, unsigned* out, bool reset);
int seeds_status_read(cudaStream_t st, unsigned* out, bool reset);
int features_status_read(cudaStream_t st, unsigned* out, bool reset);

int check_size(int w, int h);
int check_params(const sff_params* p);
size_t features_ws_bytes(int w, int h, const sff_params& p);
size_t match_ws_bytes(int w, int h, const sff_params& p);
size_t filter_ws_bytes(int w, int h);
size_t seeds_ws_bytes(int w, int h);
int launch_status();

}  // namespace sff
