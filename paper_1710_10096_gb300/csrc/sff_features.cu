// Walsh-Hadamard patch features on the box-smoothed scale space
// (Sec. 3.1, "Initialization" and "Multi-Scale Propagation").
//
// k_smooth:   S_s for every scale, one thread per pixel, RGB packed in one
//             uint32 per pixel (workspace [S][H][W]).
// k_features: one thread per pixel and scale; the 8x8 patch of each channel
//             is transformed separably with 8-point fast Walsh-Hadamard
//             butterflies (natural order), R and G packed into one int32 as
//             R + 65536 G (every intermediate stays below 2^31 in magnitude,
//             so packed adds and subtracts are exact).  The 16 kept
//             coefficients are read out through the sequency->natural index
//             map, quantised and written as one 48-byte record plus its norm.
#include <mutex>

#include "sff_internal.cuh"

namespace sff {
namespace {

// Natural-order Hadamard row of sequency k: bitreverse3(gray(k)).
__host__ __device__ constexpr int seq_to_nat(int k) {
    return (((k ^ (k >> 1)) & 1) << 2) | ((k ^ (k >> 1)) & 2) | (((k ^ (k >> 1)) >> 2) & 1);
}

// Kept coefficient m = 0..15 as (ky, kx): AC entries by ky+kx, then ky.
// Diagonal t = ky+kx holds t+1 entries and starts after 1+2+..+t - 1 = t(t+1)/2 - 1 of them.
__host__ __device__ constexpr int diag_of(int m) { return m < 2 ? 1 : m < 5 ? 2 : m < 9 ? 3 : m < 14 ? 4 : 5; }
__host__ __device__ constexpr int order_ky(int m) { return m - (diag_of(m) * (diag_of(m) + 1) / 2 - 1); }
__host__ __device__ constexpr int order_kx(int m) { return diag_of(m) - order_ky(m); }
static_assert(seq_to_nat(1) == 4 && seq_to_nat(2) == 6 && seq_to_nat(5) == 7 && seq_to_nat(7) == 1, "walsh map");
static_assert(order_ky(0) == 0 && order_kx(0) == 1 && order_ky(4) == 2 && order_kx(4) == 0, "order");
static_assert(order_ky(13) == 4 && order_kx(13) == 0 && order_ky(15) == 1 && order_kx(15) == 4, "order");

__global__ void k_smooth(const __grid_constant__ ImageJobs J, int S) {
    const ImageJob& job = J.im[blockIdx.z];
    const uint8_t* __restrict__ rgb = job.rgb;
    const int pitch = job.pitch, w = job.w, h = job.h;
    uint32_t* __restrict__ out = job.sm;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= w || y >= h) return;
    {
        const uint8_t* p = rgb + (size_t)y * pitch + 3 * x;
        out[(size_t)y * w + x] = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
    }
    for (int s = 1; s < S; ++s) {
        int n = 1 << s;
        uint32_t sr = 0, sg = 0, sb = 0;
        for (int j = -n / 2; j < n / 2; ++j) {
            const uint8_t* row = rgb + (size_t)clampi(y + j, 0, h - 1) * pitch;
            for (int i = -n / 2; i < n / 2; ++i) {
                const uint8_t* p = row + 3 * clampi(x + i, 0, w - 1);
                sr += p[0];
                sg += p[1];
                sb += p[2];
            }
        }
        uint32_t half = (uint32_t)(n * n / 2);
        uint32_t r = (sr + half) >> (2 * s), g = (sg + half) >> (2 * s), b = (sb + half) >> (2 * s);
        out[((size_t)s * h + y) * w + x] = r | (g << 8) | (b << 16);
    }
}

__device__ __forceinline__ void fwht8(int (&a)[8]) {
#pragma unroll
    for (int hstep = 1; hstep < 8; hstep <<= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if ((i & hstep) == 0) {
                int x = a[i], y = a[i + hstep];
                a[i] = x + y;
                a[i + hstep] = x - y;
            }
}

__device__ __forceinline__ int lo16(int x) { return (x << 16) >> 16; }

__global__ void k_features(const __grid_constant__ ImageJobs J, int s, int S, int qshift) {
    const ImageJob& job = J.im[blockIdx.z];
    const int w = job.w, h = job.h;
    const size_t np = (size_t)w * h;
    const uint32_t* __restrict__ sm = job.sm + s * np;
    uint8_t* __restrict__ out = job.pyr + s * np * kFeat;
    int* __restrict__ norm_out = reinterpret_cast<int*>(job.pyr + (size_t)S * np * kFeat) + s * np;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= w || y >= h) return;
    const int n = 1 << s;
    int xs[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xs[j] = clampi(x + n * (j - 3), 0, w - 1);

    // row transforms: keep the natural columns of sequency kx = 0..5
    int rg[8][6], bb[8][6];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t* row = sm + (size_t)clampi(y + n * (i - 3), 0, h - 1) * w;
        int a[8], b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t px = __ldg(row + xs[j]);
            a[j] = (int)(px & 0xffu) + 65536 * (int)((px >> 8) & 0xffu);
            b[j] = (int)((px >> 16) & 0xffu);
        }
        fwht8(a);
        fwht8(b);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            rg[i][k] = a[seq_to_nat(k)];
            bb[i][k] = b[seq_to_nat(k)];
        }
    }
    // column transforms
    int crg[8][6], cb[8][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            a[i] = rg[i][k];
            b[i] = bb[i][k];
        }
        fwht8(a);
        fwht8(b);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            crg[i][k] = a[i];
            cb[i][k] = b[i];
        }
    }
    // read out, quantise, pack
    int8_t f[48];
    int norm = 0;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        int X = crg[seq_to_nat(order_ky(m))][order_kx(m)];
        int r = lo16(X);
        int g = (X - r) >> 16;
        int b = cb[seq_to_nat(order_ky(m))][order_kx(m)];
        int q[3] = {r, g, b};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int v = clampi(q[c] >> qshift, -128, 127);
            f[c * 16 + m] = (int8_t)v;
            norm += v * v;
        }
    }
    int words[12];
#pragma unroll
    for (int k = 0; k < 12; ++k)
        words[k] = (int)((uint32_t)(uint8_t)f[4 * k] | ((uint32_t)(uint8_t)f[4 * k + 1] << 8) |
                         ((uint32_t)(uint8_t)f[4 * k + 2] << 16) | ((uint32_t)(uint8_t)f[4 * k + 3] << 24));
    const size_t i = (size_t)y * w + x;
    int4* dst = reinterpret_cast<int4*>(out + i * kFeat);
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[k] = make_int4(words[4 * k], words[4 * k + 1], words[4 * k + 2], words[4 * k + 3]);
    norm_out[i] = norm;
}

}  // namespace

size_t features_ws_bytes(int w, int h, const sff_params& p) {
    return align256((size_t)p.num_scales * w * h * sizeof(uint32_t));
}

int run_features(const ImageJob* jobs, int n, const sff_params& P, cudaStream_t st) {
    if (n < 1 || n > kMaxImages) return SFF_ERR_ARG;
    static ImageJobs J;  // host staging of the kernel parameter (copied at each launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    int mw = 0, mh = 0;
    for (int k = 0; k < n; ++k) {
        J.im[k] = jobs[k];
        mw = mw > jobs[k].w ? mw : jobs[k].w;
        mh = mh > jobs[k].h ? mh : jobs[k].h;
    }
    dim3 blk(128), grd((mw + 127) / 128, mh, n);
    SFF_LAUNCH(k_smooth, grd, blk, 0, st, J, P.num_scales);
    for (int s = 0; s < P.num_scales; ++s) SFF_LAUNCH(k_features, grd, blk, 0, st, J, s, P.num_scales, P.quant_shift);
    return launch_status();
}

}  // namespace sff

extern "C" int sff_features(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                            const sff_params* params, uint8_t* pyramid_dev, void* workspace,
                            size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!rgb_dev || !pyramid_dev || !workspace || pitch_bytes < 3 * width) return SFF_ERR_ARG;
    if (((uintptr_t)pyramid_dev & 15) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < features_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    ImageJob job{rgb_dev, pitch_bytes, width, height, (uint32_t*)workspace, pyramid_dev};
    return run_features(&job, 1, *params, (cudaStream_t)stream);
}
