// Features of the paper's own matching cost (Sec. 3.1, "Matching Cost",
// Eq. 1): per pixel and scale the first three principal components phi of a
// dense SIFT descriptor, the principal axes computed over the descriptors of
// all four images.
//
// Readings (the paper names SIFTFlow's dense SIFT and the three principal
// components, nothing more):
//   - grey (R + 2G + B + 2) >> 2 of the scale's box-smoothed image (the
//     smoothing of the WHT features: n x n box, window -n/2 .. n/2 - 1,
//     clamped, rounded half up per channel);
//   - gradient with stride n, central differences, clamped; magnitude
//     sqrt(dx^2 + dy^2) in single precision; orientation sector k of 45
//     degrees by exact integer cross products with the sector rays;
//   - 4 x 4 cells of 3 x 3 samples at stride n around the pixel (offsets
//     -6 n .. 5 n, clamped), each cell's 8 bins summing its samples in
//     row-major order; 128 sums normalised, clipped at 0.2, renormalised,
//     quantised to min(255, (int)(v 512 + 0.5));
//   - axes: exact integer sums over the full-resolution descriptors of the
//     four images, covariance in double precision, 200 power iterations per
//     axis from the all-ones vector with deflation, sign of the largest
//     component positive; each dot product of an iteration as four partial
//     sums over the indices mod 4, each by fused multiply-adds in index
//     order, combined as (s0 + s1) + (s2 + s3);
//   - phi_c = sum_k fl(a_ck) q_k in single precision, minus fl(a_c . mean).
// Every floating-point operation is written out with the _rn intrinsics, in
// the order of the definition: fused multiply-adds only where the definition
// names them (the power iteration's dot products), no reassociation, so the
// results are reproducible bit for bit on any IEEE machine.
//
// k_sift_grey:    smoothed grey image of one scale (4 images, blockIdx.z).
// k_sift_grad:    magnitude and orientation sector per pixel.
// k_sift_desc:    the quantised descriptor, four threads per pixel with 32
//                 sums each in registers; the norms handed along in bin order.
// k_sift_cov:     64 descriptors per step in shared memory, transposed;
//                 every thread accumulates 64 of the 128 x 128 products with
//                 dp4a, flushed into 64-bit sums.
// k_sift_axes:    one CTA: mean, covariance, power iterations, projection
//                 weights.
// k_sift_project: phi of every pixel of one scale of the four images.
#include <algorithm>

#include "sff_internal.cuh"

namespace sff {
namespace {

constexpr int kDesc = 128;
constexpr int kDescThreads = 128;  // threads of k_sift_desc: 32 pixels, four threads each
constexpr int kCovPix = 64;       // descriptors per step of k_sift_cov
constexpr int kCovThreads = 256;
constexpr int kCovFlush = 16384;  // descriptors between flushes of the 32-bit partial sums
constexpr int kPowerIters = 200;

struct SiftJob {
    const uint8_t* rgb[4];
    int pitch, w, h, s, n;
    uint8_t* grey;           // [4][H][W]
    float* mag;              // [4][H][W]
    uint8_t* bin;            // [4][H][W]
    uint8_t* desc;           // [4][H][W][128]
    unsigned long long* s1;  // [128] sums
    unsigned long long* s2;  // [128][128] sums of products
    double* axes;            // [3][128]
    float* proj;             // [3][128] single-precision axes, then [3] biases
    float* phi[4];           // [S][H][W][4] each
};

__device__ __forceinline__ const uint8_t* img_of(const SiftJob& J, int v) {
    return v == 0 ? J.rgb[0] : v == 1 ? J.rgb[1] : v == 2 ? J.rgb[2] : J.rgb[3];
}
__device__ __forceinline__ float* phi_of(const SiftJob& J, int v) {
    return v == 0 ? J.phi[0] : v == 1 ? J.phi[1] : v == 2 ? J.phi[2] : J.phi[3];
}

__global__ void k_sift_grey(SiftJob J) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, v = blockIdx.z;
    if (x >= J.w) return;
    const uint8_t* img = img_of(J, v);
    int c[3];
    if (J.n == 1) {
        const uint8_t* p = img + (size_t)y * J.pitch + 3 * x;
        c[0] = p[0];
        c[1] = p[1];
        c[2] = p[2];
    } else {
        int sum[3] = {0, 0, 0};
        for (int j = -J.n / 2; j <= J.n / 2 - 1; ++j)
            for (int i = -J.n / 2; i <= J.n / 2 - 1; ++i) {
                const uint8_t* p = img + (size_t)clampi(y + j, 0, J.h - 1) * J.pitch + 3 * clampi(x + i, 0, J.w - 1);
                sum[0] += p[0];
                sum[1] += p[1];
                sum[2] += p[2];
            }
        const int a = J.n * J.n;
        for (int k = 0; k < 3; ++k) c[k] = (sum[k] + a / 2) / a;
    }
    J.grey[((size_t)v * J.h + y) * J.w + x] = (uint8_t)((c[0] + 2 * c[1] + c[2] + 2) >> 2);
}

// Sector k of a direction: the rays of the sector boundaries are 45 degrees
// apart; the direction lies in [ray k, ray k+1) exactly when its cross
// product with ray k is >= 0 and with ray k+1 is < 0.
__device__ __forceinline__ int sector_of(int dx, int dy) {
    constexpr int rx[9] = {1, 1, 0, -1, -1, -1, 0, 1, 1}, ry[9] = {0, 1, 1, 1, 0, -1, -1, -1, 0};
    int k = 0;
#pragma unroll
    for (int t = 7; t >= 0; --t)
        if (rx[t] * dy - ry[t] * dx >= 0 && rx[t + 1] * dy - ry[t + 1] * dx < 0) k = t;
    return k;
}

__global__ void k_sift_grad(SiftJob J) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, v = blockIdx.z;
    if (x >= J.w) return;
    const uint8_t* g = J.grey + (size_t)v * J.h * J.w;
    const int dx = (int)g[(size_t)y * J.w + min(x + J.n, J.w - 1)] - (int)g[(size_t)y * J.w + max(x - J.n, 0)];
    const int dy = (int)g[(size_t)min(y + J.n, J.h - 1) * J.w + x] - (int)g[(size_t)max(y - J.n, 0) * J.w + x];
    const size_t o = ((size_t)v * J.h + y) * J.w + x;
    J.mag[o] = __fsqrt_rn((float)(dx * dx + dy * dy));
    J.bin[o] = (uint8_t)sector_of(dx, dy);
}

// Sum of squares of the 128 values of a pixel's four-thread group in bin
// order: thread r of the group holds bins 32 r .. 32 r + 31 and continues
// the running sum of threads 0 .. r - 1, so the sum is the sequential one.
// Every lane of the warp calls it.
__device__ __forceinline__ float group_sum_sq(const float (&h)[32], int r, int lane) {
    float ss = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (r == q) {
#pragma unroll
            for (int b = 0; b < 32; ++b) ss = __fadd_rn(ss, __fmul_rn(h[b], h[b]));
        }
        ss = __shfl_sync(0xffffffffu, ss, (lane & ~3) | q);
    }
    return ss;
}

// The descriptor of one pixel per four threads: thread r of the group holds
// the 32 sums of cell row r (bins 32 r .. 32 r + 31 in descriptor order) in
// registers.  A bin's sum adds +0 for the samples of the other sectors,
// which leaves it bit-identical to adding only its own samples.  Threads
// past the image's edge compute on the last column and store nothing, so
// that every lane takes part in the shuffles.
__global__ void __launch_bounds__(kDescThreads, 7) k_sift_desc(SiftJob J) {
    const int lane = threadIdx.x & 31, r = threadIdx.x & 3;
    const int x = blockIdx.x * (kDescThreads / 4) + (threadIdx.x >> 2), y = blockIdx.y, v = blockIdx.z;
    const bool valid = x < J.w;
    const int xs = valid ? x : J.w - 1;
    const size_t plane = (size_t)v * J.h * J.w;
    const float* mag = J.mag + plane;
    const uint8_t* bin = J.bin + plane;
    float h[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) h[b] = 0.0f;
#pragma unroll
    for (int sj = 0; sj < 3; ++sj) {
        const int qy = clampi(y + (r * 3 + sj - 6) * J.n, 0, J.h - 1);
        const float* mrow = mag + (size_t)qy * J.w;
        const uint8_t* brow = bin + (size_t)qy * J.w;
#pragma unroll
        for (int cx = 0; cx < 4; ++cx)
#pragma unroll
            for (int si = 0; si < 3; ++si) {
                const int qx = clampi(xs + (cx * 3 + si - 6) * J.n, 0, J.w - 1);
                const float m = mrow[qx];
                const int k = brow[qx];
#pragma unroll
                for (int b = 0; b < 8; ++b) h[cx * 8 + b] = __fadd_rn(h[cx * 8 + b], k == b ? m : 0.0f);
            }
    }
    const float nr = __fsqrt_rn(group_sum_sq(h, r, lane));
    if (nr > 0.0f) {
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            h[b] = __fdiv_rn(h[b], nr);
            if (h[b] > 0.2f) h[b] = 0.2f;
        }
    }
    const float nr2 = __fsqrt_rn(group_sum_sq(h, r, lane));
    uint32_t word[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) word[i] = 0u;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const float u = nr2 > 0.0f ? __fdiv_rn(h[b], nr2) : 0.0f;
        const int q = (int)__fadd_rn(__fmul_rn(u, 512.0f), 0.5f);
        word[b >> 2] |= (uint32_t)min(q, 255) << (8 * (b & 3));
    }
    if (valid) {
        uint4* out = reinterpret_cast<uint4*>(J.desc + (plane + (size_t)y * J.w + x) * kDesc + 32 * r);
        out[0] = make_uint4(word[0], word[1], word[2], word[3]);
        out[1] = make_uint4(word[4], word[5], word[6], word[7]);
    }
}

// Sums of the descriptors and of their pairwise products over the four
// images' full-resolution descriptors.
__global__ void __launch_bounds__(kCovThreads) k_sift_cov(SiftJob J, size_t count) {
    __shared__ uint32_t tile[kDesc][kCovPix / 4];  // [component][4 descriptors]
    const int t = threadIdx.x;
    uint32_t acc[kDesc * kDesc / kCovThreads];
    uint32_t s1 = 0;
#pragma unroll
    for (int e = 0; e < kDesc * kDesc / kCovThreads; ++e) acc[e] = 0;
    size_t since = 0;
    auto flush = [&]() {
#pragma unroll
        for (int e = 0; e < kDesc * kDesc / kCovThreads; ++e) {
            if (acc[e]) atomicAdd(J.s2 + t + e * kCovThreads, (unsigned long long)acc[e]);
            acc[e] = 0;
        }
        if (t < kDesc && s1) atomicAdd(J.s1 + t, (unsigned long long)s1);
        s1 = 0;
    };
    for (size_t base = (size_t)blockIdx.x * kCovPix; base < count; base += (size_t)gridDim.x * kCovPix) {
        __syncthreads();
        // transpose 64 descriptors into [component][descriptor] bytes
        for (int k = t; k < kCovPix * kDesc / 4; k += kCovThreads) {
            const int p = k / (kDesc / 4), w4 = k % (kDesc / 4);
            uint32_t word = 0;
            if (base + p < count) word = reinterpret_cast<const uint32_t*>(J.desc + (base + p) * kDesc)[w4];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                reinterpret_cast<uint8_t*>(&tile[w4 * 4 + b][p / 4])[p % 4] = (uint8_t)(word >> (8 * b));
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kDesc * kDesc / kCovThreads; ++e) {
            const int idx = t + e * kCovThreads, i = idx / kDesc, j = idx % kDesc;
            uint32_t a = acc[e];
#pragma unroll
            for (int p4 = 0; p4 < kCovPix / 4; ++p4) a = __dp4a(tile[i][p4], tile[j][p4], a);
            acc[e] = a;
        }
        if (t < kDesc)
#pragma unroll
            for (int p4 = 0; p4 < kCovPix / 4; ++p4) s1 = __dp4a(tile[t][p4], 0x01010101u, s1);
        since += kCovPix;
        if (since >= kCovFlush) {
            flush();
            since = 0;
        }
    }
    flush();
}

// Dot product of two 128-vectors in shared memory as in the power
// iteration: threads 0-3 each accumulate the indices of one residue mod 4 in
// index order by fused multiply-adds; thread 0 combines (s0 + s1) + (s2 + s3)
// into *out.  Called by the whole CTA (two barriers).
__device__ __forceinline__ void dot128_cta(const double* a, const double* b, double* part, double* out) {
    const int i = threadIdx.x;
    if (i < 4) {
        double t = 0.0;
#pragma unroll 8
        for (int k = i; k < kDesc; k += 4) t = __fma_rn(a[k], b[k], t);
        part[i] = t;
    }
    __syncthreads();
    if (i == 0) *out = __dadd_rn(__dadd_rn(part[0], part[1]), __dadd_rn(part[2], part[3]));
    __syncthreads();
}

// One CTA of 128 threads: thread i owns row i of the covariance, kept
// column-major in shared memory (Ct[j][i] = C(i, j)) so that a warp reads 32
// consecutive doubles at every step of its rows.  Every dot product of the
// iteration is four partial sums over the indices mod 4 in index order by
// fused multiply-adds, combined as (s0 + s1) + (s2 + s3).
__global__ void __launch_bounds__(kDesc) k_sift_axes(SiftJob J, double count) {
    extern __shared__ double Ct[];  // [128][128], column-major covariance
    __shared__ double mean[kDesc], v[kDesc], wv[kDesc], ax[3][kDesc], part[4], bc;
    const int i = threadIdx.x;
    mean[i] = __ddiv_rn((double)J.s1[i], count);
    __syncthreads();
    for (int j = 0; j < kDesc; ++j)
        Ct[j * kDesc + i] = __dsub_rn(__ddiv_rn((double)J.s2[i * kDesc + j], count), __dmul_rn(mean[i], mean[j]));
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        v[i] = 1.0;
        __syncthreads();
        for (int it = 0; it < kPowerIters; ++it) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
            for (int k = 0; k < kDesc; k += 4) {
                s0 = __fma_rn(Ct[(k + 0) * kDesc + i], v[k + 0], s0);
                s1 = __fma_rn(Ct[(k + 1) * kDesc + i], v[k + 1], s1);
                s2 = __fma_rn(Ct[(k + 2) * kDesc + i], v[k + 2], s2);
                s3 = __fma_rn(Ct[(k + 3) * kDesc + i], v[k + 3], s3);
            }
            wv[i] = __dadd_rn(__dadd_rn(s0, s1), __dadd_rn(s2, s3));
            __syncthreads();
            for (int e = 0; e < c; ++e) {
                dot128_cta(ax[e], wv, part, &bc);
                wv[i] = __dsub_rn(wv[i], __dmul_rn(bc, ax[e][i]));
                __syncthreads();
            }
            dot128_cta(wv, wv, part, &bc);
            const double nr = __dsqrt_rn(bc);
            v[i] = nr > 0.0 ? __ddiv_rn(wv[i], nr) : 0.0;
            __syncthreads();
        }
        if (i == 0) {
            int big = 0;
            for (int k = 1; k < kDesc; ++k)
                if (fabs(v[k]) > fabs(v[big])) big = k;
            bc = v[big] < 0.0 ? -1.0 : 1.0;
        }
        __syncthreads();
        ax[c][i] = __dmul_rn(bc, v[i]);
        J.axes[c * kDesc + i] = ax[c][i];
        __syncthreads();
    }
    // single-precision projection weights and biases fl(a_c . mean), the
    // bias a sequential sum
    for (int c = 0; c < 3; ++c) J.proj[c * kDesc + i] = (float)ax[c][i];
    if (i < 3) {
        double b = 0.0;
        for (int k = 0; k < kDesc; ++k) b = __dadd_rn(b, __dmul_rn(ax[i][k], mean[k]));
        J.proj[3 * kDesc + i] = (float)b;
    }
}

__global__ void __launch_bounds__(128) k_sift_project(SiftJob J) {
    __shared__ float a[3 * kDesc + 3];
    for (int k = threadIdx.x; k < 3 * kDesc + 3; k += blockDim.x) a[k] = J.proj[k];
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, v = blockIdx.z;
    if (x >= J.w) return;
    const size_t p = (size_t)y * J.w + x;
    const uint4* q = reinterpret_cast<const uint4*>(J.desc + ((size_t)v * J.h * J.w + p) * kDesc);
    float t[3] = {0.0f, 0.0f, 0.0f};
    for (int k16 = 0; k16 < kDesc / 16; ++k16) {  // 16 components per load, in index order
        const uint4 w = q[k16];
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const float qv = (float)((words[b >> 2] >> (8 * (b & 3))) & 0xffu);
            const int k = k16 * 16 + b;
#pragma unroll
            for (int c = 0; c < 3; ++c) t[c] = __fadd_rn(t[c], __fmul_rn(a[c * kDesc + k], qv));
        }
    }
    float r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = __fsub_rn(t[c], a[3 * kDesc + c]);
    reinterpret_cast<float4*>(phi_of(J, v))[(size_t)J.s * J.w * J.h + p] = make_float4(r[0], r[1], r[2], 0.0f);
}

struct SiftLayout {
    size_t grey, mag, bin, desc, s1, s2, axes, proj, total;
};

SiftLayout sift_layout(int w, int h) {
    const size_t np = (size_t)w * h;
    SiftLayout L;
    L.grey = 0;
    L.mag = L.grey + align256(4 * np);
    L.bin = L.mag + align256(4 * np * sizeof(float));
    L.desc = L.bin + align256(4 * np);
    L.s1 = L.desc + align256(4 * np * kDesc);
    L.s2 = L.s1 + align256(kDesc * 8);
    L.axes = L.s2 + align256(kDesc * kDesc * 8);
    L.proj = L.axes + align256(3 * kDesc * 8);
    L.total = L.proj + align256((3 * kDesc + 3) * sizeof(float));
    return L;
}

}  // namespace
}  // namespace sff

extern "C" size_t sff_sift_workspace_bytes(int32_t width, int32_t height) {
    if (sff::check_size(width, height)) return 0;
    return sff::sift_layout(width, height).total;
}

extern "C" int sff_sift_features(const uint8_t* const* rgb_dev4, int32_t pitch_bytes, int32_t width, int32_t height,
                                 const sff_params* params, float* const* phi_dev4, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params) || !rgb_dev4 || !phi_dev4 || !workspace) return SFF_ERR_ARG;
    if (pitch_bytes < 3 * width || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    for (int v = 0; v < 4; ++v)
        if (!rgb_dev4[v] || !phi_dev4[v] || ((uintptr_t)phi_dev4[v] & 15)) return SFF_ERR_ARG;
    const SiftLayout L = sift_layout(width, height);
    if (workspace_bytes < L.total) return SFF_ERR_WORKSPACE;
    char* ws = reinterpret_cast<char*>(workspace);
    SiftJob J;
    for (int v = 0; v < 4; ++v) {
        J.rgb[v] = rgb_dev4[v];
        J.phi[v] = phi_dev4[v];
    }
    J.pitch = pitch_bytes;
    J.w = width;
    J.h = height;
    J.grey = reinterpret_cast<uint8_t*>(ws + L.grey);
    J.mag = reinterpret_cast<float*>(ws + L.mag);
    J.bin = reinterpret_cast<uint8_t*>(ws + L.bin);
    J.desc = reinterpret_cast<uint8_t*>(ws + L.desc);
    J.s1 = reinterpret_cast<unsigned long long*>(ws + L.s1);
    J.s2 = reinterpret_cast<unsigned long long*>(ws + L.s2);
    J.axes = reinterpret_cast<double*>(ws + L.axes);
    J.proj = reinterpret_cast<float*>(ws + L.proj);
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g((width + 127) / 128, height, 4);
    const dim3 gd((width + kDescThreads / 4 - 1) / (kDescThreads / 4), height, 4);
    // the attribute is per device: set it on the current one at every call
    if (cudaFuncSetAttribute(k_sift_axes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kDesc * kDesc * (int)sizeof(double)) != cudaSuccess)
        return SFF_ERR_CUDA;
    for (int s = 0; s < params->num_scales; ++s) {
        J.s = s;
        J.n = 1 << s;
        SFF_LAUNCH(k_sift_grey, g, 128, 0, st, J);
        SFF_LAUNCH(k_sift_grad, g, 128, 0, st, J);
        SFF_LAUNCH(k_sift_desc, gd, kDescThreads, 0, st, J);
        if (s == 0) {  // the principal axes of the full-resolution descriptors
            if (cudaMemsetAsync(J.s1, 0, L.axes - L.s1, st) != cudaSuccess) return SFF_ERR_CUDA;
            const size_t count = 4 * (size_t)width * height;
            const int blocks = (int)std::min<size_t>((count + kCovPix - 1) / kCovPix, 152 * 4);
            SFF_LAUNCH(k_sift_cov, dim3(blocks), kCovThreads, 0, st, J, count);
            SFF_LAUNCH(k_sift_axes, dim3(1), kDesc, kDesc * kDesc * sizeof(double), st, J, (double)count);
        }
        SFF_LAUNCH(k_sift_project, g, 128, 0, st, J);
    }
    return launch_status();
}
