// Walsh-Hadamard patch features on the box-smoothed scale space
// (Sec. 3.1, "Initialization" and "Multi-Scale Propagation").
//
// k_smooth:   a 64x16 tile of output pixels per CTA; the tile's input region
//             (with the largest box's margin, edges replicated) is turned
//             into a summed-area table in shared memory, so every box sum of
//             every scale costs four lookups per channel.  Output per scale:
//             R and G packed as R + 65536 G (one int32 plane) and B (a
//             second plane), the form the transform consumes.
// k_features: one thread per pair of pixels (x, y), (x, y + n) of scale s:
//             their 8x8 patches share 7 of 8 rows, so 9 row transforms (fast
//             8-point Walsh-Hadamard butterflies, R and G packed in one
//             int32; every intermediate stays below 2^31 in magnitude, so
//             packed adds and subtracts are exact) serve both.  Each row
//             transform is folded into the 16 kept coefficients of both
//             pixels with compile-time signs of the sequency-ordered Walsh
//             rows.  The coefficients are quantised, packed and written as
//             one 48-byte record per pixel; the norm is a dp4a of the packed
//             bytes with themselves.
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
// Entry (k, i) of the sequency-ordered Walsh matrix: natural Hadamard row
// seq_to_nat(k), i.e. (-1)^popcount(seq_to_nat(k) & i).
__host__ __device__ constexpr int walsh(int k, int i) {
    return (((seq_to_nat(k) & i) & 1) ^ (((seq_to_nat(k) & i) >> 1) & 1) ^ (((seq_to_nat(k) & i) >> 2) & 1)) ? -1 : 1;
}
static_assert(seq_to_nat(1) == 4 && seq_to_nat(2) == 6 && seq_to_nat(5) == 7 && seq_to_nat(7) == 1, "walsh map");
static_assert(order_ky(0) == 0 && order_kx(0) == 1 && order_ky(4) == 2 && order_kx(4) == 0, "order");
static_assert(order_ky(13) == 4 && order_kx(13) == 0 && order_ky(15) == 1 && order_kx(15) == 4, "order");
static_assert(walsh(1, 0) == 1 && walsh(1, 4) == -1 && walsh(2, 2) == -1 && walsh(2, 6) == 1, "walsh rows");

constexpr int kSmX = 64, kSmY = 16;  // output tile of k_smooth
constexpr int kMargin = 4;           // half of the largest box (n = 8)
constexpr int kRegX = kSmX + 2 * kMargin, kRegY = kSmY + 2 * kMargin;

__global__ void __launch_bounds__(256) k_smooth(const __grid_constant__ ImageJobs J, int S) {
    __shared__ int sat[3][kRegY + 1][kRegX + 1];  // summed-area table per channel, zero first row/column
    const ImageJob& job = J.im[blockIdx.z];
    const int w = job.w, h = job.h, pitch = job.pitch;
    const int x0 = blockIdx.x * kSmX, y0 = blockIdx.y * kSmY;
    if (x0 >= w || y0 >= h) return;
    for (int k = threadIdx.x; k < (kRegY + 1) * (kRegX + 1); k += blockDim.x) {
        const int ry = k / (kRegX + 1), rx = k % (kRegX + 1);
        if (ry == 0 || rx == 0) {
            sat[0][ry][rx] = sat[1][ry][rx] = sat[2][ry][rx] = 0;
            continue;
        }
        const int x = clampi(x0 - kMargin + rx - 1, 0, w - 1), y = clampi(y0 - kMargin + ry - 1, 0, h - 1);
        const uint8_t* p = job.rgb + (size_t)y * pitch + 3 * x;
        sat[0][ry][rx] = p[0];
        sat[1][ry][rx] = p[1];
        sat[2][ry][rx] = p[2];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * kRegY; k += blockDim.x) {  // prefix along rows
        int* row = &sat[k / kRegY][1 + k % kRegY][0];
        for (int x = 1; x <= kRegX; ++x) row[x] += row[x - 1];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * kRegX; k += blockDim.x) {  // prefix along columns
        const int c = k / kRegX, x = 1 + k % kRegX;
        for (int y = 1; y <= kRegY; ++y) sat[c][y][x] += sat[c][y - 1][x];
    }
    __syncthreads();
    const size_t np = (size_t)w * h;
    int* rg_out = reinterpret_cast<int*>(job.sm);
    int* b_out = rg_out + (size_t)S * np;
    for (int k = threadIdx.x; k < kSmX * kSmY; k += blockDim.x) {
        const int lx = k % kSmX, ly = k / kSmX;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= w || y >= h) continue;
        const size_t i = (size_t)y * w + x;
        // scale 0: the pixel itself (region cell (ly + margin, lx + margin))
        {
            const int cy = ly + kMargin + 1, cx = lx + kMargin + 1;
            int v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                v[c] = sat[c][cy][cx] - sat[c][cy - 1][cx] - sat[c][cy][cx - 1] + sat[c][cy - 1][cx - 1];
            rg_out[i] = v[0] + 65536 * v[1];
            b_out[i] = v[2];
        }
        for (int s = 1; s < S; ++s) {
            const int n = 1 << s;
            // box rows/columns -n/2 .. n/2-1 around the pixel, in region cells (+1 for the zero border)
            const int ya = ly + kMargin - n / 2, yb = ly + kMargin + n / 2;  // rows [ya, yb) of the region
            const int xa = lx + kMargin - n / 2, xb = lx + kMargin + n / 2;
            int v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int sum = sat[c][yb][xb] - sat[c][ya][xb] - sat[c][yb][xa] + sat[c][ya][xa];
                v[c] = (sum + n * n / 2) >> (2 * s);
            }
            rg_out[(size_t)s * np + i] = v[0] + 65536 * v[1];
            b_out[(size_t)s * np + i] = v[2];
        }
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

// Four int32 values saturated to int8 and packed, v0 in the lowest byte:
// cvt.pack.sat converts a and b and packs them as (a << 8) | b above the
// low bits of c.
__device__ __forceinline__ int pack4_sat(int v0, int v1, int v2, int v3) {
    unsigned hi, d;
    asm("cvt.pack.sat.s8.s32.b32 %0, %1, %2, 0;" : "=r"(hi) : "r"(v3), "r"(v2));
    asm("cvt.pack.sat.s8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(v1), "r"(v0), "r"(hi));
    return (int)d;
}

// Accumulate row transform (rg[kx], b[kx], kx = 0..5 in sequency order) of
// patch row i into the 16 kept coefficients.
template <int I>
__device__ __forceinline__ void fold_row(const int (&rg)[6], const int (&bb)[6], int (&arg)[16], int (&ab)[16]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (walsh(order_ky(m), I) > 0) {
            arg[m] += rg[order_kx(m)];
            ab[m] += bb[order_kx(m)];
        } else {
            arg[m] -= rg[order_kx(m)];
            ab[m] -= bb[order_kx(m)];
        }
    }
}

// Quantised record of one pixel: chunk k (channel k) at planes[k * cs + i * rs].
__device__ __forceinline__ void write_record(const int (&arg)[16], const int (&ab)[16], int qshift, int4* planes,
                                             size_t cs, size_t rs, size_t i, int* norm) {
    // R = low 16 bits (signed), G = the rest; arithmetic shifts floor, as the
    // quantisation does
    int q[3][16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int lo = arg[m] << 16;
        q[0][m] = lo >> (16 + qshift);
        q[1][m] = (arg[m] - (lo >> 16)) >> (16 + qshift);
        q[2][m] = ab[m] >> qshift;
    }
    int words[12];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            words[4 * c + k] = pack4_sat(q[c][4 * k], q[c][4 * k + 1], q[c][4 * k + 2], q[c][4 * k + 3]);
    int nn = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) nn = __dp4a(words[k], words[k], nn);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        planes[k * cs + i * rs] = make_int4(words[4 * k], words[4 * k + 1], words[4 * k + 2], words[4 * k + 3]);
    *norm = nn;
}

__global__ void __launch_bounds__(128) k_features(const __grid_constant__ ImageJobs J, int s, int S, int qshift) {
    const ImageJob& job = J.im[blockIdx.z];
    const int w = job.w, h = job.h;
    const int n = 1 << s;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    // pair row p covers (y, y + n) with y = (p / n) * 2n + p % n
    const int p = blockIdx.y;
    const int y = (p / n) * 2 * n + p % n;
    if (x >= w || y >= h) return;
    const bool second = y + n < h;
    const size_t np = (size_t)w * h;
    const int* rgp = reinterpret_cast<const int*>(job.sm) + (size_t)s * np;
    const int* bp = reinterpret_cast<const int*>(job.sm) + (size_t)S * np + (size_t)s * np;
    int xs[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xs[j] = clampi(x + n * (j - 3), 0, w - 1);
    int a_rg[16], a_b[16], b_rg[16], b_b[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) a_rg[m] = a_b[m] = b_rg[m] = b_b[m] = 0;
    // rows y + n (k - 3), k = 0..8: pixel (x, y) uses k = 0..7 as patch row k,
    // pixel (x, y + n) uses k = 1..8 as patch row k - 1
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const size_t row = (size_t)clampi(y + n * (k - 3), 0, h - 1) * w;
        int a[8], b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            a[j] = __ldg(rgp + row + xs[j]);
            b[j] = __ldg(bp + row + xs[j]);
        }
        fwht8(a);
        fwht8(b);
        int rg[6], bb[6];
#pragma unroll
        for (int kx = 0; kx < 6; ++kx) {
            rg[kx] = a[seq_to_nat(kx)];
            bb[kx] = b[seq_to_nat(kx)];
        }
        // compile-time patch row of each pixel
        switch (k) {
            case 0: fold_row<0>(rg, bb, a_rg, a_b); break;
            case 1: fold_row<1>(rg, bb, a_rg, a_b); fold_row<0>(rg, bb, b_rg, b_b); break;
            case 2: fold_row<2>(rg, bb, a_rg, a_b); fold_row<1>(rg, bb, b_rg, b_b); break;
            case 3: fold_row<3>(rg, bb, a_rg, a_b); fold_row<2>(rg, bb, b_rg, b_b); break;
            case 4: fold_row<4>(rg, bb, a_rg, a_b); fold_row<3>(rg, bb, b_rg, b_b); break;
            case 5: fold_row<5>(rg, bb, a_rg, a_b); fold_row<4>(rg, bb, b_rg, b_b); break;
            case 6: fold_row<6>(rg, bb, a_rg, a_b); fold_row<5>(rg, bb, b_rg, b_b); break;
            case 7: fold_row<7>(rg, bb, a_rg, a_b); fold_row<6>(rg, bb, b_rg, b_b); break;
            default: fold_row<7>(rg, bb, b_rg, b_b); break;
        }
    }
    int4* feat = reinterpret_cast<int4*>(job.pyr + (size_t)s * np * kFeat);
    int* norms = reinterpret_cast<int*>(job.pyr + (size_t)S * np * kFeat) + (size_t)s * np;
    const size_t i = (size_t)y * w + x;
    const size_t cs = chunk_planes(s) ? np : 1, rs = chunk_planes(s) ? 1 : 3;
    write_record(a_rg, a_b, qshift, feat, cs, rs, i, norms + i);
    if (second) write_record(b_rg, b_b, qshift, feat, cs, rs, i + (size_t)n * w, norms + i + (size_t)n * w);
}

}  // namespace

// Scratch of one image: the smoothed scale space as two int32 planes per
// scale (R + 65536 G, and B).
size_t features_ws_bytes(int w, int h, const sff_params& p) {
    return align256((size_t)2 * p.num_scales * w * h * sizeof(int));
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
    dim3 gs((mw + kSmX - 1) / kSmX, (mh + kSmY - 1) / kSmY, n);
    SFF_LAUNCH(k_smooth, gs, 256, 0, st, J, P.num_scales);
    for (int s = 0; s < P.num_scales; ++s) {
        const int nn = 1 << s;
        // pair rows: ceil(H / 2n) pairs per residue class of rows mod n
        dim3 gf((mw + 127) / 128, ((mh + 2 * nn - 1) / (2 * nn)) * nn, n);
        SFF_LAUNCH(k_features, gf, 128, 0, st, J, s, P.num_scales, P.quant_shift);
    }
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
