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
#include <cuda_fp16.h>

#include <mutex>

#include "sff_internal.cuh"
#include "sff_tc.cuh"

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

// Writes the smoothed planes of scales s_lo..s_hi (of S).
__global__ void __launch_bounds__(256) k_smooth(const __grid_constant__ ImageJobs J, int S, int s_lo, int s_hi) {
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
        if (s_lo == 0) {
            const int cy = ly + kMargin + 1, cx = lx + kMargin + 1;
            int v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                v[c] = sat[c][cy][cx] - sat[c][cy - 1][cx] - sat[c][cy][cx - 1] + sat[c][cy - 1][cx - 1];
            rg_out[i] = v[0] + 65536 * v[1];
            b_out[i] = v[2];
        }
        for (int s = s_lo > 1 ? s_lo : 1; s <= s_hi; ++s) {
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

// ---------------------------------------------------------------------------
// Separable form (k_features_sep, the default; identical records).  The row
// transform of image row yy at column x (the 8-point Walsh transform of the
// samples yy, x + n (j - 3)) serves every pixel whose patch contains that
// row: the 8 pixels (x, yy - n (i - 3)).  A CTA takes kSepTX columns x kSepTY
// rows of one residue class of rows mod n (rows r, r + n, r + 2n, ...): it
// first computes the row transforms of the kSepTY + 7 rows those patches use
// once, into shared memory (kept sequencies kx = 0..5 of R + 65536 G and of
// B), then each thread takes two vertically adjacent pixels, which share 7
// of their 9 rows, and transforms their rows column-wise with one 8-point
// butterfly per kx and pixel, of which only the outputs of the kept (ky, kx)
// pairs are used (the compiler drops the rest).  The sums are exact integers
// in any order, so the records equal those of k_features (the pixel-pair
// form above) bit for bit.
constexpr int kSepTX = 32, kSepTY = 24, kSepRows = kSepTY + 7, kSepThreads = 192;

// Index m of kept coefficient (ky, kx): diagonal t = ky + kx starts at t(t+1)/2 - 1.
__host__ __device__ constexpr int kept_index(int ky, int kx) { return (ky + kx) * (ky + kx + 1) / 2 - 1 + ky; }
static_assert(kept_index(0, 1) == 0 && kept_index(1, 0) == 1 && kept_index(4, 0) == 13 && kept_index(1, 4) == 15,
              "kept order");
// Kept ky range for sequency kx (the kept set is 1 <= ky + kx <= 4, plus (0, 5) and (1, 4)).
__host__ __device__ constexpr int kept_ky_max(int kx) { return kx == 0 ? 4 : kx == 1 ? 3 : kx == 2 ? 2 : kx <= 4 ? 1 : 0; }
__host__ __device__ constexpr int kept_ky_min(int kx) { return kx == 0 ? 1 : 0; }

__global__ void __launch_bounds__(kSepThreads) k_features_sep(const __grid_constant__ ImageJobs J, int s, int S,
                                                              int qshift, int tiles_per_residue) {
    // row transforms [tile row][k][column], k = kx 0..5 of R + 65536 G, then
    // of B: a warp's 32 columns of one (row, k) in one wavefront
    __shared__ int sR[kSepRows][12][kSepTX];
    const ImageJob& job = J.im[blockIdx.z];
    const int w = job.w, h = job.h;
    const int n = 1 << s;
    const int x0 = blockIdx.x * kSepTX;
    const int r = blockIdx.y / tiles_per_residue, m0 = (blockIdx.y % tiles_per_residue) * kSepTY;
    const int rows_r = (h - r + n - 1) / n;  // rows r, r + n, ... of this image
    if (x0 >= w || r >= h || m0 >= rows_r) return;  // whole CTA beyond this image
    const size_t np = (size_t)w * h;
    const int* rgp = reinterpret_cast<const int*>(job.sm) + (size_t)s * np;
    const int* bp = reinterpret_cast<const int*>(job.sm) + (size_t)S * np + (size_t)s * np;
    // phase 1: row transforms of image rows clamp(r + n (m0 + t - 3)), t < kSepRows
    for (int e = threadIdx.x; e < kSepRows * kSepTX; e += kSepThreads) {
        const int t = e / kSepTX, lx = e % kSepTX;
        const int x = x0 + lx;
        if (x >= w) continue;  // never read
        const size_t row = (size_t)clampi(r + n * (m0 + t - 3), 0, h - 1) * w;
        int a[8], b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int xj = clampi(x + n * (j - 3), 0, w - 1);
            a[j] = __ldg(rgp + row + xj);
            b[j] = __ldg(bp + row + xj);
        }
        fwht8(a);
        fwht8(b);
#pragma unroll
        for (int kx = 0; kx < 6; ++kx) {
            sR[t][kx][lx] = a[seq_to_nat(kx)];
            sR[t][6 + kx][lx] = b[seq_to_nat(kx)];
        }
    }
    __syncthreads();
    // phase 2: the pixel pair (x0 + lx, r + n (m0 + ly)), ly = ly0, ly0 + 1,
    // takes tile rows ly0 .. ly0 + 8 (pixel q its rows ly0 + q .. ly0 + q + 7)
    int4* feat = reinterpret_cast<int4*>(job.pyr + (size_t)s * np * kFeat);
    int* norms = reinterpret_cast<int*>(job.pyr + (size_t)S * np * kFeat) + (size_t)s * np;
    const size_t cs = chunk_planes(s) ? np : 1, rs = chunk_planes(s) ? 1 : 3;
    for (int e = threadIdx.x; e < (kSepTY / 2) * kSepTX; e += kSepThreads) {
        const int ly0 = 2 * (e / kSepTX), lx = e % kSepTX;
        const int x = x0 + lx, m = m0 + ly0;
        if (x >= w || m >= rows_r) continue;
        int arg[2][16], ab[2][16];
#pragma unroll
        for (int kx = 0; kx < 6; ++kx) {
            int c[9], d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                c[i] = sR[ly0 + i][kx][lx];
                d[i] = sR[ly0 + i][6 + kx][lx];
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int cq[8], dq[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    cq[i] = c[q + i];
                    dq[i] = d[q + i];
                }
                fwht8(cq);
                fwht8(dq);
#pragma unroll
                for (int ky = kept_ky_min(kx); ky <= kept_ky_max(kx); ++ky) {
                    arg[q][kept_index(ky, kx)] = cq[seq_to_nat(ky)];
                    ab[q][kept_index(ky, kx)] = dq[seq_to_nat(ky)];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (m + q >= rows_r) break;
            const size_t i = (size_t)(r + n * (m + q)) * w + x;
            write_record(arg[q], ab[q], qshift, feat, cs, rs, i, norms + i);
        }
    }
}

// ---------------------------------------------------------------------------
// The same features with the transform on the tensor cores (k_features_tc).
//
// For one scale and channel, the 16 kept coefficients of the pixels of a row
// segment are one matrix product D = A B^T: A is the 128 x 64 matrix of the
// pixels' 8x8 patches (row p: P[i][j] of pixel p, k = 8 i + j), B the 16 x 64
// matrix of the kept Walsh products (row m: walsh(ky(m), i) walsh(kx(m), j)).
// Patch values are integers 0..255 and B entries +-1, exact in fp16; every
// product and partial sum is an integer of magnitude <= 64 * 255 = 16320,
// exact in the fp32 accumulator whatever the order of the sums.  One CTA of
// 128 threads walks down a column of tiles (128 pixels of one row, the rows y,
// y + n, y + 2n, ... of one residue class), so each step stages one new patch
// row: the 8 patch rows of the current tile are a ring of smoothed rows in
// shared memory (fp16 per channel).  A is stored MN-major (8 consecutive
// pixels of one (channel, i, j) in 16 bytes), so each 16-byte chunk of A is 8
// consecutive fp16 of one staged row starting at column 8 g + n j: aligned
// vector copies (at n = 1 from a copy of the row shifted by one element when
// the start is odd).  Per tile: 3 channels x 4 MMAs (M 128, N 16, K 16) into
// tensor memory, one commit, then each thread reads its pixel's 48
// coefficients (TMEM lane = pixel), quantises and stores the record.
constexpr int kTcfPx = 128;                    // pixels per tile = M = threads
constexpr int kTcfSeg = 16;                    // tiles (rows) per CTA
constexpr int kTcfRowCols = kTcfPx + 7 * 8;    // staged columns for the widest stride (n = 8)
constexpr int kTcfKGroup = kTcfPx * 16;        // bytes between K groups of A (2048)
constexpr int kTcfABytes = 24 * kTcfKGroup;    // 3 channels x 8 patch rows of 8 K-columns: 48 KB
constexpr int kTcfBBytes = 16 * 64 * 2;        // 16 coefficients x 64 patch entries, fp16: 2 KB
constexpr int kTcfRingBytes = 2 * 3 * 8 * kTcfRowCols * 2;  // two copies x 3 channels x 8 rows, fp16
constexpr int kTcfOffB = kTcfABytes;
constexpr int kTcfOffRing = kTcfOffB + kTcfBBytes;
constexpr int kTcfOffBar = kTcfOffRing + kTcfRingBytes;
constexpr int kTcfSmemBytes = kTcfOffBar + 64 + 1024;  // + alignment slack
constexpr int kTcfCols = 64;                           // TMEM columns (48 used)
// instruction descriptor, kind::f16: fp32 D (bits 4-5 = 1), fp16 A and B
// (bits 7-12 = 0), A MN-major (bit 15), B K-major, N = 16, M = 128
constexpr uint32_t kTcfIdesc = (1u << 4) | (1u << 15) | ((16u >> 3) << 17) | ((uint32_t)(kTcfPx >> 4) << 24);

__device__ unsigned int g_features_status;  // bit 0: a bounded wait of k_features_tc gave up

template <int S>
__global__ void __launch_bounds__(kTcfPx) k_features_tc(const __grid_constant__ ImageJobs J, int NS, int qshift) {
    constexpr int n = 1 << S;
    constexpr int kCols = kTcfPx + 7 * n;  // staged columns: x0 - 3n .. x0 + 127 + 4n
    extern __shared__ uint8_t smem_raw[];
    const ImageJob& job = J.im[blockIdx.z];
    const int w = job.w, h = job.h;
    const int tiles_x = (w + kTcfPx - 1) / kTcfPx;
    const int rows_n = (h + n - 1) / n;  // rows per residue class (at most)
    const int segs = (rows_n + kTcfSeg - 1) / kTcfSeg;
    const int item = blockIdx.x;  // (segment, residue, tile column)
    if (item >= tiles_x * n * segs) return;  // CTA-uniform, before any allocation
    const int tx = item % tiles_x, ph = (item / tiles_x) % n, seg = item / (tiles_x * n);
    const int x0 = tx * kTcfPx;
    const int y_first = ph + seg * kTcfSeg * n;
    if (y_first >= h) return;
    uint8_t* sm = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    uint8_t* sA = sm;
    uint8_t* sB = sm + kTcfOffB;
    __half* ring = reinterpret_cast<__half*>(sm + kTcfOffRing);  // [copy][c][slot][col]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTcfOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kTcfOffBar + 8);
    const int t = threadIdx.x;
    const size_t np = (size_t)w * h;
    const int* rgp = reinterpret_cast<const int*>(job.sm) + (size_t)S * np;
    const int* bp = reinterpret_cast<const int*>(job.sm) + (size_t)NS * np + (size_t)S * np;

    if (t == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    if (t < 32) tmem_alloc(tmem_slot, kTcfCols);
    // B: row m (kept coefficient), column k = 8 i + j, K-major core matrices
    for (int e = t; e < 16 * 64; e += kTcfPx) {
        const int m = e >> 6, k = e & 63, i = k >> 3, j = k & 7;
        const int v = walsh(order_ky(m), i) * walsh(order_kx(m), j);
        *reinterpret_cast<__half*>(sB + (k >> 3) * 256 + (m >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2) =
            __int2half_rn(v);
    }
    // A staged row: columns c0 = t, t + 128 of image row yi (x clamped).  The
    // loads of the next tile's new row are issued one tile ahead into
    // registers (rg, b pairs) and written into the ring when that tile starts.
    constexpr int kPre = (kCols + kTcfPx - 1) / kTcfPx;
    auto load_row = [&](int yi, int2 (&pre)[kPre]) {
        const size_t row = (size_t)clampi(yi, 0, h - 1) * w;
#pragma unroll
        for (int e = 0; e < kPre; ++e) {
            const int c0 = t + e * kTcfPx;
            if (c0 < kCols) {
                const int x = clampi(x0 - 3 * n + c0, 0, w - 1);
                pre[e] = make_int2(__ldg(rgp + row + x), __ldg(bp + row + x));
            }
        }
    };
    auto put_row = [&](int slot, const int2 (&pre)[kPre]) {
#pragma unroll
        for (int e = 0; e < kPre; ++e) {
            const int c0 = t + e * kTcfPx;
            if (c0 < kCols) {
                const __half v[3] = {__int2half_rn(pre[e].x & 0xffff), __int2half_rn(pre[e].x >> 16),
                                     __int2half_rn(pre[e].y)};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ring[((0 * 3 + c) * 8 + slot) * kTcfRowCols + c0] = v[c];
                    if (n == 1 && c0 > 0) ring[((1 * 3 + c) * 8 + slot) * kTcfRowCols + c0 - 1] = v[c];
                }
            }
        }
    };
    int2 pre[kPre];
    for (int i = 0; i < 8; ++i) {
        load_row(y_first + n * (i - 3), pre);
        put_row(i, pre);
    }
    load_row(y_first + n + 4 * n, pre);  // the new row of tile 1
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const unsigned long long wait_ns = kDefaultWaitNs;
    bool failed = false;
    int failed_k = -1;  // the tile whose wait gave up (its MMAs may still run)
    int4* feat = reinterpret_cast<int4*>(job.pyr + (size_t)S * np * kFeat);
    int* norms = reinterpret_cast<int*>(job.pyr + (size_t)NS * np * kFeat) + (size_t)S * np;
    const size_t cs = chunk_planes(S) ? np : 1, rs = chunk_planes(S) ? 1 : 3;

    for (int k = 0; k < kTcfSeg; ++k) {
        const int y = y_first + k * n;
        if (y >= h) break;  // CTA-uniform
        if (k > 0) {
            put_row((k + 7) & 7, pre);  // the slot of the previous tile's patch row 0
            __syncthreads();
            if (k + 1 < kTcfSeg) load_row(y + n + 4 * n, pre);  // next tile's new row, in flight meanwhile
        }
        // A: 3072 chunks of 16 bytes, chunk e = (K group ci, pixel group g,
        // row j) with j fastest, so a warp writes 512 contiguous bytes; each
        // is 8 consecutive staged fp16 of row (channel, patch row i) from
        // column 8 g + n j
#pragma unroll 4
        for (int r = 0; r < 24; ++r) {
            const int e = t + r * kTcfPx;
            const int j = e & 7, g = (e >> 3) & 15, ci = e >> 7, c = ci >> 3, i = ci & 7;
            const int slot = (k + i) & 7;
            const int o = 8 * g + n * j;  // first staged column of the chunk
            uint4 v;
            if (n >= 8) {
                v = *reinterpret_cast<const uint4*>(ring + (c * 8 + slot) * kTcfRowCols + o);
            } else if (n >= 4) {
                const uint2* src = reinterpret_cast<const uint2*>(ring + (c * 8 + slot) * kTcfRowCols + o);
                v = make_uint4(src[0].x, src[0].y, src[1].x, src[1].y);
            } else {
                // n = 1: odd starts read the copy shifted by one element
                const int copy = (n == 1) ? (o & 1) : 0;
                const uint32_t* src =
                    reinterpret_cast<const uint32_t*>(ring + ((copy * 3 + c) * 8 + slot) * kTcfRowCols + o - copy);
                v = make_uint4(src[0], src[1], src[2], src[3]);
            }
            *reinterpret_cast<uint4*>(sA + ci * kTcfKGroup + g * 128 + j * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A visible to the tensor core
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0 && !failed) {
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem + (uint32_t)(16 * c), smem_desc(a0 + (c * 8 + 2 * kk) * kTcfKGroup, kTcfKGroup, 128),
                           smem_desc(b0 + 2 * kk * 256, 256, 128), kTcfIdesc, kk > 0);
            tc_commit(bar);
        }
        // every thread waits for the MMAs of this tile (bounded)
        bool ok = !failed && mbar_wait(bar, (unsigned)(k & 1), wait_ns);
        ok = __syncthreads_and(ok);
        if (!ok) {
            if (t == 0) atomicOr(&g_features_status, 1u);
            failed = true;
            failed_k = k;
            break;
        }
        tc_fence_after();
        // epilogue: this thread's pixel = TMEM lane t
        uint32_t r[48];
        {
            uint32_t q0[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (t >> 5)) << 16), q0, 0);
            tmem_ld_wait(q0);
#pragma unroll
            for (int e = 0; e < 32; ++e) r[e] = q0[e];
            uint32_t q1[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (t >> 5)) << 16), q1, 32);
            tmem_ld_wait(q1);
#pragma unroll
            for (int e = 0; e < 16; ++e) r[32 + e] = q1[e];
        }
        tc_fence_before();
        const int x = x0 + t;
        if (x < w) {
            int words[12];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = ((int)__uint_as_float(r[16 * c + 4 * q + e])) >> qshift;
                    words[4 * c + q] = pack4_sat(v[0], v[1], v[2], v[3]);
                }
            int nn = 0;
#pragma unroll
            for (int e = 0; e < 12; ++e) nn = __dp4a(words[e], words[e], nn);
            const size_t i = (size_t)y * w + x;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                feat[c * cs + i * rs] = make_int4(words[4 * c], words[4 * c + 1], words[4 * c + 2], words[4 * c + 3]);
            norms[i] = nn;
        }
    }
    if (failed && t == 0 && !mbar_wait(bar, (unsigned)(failed_k & 1), kDrainFactor * wait_ns)) {
        // drain: the MMAs of the failed tile complete before the tensor
        // memory is released; a drain that gives up is recorded (bit 1)
        atomicOr(&g_features_status, 2u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t < 32) tmem_dealloc(tmem, kTcfCols);
}

}  // namespace

// Scratch of one image: the smoothed scale space as two int32 planes per
// scale (R + 65536 G, and B).
size_t features_ws_bytes(int w, int h, const sff_params& p) {
    return align256((size_t)2 * p.num_scales * w * h * sizeof(int));
}

// Opts the tensor-core kernels into their dynamic shared memory, once per device.
bool features_tc_ready() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(k_features_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcfSmemBytes) ||
            cudaFuncSetAttribute(k_features_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcfSmemBytes) ||
            cudaFuncSetAttribute(k_features_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcfSmemBytes) ||
            cudaFuncSetAttribute(k_features_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcfSmemBytes))
            return false;
        done[dev] = true;
    }
    return true;
}

// Reads (and with reset clears) the condition bits of the feature kernels,
// in stream order; the caller synchronises the stream.
int features_status_read(cudaStream_t st, unsigned* out, bool reset) {
    static const unsigned zero = 0;
    if (cudaMemcpyFromSymbolAsync(out, g_features_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return SFF_ERR_CUDA;
    if (reset && cudaMemcpyToSymbolAsync(g_features_status, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st) !=
                     cudaSuccess)
        return SFF_ERR_CUDA;
    return SFF_OK;
}

int run_features(const ImageJob* jobs, int n, const sff_params& P, cudaStream_t st, int form, bool smooth, int s_lo,
                 int s_hi, int smooth_lo, int smooth_hi) {
    if (n < 1 || n > kMaxImages || (form != kFeaturesSeparable && form != kFeaturesTensor && form != kFeaturesPairs))
        return SFF_ERR_ARG;
    if (s_hi < 0) s_hi = P.num_scales - 1;
    if (smooth_lo < 0) smooth_lo = s_lo;
    if (s_lo < 0 || s_hi >= P.num_scales || smooth_hi >= P.num_scales || (smooth && smooth_lo > s_lo))
        return SFF_ERR_ARG;
    const int nsmooth_hi = smooth_hi < 0 ? s_hi : smooth_hi;
    if (smooth && nsmooth_hi < s_hi) return SFF_ERR_ARG;  // every computed scale smoothed first
    if (form == kFeaturesTensor && !features_tc_ready()) return SFF_ERR_CUDA;
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
    if (smooth) SFF_LAUNCH(k_smooth, gs, 256, 0, st, J, P.num_scales, smooth_lo, nsmooth_hi);
    for (int s = s_lo; s <= s_hi; ++s) {
        const int nn = 1 << s;
        if (form == kFeaturesTensor) {
            // (segment, residue, tile column) items of the largest image
            const int items = ((mw + kTcfPx - 1) / kTcfPx) * nn * (((mh + nn - 1) / nn + kTcfSeg - 1) / kTcfSeg);
            const dim3 gt(items, 1, n);
            switch (s) {
                case 0: SFF_LAUNCH(k_features_tc<0>, gt, kTcfPx, kTcfSmemBytes, st, J, P.num_scales, P.quant_shift); break;
                case 1: SFF_LAUNCH(k_features_tc<1>, gt, kTcfPx, kTcfSmemBytes, st, J, P.num_scales, P.quant_shift); break;
                case 2: SFF_LAUNCH(k_features_tc<2>, gt, kTcfPx, kTcfSmemBytes, st, J, P.num_scales, P.quant_shift); break;
                default: SFF_LAUNCH(k_features_tc<3>, gt, kTcfPx, kTcfSmemBytes, st, J, P.num_scales, P.quant_shift); break;
            }
            continue;
        }
        if (form == kFeaturesSeparable) {
            // tiles of kSepTY rows per residue class of rows mod n
            const int tiles = ((mh + nn - 1) / nn + kSepTY - 1) / kSepTY;
            dim3 gp((mw + kSepTX - 1) / kSepTX, tiles * nn, n);
            SFF_LAUNCH(k_features_sep, gp, kSepThreads, 0, st, J, s, P.num_scales, P.quant_shift, tiles);
            continue;
        }
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

extern "C" int sff_features_pairs(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                                const sff_params* params, uint8_t* pyramid_dev, void* workspace,
                                size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!rgb_dev || !pyramid_dev || !workspace || pitch_bytes < 3 * width) return SFF_ERR_ARG;
    if (((uintptr_t)pyramid_dev & 15) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < features_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    ImageJob job{rgb_dev, pitch_bytes, width, height, (uint32_t*)workspace, pyramid_dev};
    return run_features(&job, 1, *params, (cudaStream_t)stream, kFeaturesPairs);
}

extern "C" int sff_features_tc(const uint8_t* rgb_dev, int32_t width, int32_t height, int32_t pitch_bytes,
                            const sff_params* params, uint8_t* pyramid_dev, void* workspace,
                            size_t workspace_bytes, void* stream) {
    using namespace sff;
    if (check_size(width, height) || check_params(params)) return SFF_ERR_ARG;
    if (!rgb_dev || !pyramid_dev || !workspace || pitch_bytes < 3 * width) return SFF_ERR_ARG;
    if (((uintptr_t)pyramid_dev & 15) || ((uintptr_t)workspace & 255)) return SFF_ERR_ARG;
    if (workspace_bytes < features_ws_bytes(width, height, *params)) return SFF_ERR_WORKSPACE;
    ImageJob job{rgb_dev, pitch_bytes, width, height, (uint32_t*)workspace, pyramid_dev};
    return run_features(&job, 1, *params, (cudaStream_t)stream, kFeaturesTensor);
}
