// Opt-in per-kernel timing: CUDA events recorded on the launch stream
// before and after each kernel launch, summed per kernel name on collect.
// A span brackets several back-to-back launches of one kernel with a single
// pair of events (the iteration kernel's launches of one scale): on short
// kernels an event node per launch costs more than the launch gap it hides.
// On a stream that is being captured into a CUDA graph the events become
// event-record nodes of the graph (cudaEventRecordExternal), so a replay
// times the kernels as the graph runs them, without the host's launch gaps
// that separate plain launches of short kernels.
#include <mutex>
#include <string>
#include <vector>

#include "sff_internal.cuh"

namespace sff {
namespace {

struct Mark {
    const char* name;
    cudaEvent_t start, stop;
    int launches, units;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Mark> g_marks;
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_pending = nullptr;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void release_all() {
    for (auto& m : g_marks) {
        g_pool.push_back(m.start);
        g_pool.push_back(m.stop);
    }
    g_marks.clear();
    if (g_pending) g_pool.push_back(g_pending);
    g_pending = nullptr;
}

}  // namespace

bool profiling() { return g_on; }

static void record_mark(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void profile_mark(const char* name, cudaStream_t st, bool after, int launches, int units) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!after) {
        g_pending = take_event();
        record_mark(g_pending, st);
    } else {
        cudaEvent_t stop = take_event();
        record_mark(stop, st);
        g_marks.push_back(Mark{name, g_pending, stop, launches, units < 0 ? launches : units});
        g_pending = nullptr;
    }
}

}  // namespace sff

extern "C" int sff_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(sff::g_mu);
    sff::release_all();
    sff::g_on = on != 0;
    return SFF_OK;
}

extern "C" int sff_profile_collect(sff_kernel_time* out, int32_t capacity, int32_t* n_out) {
    if (!n_out || capacity < 0 || (capacity > 0 && !out)) return SFF_ERR_ARG;
    std::lock_guard<std::mutex> lk(sff::g_mu);
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int> count, units;
    int status = SFF_OK;
    for (auto& m : sff::g_marks) {
        if (cudaEventSynchronize(m.stop) != cudaSuccess) status = SFF_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.start, m.stop) != cudaSuccess) status = SFF_ERR_CUDA;
        size_t k = 0;
        while (k < names.size() && names[k] != m.name) ++k;
        if (k == names.size()) {
            names.emplace_back(m.name);
            ms.push_back(0.0);
            count.push_back(0);
            units.push_back(0);
        }
        ms[k] += t;
        count[k] += m.launches;
        units[k] += m.units;
    }
    for (size_t k = 0; k < names.size() && (int)k < capacity; ++k) {
        size_t len = names[k].size() < 39 ? names[k].size() : 39;
        names[k].copy(out[k].name, len);
        out[k].name[len] = 0;
        out[k].launches = count[k];
        out[k].units = units[k];
        out[k].total_ms = ms[k];
    }
    *n_out = (int32_t)names.size();
    sff::release_all();
    return status;
}

// ---------------------------------------------------------------------------
// Integer peaks for the roofline of the matching kernels: dp4a and 32-bit
// multiply-add throughput measured with CUDA events.  Each thread runs eight
// independent dependency chains (enough to hide the pipeline latency with
// several warps per scheduler); a result is stored only when it equals a
// value the inputs never produce, which keeps the chains live.
namespace sff {
namespace {

__device__ int g_peak_sink;

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) k_peak_dp4a(int iters, int seed) {
    int acc[kPeakChains];
    const int b = (int)(threadIdx.x * 0x01010101u) ^ seed;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc[k] = (int)(threadIdx.x + 97 * k + blockIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) acc[k] = __dp4a(acc[k], b, acc[k]);
    }
    int x = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x ^= acc[k];
    if (x == 0x7fedcba9) g_peak_sink = x;
}

__global__ void __launch_bounds__(256) k_peak_imad(int iters, int seed) {
    int acc[kPeakChains];
    const int b = (int)(threadIdx.x | 1u) ^ seed, c = (int)blockIdx.x;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc[k] = (int)(threadIdx.x + 97 * k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) acc[k] = acc[k] * b + c;
    }
    int x = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x ^= acc[k];
    if (x == 0x7fedcba9) g_peak_sink = x;
}

}  // namespace
}  // namespace sff

extern "C" int sff_int_peak(int32_t kind, double* ops_per_s, void* stream) {
    if (!ops_per_s || (kind != 0 && kind != 1)) return SFF_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SFF_ERR_CUDA;
    constexpr int kThreads = 256, kPerSm = 8, kIters = 4096;
    const int blocks = sms * kPerSm;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return SFF_ERR_CUDA;
    int status = SFF_OK;
    float best_ms = 0.f;
    for (int rep = 0; rep < 4 && status == SFF_OK; ++rep) {  // the first launch warms up
        cudaEventRecord(a, st);
        if (kind == 0)
            sff::k_peak_dp4a<<<blocks, kThreads, 0, st>>>(kIters, rep);
        else
            sff::k_peak_imad<<<blocks, kThreads, 0, st>>>(kIters, rep);
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
            status = SFF_ERR_CUDA;
        else if (rep > 0 && (best_ms == 0.f || ms < best_ms))
            best_ms = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (status != SFF_OK || best_ms <= 0.f) return status ? status : SFF_ERR_CUDA;
    const double ops = (double)blocks * kThreads * kIters * 16.0 * sff::kPeakChains;
    *ops_per_s = ops / (best_ms * 1e-3);
    return SFF_OK;
}
