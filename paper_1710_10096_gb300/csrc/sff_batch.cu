// The whole stage for a batch of quads of any sizes (up to 32): features of
// all 4n images, both fields of all n quads, the filter and the seeds, each
// phase in shared launches (blockIdx.z selects the image / field / quad), so
// small quads and coarse scales fill the GPU together and one CUDA graph can
// hold the whole batch.  Every quad's outputs are identical to running the
// four calls on it alone.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "sff_internal.cuh"

namespace sff {

// Per-quad scratch: the smoothed images of the four views (read by the
// features of every scale), then the two fields' scratch, which the features
// of the finer scales may still be reading from the first part; the filter
// and, after it, the seeds, which run after both, reuse the start (the seeds'
// scratch follows the filter's: the seed kernels read the filter's union-find
// arrays).
size_t quad_ws_bytes(int w, int h, const sff_params& p) {
    size_t b = 4 * features_ws_bytes(w, h, p) + 2 * field_ws_bytes(w, h, p);
    b = std::max(b, filter_ws_bytes(w, h) + seeds_ws_bytes(w, h));
    return b;
}

namespace {

// The second stream of the feature overlap and its events, one set per
// (device, caller stream), created at the first call on that pair and kept
// until exit.  Calls on one caller stream are issued in host order, so they
// may reuse the set.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t ready[SFF_MAX_SCALES] = {};
};

std::mutex g_side_mu;
std::map<std::pair<int, cudaStream_t>, SideStream> g_side;

// The set of the current device and `st`, or nullptr when it cannot be made.
const SideStream* side_stream(cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_side_mu);
    auto it = g_side.find({dev, st});
    if (it != g_side.end()) return &it->second;
    SideStream ss;
    bool ok = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < SFF_MAX_SCALES; ++k)
        ok = cudaEventCreateWithFlags(&ss.ready[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    return &g_side.emplace(std::make_pair(dev, st), ss).first->second;
}

// The feature overlap of one sff_run_batch call (sff_tuning.overlap).
struct Fork {
    const SideStream* side;
    const ImageJob* img;
    int n_img;
    const sff_params* P;
    int form;
    int joined_at;  // the last scale whose event the second stream recorded (-1: none)
};

// ForkHook of run_fields (before the K-NN): forks the second stream from
// `main` and issues the features of scales S - 2 .. 0 on it, coarse to
// fine, each followed by its event.  Every event is recorded even after a
// failed launch, so that the caller's stream always joins the second one
// (a capture stays whole).
int fork_features(void* ctx, cudaStream_t main) {
    Fork& f = *static_cast<Fork*>(ctx);
    if (cudaEventRecord(f.side->fork, main) != cudaSuccess || cudaStreamWaitEvent(f.side->s, f.side->fork, 0) != cudaSuccess)
        return SFF_ERR_CUDA;
    int status = SFF_OK;
    for (int s = f.P->num_scales - 2; s >= 0; --s) {
        const int st_s = run_features(f.img, f.n_img, *f.P, f.side->s, f.form, false, s, s);
        if (!status) status = st_s;
        if (cudaEventRecord(f.side->ready[s], f.side->s) != cudaSuccess && !status) status = SFF_ERR_CUDA;
        f.joined_at = s;
    }
    return status;
}

}  // namespace

}  // namespace sff

extern "C" size_t sff_quad_workspace_bytes(int32_t width, int32_t height, const sff_params* params) {
    if (sff::check_size(width, height) || sff::check_params(params)) return 0;
    return sff::quad_ws_bytes(width, height, *params);
}

extern "C" int sff_run_batch(const sff_quad* quads, int32_t n, const sff_params* params, const sff_tuning* tuning,
                             void* stream) {
    using namespace sff;
    if (!quads || n < 1 || n > SFF_MAX_BATCH || n > kMaxQuads || check_params(params)) return SFF_ERR_ARG;
    sff_tuning t;
    if (tuning) {
        t = *tuning;
    } else {
        sff_default_tuning(&t);
    }
    if (!sff_tuning_supported(&t)) return SFF_ERR_ARG;
    const sff_params& P = *params;
    for (int k = 0; k < n; ++k) {
        const sff_quad& q = quads[k];
        if (check_size(q.width, q.height) || q.pitch_bytes < 3 * q.width || !q.workspace || q.capacity < 0)
            return SFF_ERR_ARG;
        for (int j = 0; j < 4; ++j)
            if (!q.rgb[j] || !q.pyramid[j] || ((uintptr_t)q.pyramid[j] & 15)) return SFF_ERR_ARG;
        if (!q.fwd || !q.inv || !q.fwd_cost || !q.inv_cost || !q.keep || !q.cerr || !q.count ||
            (q.capacity > 0 && !q.seeds))
            return SFF_ERR_ARG;
        if (((uintptr_t)q.fwd & 7) || ((uintptr_t)q.inv & 7) || ((uintptr_t)q.fwd_cost & 3) ||
            ((uintptr_t)q.inv_cost & 3) || ((uintptr_t)q.workspace & 255) || ((uintptr_t)q.seeds & 3))
            return SFF_ERR_ARG;
        if (q.workspace_bytes < quad_ws_bytes(q.width, q.height, P)) return SFF_ERR_WORKSPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;

    // features of all images
    ImageJob img[kMaxImages];
    for (int k = 0; k < n; ++k) {
        const sff_quad& q = quads[k];
        const size_t fw = features_ws_bytes(q.width, q.height, P);
        for (int j = 0; j < 4; ++j)
            img[4 * k + j] = ImageJob{q.rgb[j], q.pitch_bytes, q.width, q.height,
                                      reinterpret_cast<uint32_t*>((char*)q.workspace + j * fw), q.pyramid[j]};
    }
    static_assert(kFeaturesSeparable == 0 && kFeaturesTensor == 1 && kFeaturesPairs == 2,
                  "sff_tuning.features_form values");
    // With the overlap, the stream smooths the images (every scale: smoothing
    // the finer scales on the second stream instead made the step slower, as
    // the features then ran later, beside more of the iterations), computes
    // the coarsest scale's features (the K-NN and the first iterations read
    // only those) and gathers the
    // coarsest grid; then the finer scales' features run on the second
    // stream, coarse to fine, one event per scale, beside the K-NN (which
    // leaves SMs idle), the initialisation and the coarse iterations.  The
    // inheritance into scale s waits for event s, and the wait on the finest
    // scale's event joins the two streams again.  (Forked before the grid is
    // gathered instead, the step took the same time: the features' CTAs then
    // delayed the gathering rather than the K-NN.  Holding the features of
    // scales 1 and 0 back until the coarsest scale is matched sped up its
    // fused iterations but slowed scale 1's more: 1.406 against 1.351 ms.)
    const int S = P.num_scales;
    const SideStream* side = t.overlap && S > 1 ? side_stream(st) : nullptr;
    int status = side ? run_features(img, 4 * n, P, st, t.features_form, true, S - 1, S - 1, 0, S - 1)
                      : run_features(img, 4 * n, P, st, t.features_form);
    if (status) return status;
    Fork fork{side, img, 4 * n, &P, t.features_form, -1};
    const ForkHook hook{fork_features, &fork};

    // both fields of every quad (pyramids in the order L0, R0, L1, R1)
    FieldSpec fs[kMaxBatchFields];
    for (int k = 0; k < n; ++k) {
        const sff_quad& q = quads[k];
        char* ws = reinterpret_cast<char*>(q.workspace) + 4 * features_ws_bytes(q.width, q.height, P);
        const size_t half = field_ws_bytes(q.width, q.height, P);
        fs[2 * k] = FieldSpec{q.pyramid[0], q.pyramid[2], q.pyramid[1], q.pyramid[3], q.fwd, q.fwd_cost, 0,
                              q.width,      q.height,     q.seed,       ws};
        fs[2 * k + 1] = FieldSpec{q.pyramid[3], q.pyramid[1], q.pyramid[2], q.pyramid[0], q.inv, q.inv_cost, 1,
                                  q.width,      q.height,     q.seed,       ws + half};
    }
    status = run_fields(fs, 2 * n, P, t, st, false, side ? side->ready : nullptr, side ? &hook : nullptr);
    // joined already, unless run_fields failed early
    if (fork.joined_at >= 0) cudaStreamWaitEvent(st, side->ready[fork.joined_at], 0);
    if (status) return status;

    // consistency + region filter, then seeds
    FilterJob fj[kMaxQuads];
    SeedJob sj[kMaxQuads];
    for (int k = 0; k < n; ++k) {
        const sff_quad& q = quads[k];
        fj[k] = FilterJob{reinterpret_cast<const uint2*>(q.fwd), q.fwd_cost, reinterpret_cast<const uint2*>(q.inv),
                          q.inv_cost, q.width, q.height, q.keep, q.cerr, nullptr, nullptr, nullptr};
        filter_carve(q.workspace, q.width, q.height, &fj[k].parent, &fj[k].size, &fj[k].joinable);
    }
    // the removal of small joinable regions is done by the seed kernels
    status = run_filter(fj, n, P, st, false);
    if (status) return status;
    for (int k = 0; k < n; ++k) {
        const sff_quad& q = quads[k];
        sj[k] = SeedJob{reinterpret_cast<const uint2*>(q.fwd), q.fwd_cost, q.keep, q.cerr, q.width, q.height,
                        nullptr, nullptr, q.seeds, q.capacity, q.count, nullptr, 0,
                        fj[k].parent, fj[k].size, fj[k].joinable, P.region_min, q.keep};
        seeds_carve(reinterpret_cast<char*>(q.workspace) + filter_ws_bytes(q.width, q.height), q.width, q.height,
                    &sj[k].best, &sj[k].chunk);
    }
    return run_seeds(sj, n, st);
}
