// Parameter defaults, size queries and status strings of the C ABI.
#include "sff_internal.cuh"

namespace sff {

int check_size(int w, int h) {
    if (w < 8 || h < 8 || w > 16384 || h > 16384) return SFF_ERR_ARG;
    return SFF_OK;
}

int check_params(const sff_params* p) {
    if (!p) return SFF_ERR_ARG;
    if (p->num_scales < 1 || p->num_scales > SFF_MAX_SCALES) return SFF_ERR_ARG;
    if (p->iterations < 0 || p->iterations > 64) return SFF_ERR_ARG;
    if (p->tau_c < 0 || p->tau_c > 255 || p->tau_r < 0 || p->tau_r > 255) return SFF_ERR_ARG;
    if (p->region_min < 0) return SFF_ERR_ARG;
    if (p->quant_shift < 0 || p->quant_shift > 8) return SFF_ERR_ARG;
    if (p->knn_temporal < 1 || p->knn_temporal > SFF_MAX_KNN) return SFF_ERR_ARG;
    if (p->knn_epipolar < 1 || p->knn_epipolar > SFF_MAX_KNN) return SFF_ERR_ARG;
    return SFF_OK;
}

int launch_status() { return cudaGetLastError() == cudaSuccess ? SFF_OK : SFF_ERR_CUDA; }

}  // namespace sff

extern "C" int sff_default_params(sff_params* out) {
    if (!out) return SFF_ERR_ARG;
    out->num_scales = 4;   // k = 3 subscales + full resolution (Sec. 5)
    out->iterations = 12;  // per scale (Sec. 5)
    out->tau_c = 1;        // Sec. 5
    out->region_min = 150; // s_c, Sec. 5
    out->tau_r = 1;
    out->quant_shift = 4;
    out->knn_temporal = 4;
    out->knn_epipolar = 2;
    return SFF_OK;
}

extern "C" size_t sff_pyramid_bytes(int32_t width, int32_t height, const sff_params* params) {
    if (sff::check_size(width, height) || sff::check_params(params)) return 0;
    return (size_t)params->num_scales * width * height * SFF_PYRAMID_PIXEL_BYTES;
}

extern "C" size_t sff_workspace_bytes(int32_t width, int32_t height, const sff_params* params) {
    if (sff::check_size(width, height) || sff::check_params(params)) return 0;
    size_t b = sff::features_ws_bytes(width, height, *params);
    size_t m = sff::match_ws_bytes(width, height, *params);
    size_t f = sff::filter_ws_bytes(width, height);
    size_t s = sff::seeds_ws_bytes(width, height);
    if (m > b) b = m;
    if (f > b) b = f;
    if (s > b) b = s;
    return b;
}

extern "C" const char* sff_status_string(int status) {
    switch (status) {
        case SFF_OK: return "ok";
        case SFF_ERR_ARG: return "invalid argument";
        case SFF_ERR_CUDA: return "CUDA error";
        case SFF_ERR_WORKSPACE: return "workspace too small";
        case SFF_ERR_TIMEOUT: return "a bounded device wait gave up";
        case SFF_ERR_CAPACITY: return "seed buffer too small";
        default: return "unknown status";
    }
}

extern "C" int sff_device_status(void* stream, int32_t reset) {
    const cudaStream_t st = (cudaStream_t)stream;
    unsigned m = 0, s = 0, f = 0;
    if (sff::match_status_read(st, &m, reset != 0) != SFF_OK) return SFF_ERR_CUDA;
    if (sff::seeds_status_read(st, &s, reset != 0) != SFF_OK) return SFF_ERR_CUDA;
    if (sff::features_status_read(st, &f, reset != 0) != SFF_OK) return SFF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SFF_ERR_CUDA;
    if ((m & 1u) || f) return SFF_ERR_TIMEOUT;
    if (s) return SFF_ERR_CAPACITY;
    return SFF_OK;
}
