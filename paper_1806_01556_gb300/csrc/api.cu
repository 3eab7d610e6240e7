// C ABI entry points of libfdas: argument checks, workspace carving and kernel launches.
// Declarations and the full contract of each call are in include/fdas.h.
#include <cuda.h>  // driver API types only; the entry points are looked up through the runtime

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fdas_internal.cuh"

using fdas::Geometry;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fdas_status check_shape(const fdas_params *p, size_t n, size_t ld) {
    if (n < 1 || n > FDAS_MAX_N || ld < n) return FDAS_ERR_INVALID_ARG;
    if ((unsigned long long)ld * (unsigned long long)p->n_temp > (1ull << 40)) return FDAS_ERR_INVALID_ARG;
    return FDAS_OK;
}

#define cuda_status(e) FDAS_STATUS(e)

struct LastError {
    cudaError_t code;
    char text[320];
};
thread_local LastError g_last_error{cudaSuccess, {0}};

// S_k(x) = P(Gamma(k,1) > x) = exp(-x) sum_{m<k} x^m / m!, integer k >= 1.
double gamma_survival(int k, double x) {
    double term = 1.0, total = 1.0;
    for (int m = 1; m < k; ++m) {
        term *= x / m;
        total += term;
    }
    return std::exp(-x) * total;
}

// The x > 0 with S_k(x) = p, by bisection (S_k decreases strictly from 1 to 0).
double gamma_threshold(int k, double p) {
    double lo = 0.0, hi = 1.0;
    while (gamma_survival(k, hi) > p) hi *= 2.0;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (gamma_survival(k, mid) > p)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

cudaError_t fdas::note(cudaError_t e, const char *where, int line) {
    if (e == cudaSuccess) return e;
    // An outer frame passing on the error a deeper call recorded keeps the deeper location.
    if (e != g_last_error.code) {
        g_last_error.code = e;
        std::snprintf(g_last_error.text, sizeof(g_last_error.text), "%s (%s) in %s, line %d", cudaGetErrorName(e),
                      cudaGetErrorString(e), where, line);
    }
    // The runtime keeps the error as this thread's last error too; clear it, so that a later launch
    // check (cudaGetLastError) does not report it again. A sticky error stays regardless.
    (void)cudaGetLastError();
    return e;
}

fdas_status fdas::fail(cudaError_t e, const char *where, int line) {
    if (e == cudaSuccess) return FDAS_OK;
    note(e, where, line);
    return FDAS_ERR_CUDA;
}

cudaError_t fdas::current_context_id(unsigned long long *id) {
    // cuCtxGetCurrent and cuCtxGetId from the driver, through the runtime (no link to libcuda).
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static cudaError_t init = cudaErrorUnknown;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        init = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (init == cudaSuccess) init = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (init == cudaSuccess && (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2))
            init = cudaErrorNotSupported;
        get_current = reinterpret_cast<GetCurrent>(f1);
        get_id = reinterpret_cast<GetId>(f2);
    });
    if (init != cudaSuccess) return init;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    if (ctx == nullptr) {
        // No context is current on this thread yet: cudaSetDevice makes the device's primary context
        // current (and creates it if needed).
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorUnknown;
    }
    return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

fdas_status fdas::harmonic_sum_checked(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                       const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts,
                                       fdas_cand *d_peaks, void *d_ws, size_t ws_bytes, cudaStream_t stream,
                                       bool concurrent) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_plane || !d_thresh || !d_cands || !d_counts || !d_ws) return FDAS_ERR_INVALID_ARG;
    if (!aligned16(d_plane) || !aligned16(d_ws) || ((uintptr_t)d_thresh & 3u) || ((uintptr_t)d_cands & 3u) ||
        ((uintptr_t)d_counts & 3u) || ((uintptr_t)d_peaks & 3u))
        return FDAS_ERR_INVALID_ARG;
    if (ws_bytes < fdas_workspace_bytes(p, n)) return FDAS_ERR_WORKSPACE;
    const fdas::HsWorkspace ws = fdas::hs_workspace(d_ws, p->n_harm);
    return cuda_status(fdas::launch_harmonic(*p, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, ws, stream,
                                             false, concurrent));
}

extern "C" {

void fdas_default_params(fdas_params *p) {
    if (!p) return;
    p->n_temp = 85;
    p->z_min = -42;
    p->z_step = 1;
    p->n_tap = 421;
    p->fft_len = 2048;
    p->n_harm = 8;
    p->harm_mask = 0xFFu;
    p->cand_cap = 200;
    p->precision = FDAS_FP32;
    p->harm_index = FDAS_INDEX_FUNDAMENTAL;
}

fdas_status fdas_check_params(const fdas_params *p) {
    if (!p) return FDAS_ERR_INVALID_ARG;
    if (p->n_temp < 3 || p->n_temp > 255 || (p->n_temp & 1) == 0) return FDAS_ERR_INVALID_ARG;
    if (p->z_step < 1 || p->z_step > 1024) return FDAS_ERR_INVALID_ARG;
    if ((long long)p->z_min != -(long long)((p->n_temp - 1) / 2) * p->z_step) return FDAS_ERR_INVALID_ARG;
    if (p->fft_len < 64 || p->fft_len > 8192 || (p->fft_len & (p->fft_len - 1)) != 0) return FDAS_ERR_INVALID_ARG;
    if (p->n_tap < 3 || (p->n_tap & 1) == 0 || p->n_tap > p->fft_len / 2) return FDAS_ERR_INVALID_ARG;
    if (p->n_harm < 1 || p->n_harm > FDAS_MAX_HARM) return FDAS_ERR_INVALID_ARG;
    if (p->harm_mask == 0u || (p->n_harm < 32 && (p->harm_mask >> p->n_harm) != 0u)) return FDAS_ERR_INVALID_ARG;
    if (p->cand_cap < 1 || p->cand_cap > FDAS_MAX_CAND_CAP) return FDAS_ERR_INVALID_ARG;
    if (p->precision != FDAS_FP32 && p->precision != FDAS_BF16X3 && p->precision != FDAS_FP16S)
        return FDAS_ERR_INVALID_ARG;
    if (p->harm_index != FDAS_INDEX_FUNDAMENTAL && p->harm_index != FDAS_INDEX_HIGHEST) return FDAS_ERR_INVALID_ARG;
    if (p->fft_len != 2048) return FDAS_ERR_UNSUPPORTED;
    return FDAS_OK;
}

const char *fdas_last_error(void) { return g_last_error.text; }

const char *fdas_status_string(fdas_status s) {
    switch (s) {
        case FDAS_OK: return "ok";
        case FDAS_ERR_INVALID_ARG: return "invalid argument";
        case FDAS_ERR_UNSUPPORTED: return "unsupported parameters";
        case FDAS_ERR_WORKSPACE: return "workspace too small";
        case FDAS_ERR_CUDA: return "CUDA error";
        case FDAS_ERR_TIMEOUT: return "a kernel gave up on a bounded device wait";
        default: return "unknown status";
    }
}

fdas_status fdas_device_status(uint32_t *flags, int clear) {
    if (!flags) return FDAS_ERR_INVALID_ARG;
    unsigned v = 0u;
    if (const fdas_status st = cuda_status(fdas::device_status(&v, clear != 0))) return st;
    *flags = v;
    return FDAS_OK;
}

fdas_status fdas_set_device_status(uint32_t flags) {
    return cuda_status(fdas::set_device_status(flags));
}

fdas_status fdas_measure_fp32_peak(float ms, double *tflops, float *elapsed_ms) {
    if (!tflops || !elapsed_ms || !(ms >= 10.0f) || ms > 2000.0f) return FDAS_ERR_INVALID_ARG;
    return cuda_status(fdas::measure_fp32_peak(ms, tflops, elapsed_ms));
}

fdas_status fdas_check_wait_timeout(uint32_t *flags) {
    if (!flags) return FDAS_ERR_INVALID_ARG;
    unsigned v = 0u;
    if (const fdas_status st = cuda_status(fdas::check_wait_timeout(&v))) return st;
    *flags = v;
    return FDAS_OK;
}

size_t fdas_templates_bytes(const fdas_params *p) {
    if (fdas_check_params(p) == FDAS_ERR_INVALID_ARG) return 0;
    return (size_t)(p->n_temp + 1) * (size_t)p->fft_len * 8u;
}

size_t fdas_plane_bytes(const fdas_params *p, size_t n, size_t ld) {
    if (fdas_check_params(p) == FDAS_ERR_INVALID_ARG || ld < n) return 0;
    return (size_t)p->n_temp * ld * 4u;
}

size_t fdas_workspace_bytes(const fdas_params *p, size_t n) {
    (void)n;
    if (fdas_check_params(p) == FDAS_ERR_INVALID_ARG) return 0;
    return fdas::hs_workspace_words(p->n_harm) * 8u;
}

fdas_status fdas_default_thresholds(const fdas_params *p, double sigma, int kind, float *h_thresh) {
    fdas_status st = fdas_check_params(p);
    if (st == FDAS_ERR_INVALID_ARG) return st;
    if (!h_thresh || !(sigma > 0.0) || sigma > 30.0 || (kind != 0 && kind != 1)) return FDAS_ERR_INVALID_ARG;
    const double tail = 0.5 * std::erfc(sigma / std::sqrt(2.0));
    for (int k = 1; k <= p->n_harm; ++k) {
        const double v = kind == 0 ? gamma_threshold(k, tail) : k + sigma * std::sqrt((double)k);
        for (int t = 0; t < p->n_temp; ++t) h_thresh[(size_t)(k - 1) * p->n_temp + t] = (float)v;
    }
    return FDAS_OK;
}

fdas_status fdas_make_templates(const fdas_params *p, void *d_tmpl, fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if (!d_tmpl || !aligned16(d_tmpl)) return FDAS_ERR_INVALID_ARG;
    // The harmonic sum's auxiliary streams for this thread and stream, made here so that a later
    // graph capture of a search on the same stream finds them.
    if (const fdas_status st = cuda_status(fdas::prepare_streams(stream))) return st;
    return cuda_status(fdas::launch_templates(*p, d_tmpl, stream));
}

fdas_status fdas_convolve_cfg(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl, float *d_plane,
                              size_t ld, const fdas_launch_config *cfg, fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_spec || !d_tmpl || !d_plane) return FDAS_ERR_INVALID_ARG;
    if (!aligned16(d_spec) || !aligned16(d_tmpl) || !aligned16(d_plane)) return FDAS_ERR_INVALID_ARG;
    const int ctas = cfg ? cfg->ctas_per_sm : 0;
    const int tpi = cfg ? cfg->templates_per_item : 0;
    if (ctas < 0 || ctas > 64 || tpi < 0) return FDAS_ERR_INVALID_ARG;
    const Geometry g = fdas::geometry(*p);
    return cuda_status(fdas::launch_convolve(g, static_cast<const float2 *>(d_spec), n,
                                             static_cast<const float2 *>(d_tmpl), d_plane, ld, ctas, tpi, stream));
}

fdas_status fdas_convolve(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl, float *d_plane,
                          size_t ld, fdas_stream_t stream) {
    return fdas_convolve_cfg(p, d_spec, n, d_tmpl, d_plane, ld, nullptr, stream);
}

fdas_status fdas_harmonic_sum(const fdas_params *p, const float *d_plane, size_t n, size_t ld, const float *d_thresh,
                              fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks, void *d_ws, size_t ws_bytes,
                              fdas_stream_t stream) {
    return fdas::harmonic_sum_checked(p, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes, stream,
                                      true);
}

fdas_status fdas_search_convolve(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl,
                                 float *d_plane, size_t ld, const float *d_thresh, void *d_ws, size_t ws_bytes,
                                 fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_spec || !d_tmpl || !d_plane || !d_thresh || !d_ws) return FDAS_ERR_INVALID_ARG;
    if (!aligned16(d_spec) || !aligned16(d_tmpl) || !aligned16(d_plane) || !aligned16(d_ws)) return FDAS_ERR_INVALID_ARG;
    if ((uintptr_t)d_thresh & 3u) return FDAS_ERR_INVALID_ARG;
    if (ws_bytes < fdas_workspace_bytes(p, n)) return FDAS_ERR_WORKSPACE;
    const Geometry g = fdas::geometry(*p);
    const fdas::HsWorkspace ws = fdas::hs_workspace(d_ws, p->n_harm);
    cudaError_t e = fdas::launch_hs_reset(*p, ws, stream);
    if (e != cudaSuccess) return cuda_status(e);
    const float2 *spec = static_cast<const float2 *>(d_spec);
    const float2 *tmpl = static_cast<const float2 *>(d_tmpl);
    if (g.precision == FDAS_FP32 && p->harm_index == FDAS_INDEX_FUNDAMENTAL)
        e = fdas::launch_convolve_hp1(g, spec, n, tmpl, d_plane, ld, d_thresh, p->harm_mask, p->n_harm, ws, stream);
    else
        e = fdas::launch_convolve(g, spec, n, tmpl, d_plane, ld, 0, 0, stream);
    return cuda_status(e);
}

fdas_status fdas_search_harmonic(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                 const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                                 void *d_ws, size_t ws_bytes, fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_plane || !d_thresh || !d_cands || !d_counts || !d_ws) return FDAS_ERR_INVALID_ARG;
    if (!aligned16(d_plane) || !aligned16(d_ws) || ((uintptr_t)d_thresh & 3u) || ((uintptr_t)d_cands & 3u) ||
        ((uintptr_t)d_counts & 3u) || ((uintptr_t)d_peaks & 3u))
        return FDAS_ERR_INVALID_ARG;
    if (ws_bytes < fdas_workspace_bytes(p, n)) return FDAS_ERR_WORKSPACE;
    const fdas::HsWorkspace ws = fdas::hs_workspace(d_ws, p->n_harm);
    return cuda_status(fdas::launch_harmonic(*p, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, ws, stream,
                                             /*hp1_done=*/p->precision == FDAS_FP32 &&
                                                 p->harm_index == FDAS_INDEX_FUNDAMENTAL));
}

fdas_status fdas_search(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl, float *d_plane,
                        size_t ld, const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                        void *d_ws, size_t ws_bytes, fdas_stream_t stream) {
    // Check everything before enqueueing anything.
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_spec || !d_tmpl || !d_plane || !d_thresh || !d_cands || !d_counts || !d_ws) return FDAS_ERR_INVALID_ARG;
    if (!aligned16(d_spec) || !aligned16(d_tmpl) || !aligned16(d_plane) || !aligned16(d_ws)) return FDAS_ERR_INVALID_ARG;
    if (((uintptr_t)d_thresh & 3u) || ((uintptr_t)d_cands & 3u) || ((uintptr_t)d_counts & 3u) ||
        ((uintptr_t)d_peaks & 3u))
        return FDAS_ERR_INVALID_ARG;
    if (ws_bytes < fdas_workspace_bytes(p, n)) return FDAS_ERR_WORKSPACE;
    st = fdas_search_convolve(p, d_spec, n, d_tmpl, d_plane, ld, d_thresh, d_ws, ws_bytes, stream);
    if (st != FDAS_OK) return st;
    return fdas_search_harmonic(p, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes, stream);
}

fdas_status fdas_search_host(const fdas_params *p, const void *h_spec, size_t n, void *d_spec, const void *d_tmpl,
                             float *d_plane, size_t ld, const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts,
                             fdas_cand *d_peaks, fdas_cand *h_cands, uint32_t *h_counts, fdas_cand *h_peaks,
                             void *d_ws, size_t ws_bytes, fdas_stream_t stream) {
    const fdas_status st = fdas_search_host_async(p, h_spec, n, d_spec, d_tmpl, d_plane, ld, d_thresh, d_cands, d_counts,
                                                  d_peaks, h_cands, h_counts, h_peaks, d_ws, ws_bytes, stream);
    if (st != FDAS_OK) return st;
    // The device status words, read on the same stream behind the search.
    unsigned flags[2] = {0u, 0u};
    cudaError_t e = fdas::device_status_async(flags, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    return ((flags[0] | flags[1]) & FDAS_DEV_WAIT_TIMEOUT) ? FDAS_ERR_TIMEOUT : FDAS_OK;
}

fdas_status fdas_search_host_async(const fdas_params *p, const void *h_spec, size_t n, void *d_spec,
                                   const void *d_tmpl, float *d_plane, size_t ld, const float *d_thresh,
                                   fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks, fdas_cand *h_cands,
                                   uint32_t *h_counts, fdas_cand *h_peaks, void *d_ws, size_t ws_bytes,
                                   fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if (!h_spec || !h_cands || !h_counts || (h_peaks && !d_peaks)) return FDAS_ERR_INVALID_ARG;
    if ((st = check_shape(p, n, ld)) != FDAS_OK) return st;
    if (!d_spec || !aligned16(d_spec)) return FDAS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(d_spec, h_spec, n * 8u, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_status(e);
    st = fdas_search(p, d_spec, n, d_tmpl, d_plane, ld, d_thresh, d_cands, d_counts, d_peaks, d_ws, ws_bytes, stream);
    if (st != FDAS_OK) return st;
    const size_t cand_bytes = (size_t)p->n_harm * p->cand_cap * sizeof(fdas_cand);
    if ((e = cudaMemcpyAsync(h_cands, d_cands, cand_bytes, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(h_counts, d_counts, p->n_harm * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream)) !=
        cudaSuccess)
        return cuda_status(e);
    if (h_peaks && (e = cudaMemcpyAsync(h_peaks, d_peaks, p->n_harm * sizeof(fdas_cand), cudaMemcpyDeviceToHost,
                                        stream)) != cudaSuccess)
        return cuda_status(e);
    return FDAS_OK;
}

}  // extern "C"
