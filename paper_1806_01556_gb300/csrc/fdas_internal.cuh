// Internal declarations shared by the FDAS CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/fdas.h"

namespace fdas {

// The last CUDA error met on this thread (fdas_last_error): note() records e with the function and
// line that met it and returns e unchanged; fail() turns e into a status, recording it unless the
// record already holds the same error from a deeper call.
cudaError_t note(cudaError_t e, const char *where, int line);
fdas_status fail(cudaError_t e, const char *where, int line);
#define FDAS_NOTE(e) ::fdas::note((e), __func__, __LINE__)
#define FDAS_STATUS(e) ::fdas::fail((e), __func__, __LINE__)

// Derived sizes of one parameter set.
struct Geometry {
    int n_temp;   // template rows
    int c;        // centre row (zero drift), (n_temp-1)/2
    int n_tap;    // taps per template
    int h;        // half width, (n_tap-1)/2
    int fft_len;  // overlap-save segment length F
    int keep;     // valid outputs per segment, L = F - n_tap + 1
    int precision;  // FDAS_FP32, FDAS_BF16X3 or FDAS_FP16S
};

inline Geometry geometry(const fdas_params &p) {
    Geometry g;
    g.n_temp = p.n_temp;
    g.c = (p.n_temp - 1) / 2;
    g.n_tap = p.n_tap;
    g.h = (p.n_tap - 1) / 2;
    g.fft_len = p.fft_len;
    g.keep = p.fft_len - p.n_tap + 1;
    g.precision = p.precision;
    return g;
}

// Workspace layout of the harmonic-sum stage (all 8-byte words):
//   [0, n_harm)                 raw crossing counters (low 32 bits used)
//   [n_harm, 2 n_harm)          peak keys, one per plane
//   [4 n_harm, 4 n_harm + n_harm*FDAS_RAW_CAP)  raw candidate keys, FDAS_RAW_CAP per plane
struct HsWorkspace {
    unsigned long long *counters;
    unsigned long long *peaks;
    unsigned long long *raw;
};

inline HsWorkspace hs_workspace(void *ws, int n_harm) {
    unsigned long long *w = static_cast<unsigned long long *>(ws);
    return HsWorkspace{w, w + n_harm, w + 4 * n_harm};
}

inline size_t hs_workspace_words(int n_harm) { return (size_t)n_harm * (FDAS_RAW_CAP + 4); }

// Largest batch: the per-spectrum tables travel as kernel parameters (a few KB to 20 KB).
constexpr int kMaxBatch = FDAS_MAX_BATCH;

// One spectrum of a batch, as the batched convolution kernel reads it.
struct ConvJob {
    const float2 *spec;
    float *plane;
    unsigned long long ld;
    int n;
    int item0;  // first work item of this spectrum in the batch
    // This spectrum's harmonic-sum workspace (HsWorkspace), for HP_1 taken in the convolution.
    unsigned long long *counters;
    unsigned long long *peaks;
    unsigned long long *raw;
};
struct ConvBatch {
    int count;
    int total_items;
    ConvJob job[kMaxBatch];
};

// One spectrum of a batch, as the batched harmonic-sum kernels read it.
struct HsJob {
    const float *plane;
    unsigned long long ld;
    int n;
    int blk0;   // first CTA of this spectrum in harmonic-sum launches of 12288-column CTAs
    int blk1;   // first CTA of this spectrum in harmonic-sum launches of 4096-column CTAs
    int blk2;   // first CTA of this spectrum in harmonic-sum launches of 16384-column CTAs
    unsigned long long *counters;  // this spectrum's workspace (HsWorkspace)
    unsigned long long *peaks;
    unsigned long long *raw;
    fdas_cand *cands;
    uint32_t *counts;
    fdas_cand *peak_out;
};
struct HsBatch {
    int count;
    HsJob job[kMaxBatch];
};

// Kernel launchers (each returns cudaGetLastError() of its launch).
cudaError_t launch_templates(const fdas_params &p, void *d_tmpl, cudaStream_t s);
// Convolution launch for g.precision: the FP32 kernel or the tensor-core kernel.
cudaError_t launch_convolve(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                            size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s);
cudaError_t launch_convolve_fp32(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl,
                                 float *plane, size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s);
// Tensor-core form: one CTA per SM (all of Tensor Memory), default 44 templates per work item.
constexpr int kTcMaxCtasPerSm = 1;
constexpr int kTcDefaultTemplatesPerItem = 44;
cudaError_t launch_convolve_tc(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                               size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s);
cudaError_t prepare_convolve_batch_tc();
cudaError_t launch_convolve_batch_tc(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                     int templates_per_item, cudaStream_t s);
cudaError_t device_status_tc(unsigned *flags, bool clear);
cudaError_t device_status_tc_async(unsigned *h_flags, cudaStream_t s);
// Resident CTAs per SM of the convolution kernel for g.precision.
inline int convolve_ctas_per_sm(const Geometry &g) { return g.precision == FDAS_FP32 ? 3 : kTcMaxCtasPerSm; }
// Zeroes the harmonic-sum workspace's counters and peak keys.
cudaError_t launch_hs_reset(const fdas_params &p, const HsWorkspace &ws, cudaStream_t s);
// FP32 convolution that also emits, for the single-plane rows (|i| > c/2; all rows when n_harm = 1),
// the HP_1 candidates (threshold thresh[0..n_temp), when bit 0 of harm_mask is set) and their HP_1
// peak into the workspace, which must have been reset.
cudaError_t launch_convolve_hp1(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                                size_t ld, const float *thresh, unsigned harm_mask, int n_harm, const HsWorkspace &ws,
                                cudaStream_t s);
// Status bits set by kernels on the device (bit 0: a bounded wait timed out); optionally cleared.
cudaError_t device_status(unsigned *flags, bool clear);
// Enqueues on s copies of the two translation units' status words into h_flags2[0] and h_flags2[1]
// (valid once s reaches them; with pageable host memory the call itself waits for that).
cudaError_t device_status_async(unsigned *h_flags2, cudaStream_t s);
// Sets the status word to flags (the tensor-core unit's word is cleared).
cudaError_t set_device_status(unsigned flags);
// FP32 FFMA-chain throughput of the current device over about ms milliseconds (diag.cu).
cudaError_t measure_fp32_peak(float ms, double *tflops, float *elapsed_ms);
// Runs a kernel whose bounded wait must give up; returns the status bits it left (then cleared).
cudaError_t check_wait_timeout(unsigned *flags);
// Batched convolution: one persistent launch over every segment of every spectrum.
cudaError_t prepare_convolve_batch();
int convolve_items(const Geometry &g, size_t n, int templates_per_item);
cudaError_t launch_convolve_batch(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                  int templates_per_item, cudaStream_t s);
// The FP32 batched convolution that also takes HP_1 of every spectrum's single-plane rows into its
// workspace (ConvJob counters / peaks / raw, reset beforehand).
cudaError_t launch_convolve_batch_hp1(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                      int templates_per_item, const float *thresh, unsigned harm_mask, int n_harm,
                                      cudaStream_t s);
// Harmonic sum. With hp1_done the workspace was reset before the convolution, which already took
// HP_1 of the single-plane rows (launch_convolve_hp1). With concurrent the row-group launches run
// side by side on two auxiliary streams of the library (one pair per host thread, context and caller
// stream).
cudaError_t launch_harmonic(const fdas_params &p, const float *plane, size_t n, size_t ld,
                            const float *thresh, fdas_cand *cands, uint32_t *counts, fdas_cand *peaks,
                            const HsWorkspace &ws, cudaStream_t s, bool hp1_done = false, bool concurrent = true);
// fdas_harmonic_sum with the choice of concurrent launches (fdas_harmonic_sum_noalloc: none).
fdas_status harmonic_sum_checked(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                 const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                                 void *d_ws, size_t ws_bytes, cudaStream_t stream, bool concurrent);
// Creates the calling thread's auxiliary streams of the harmonic sum for caller stream s on the
// current context, unless they exist or s is being captured.
cudaError_t prepare_streams(cudaStream_t s);
// The driver's id of the current device's context (made current if it is not), unique for the life
// of the process: caches keyed by it never hand out a resource of a context that cudaDeviceReset
// destroyed.
cudaError_t current_context_id(unsigned long long *id);
// Batched harmonic sum: reset, one launch per group of rows over every spectrum, finalize.
void harmonic_blocks(const fdas_params &p, size_t n, int *blocks_16k, int *blocks_12k, int *blocks_4k);
cudaError_t prepare_harmonic_batch();
// hp1_done: the workspaces were reset before the convolution, which took HP_1 of the single-plane
// rows (launch_convolve_batch_hp1); no reset and no single-plane launch run here then.
cudaError_t launch_harmonic_batch(const fdas_params &p, const HsBatch &batch, int total_16k, int total_12k,
                                  int total_4k, const float *thresh, cudaStream_t s, bool hp1_done = false);
// Zeroes every spectrum's counters and peak keys.
cudaError_t launch_hs_reset_batch(const fdas_params &p, const HsBatch &batch, cudaStream_t s);

}  // namespace fdas
