// Batched FDAS search: many spectra of uneven length in one launch per stage, a plan object that
// replays the launches as a CUDA graph, and an autotuner for the convolution's launch shape.
// Declarations and the full contract are in include/fdas.h.
#include <cstdlib>
#include <cstring>
#include <new>

#include "fdas_internal.cuh"

using fdas::ConvBatch;
using fdas::HsBatch;

namespace {

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

size_t hs_ws_stride(const fdas_params &p) { return (fdas::hs_workspace_words(p.n_harm) * 8u + 255u) / 256u * 256u; }

// with_spec: the items' spectra and the template bank are used (a search); without, only the planes
// are read (a harmonic sum).
fdas_status check_items(const fdas_params *p, const fdas_batch_item *items, int count, const void *d_tmpl,
                        const float *d_thresh, void *d_ws, size_t ws_bytes, bool with_spec = true) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if (p->harm_index != FDAS_INDEX_FUNDAMENTAL) return FDAS_ERR_UNSUPPORTED;  // the batched launches index by fundamental
    if (!items || count < 1 || count > FDAS_MAX_BATCH || !d_thresh || !d_ws) return FDAS_ERR_INVALID_ARG;
    if (with_spec && (!d_tmpl || !aligned(d_tmpl, 16))) return FDAS_ERR_INVALID_ARG;
    if (!aligned(d_ws, 16) || !aligned(d_thresh, 4)) return FDAS_ERR_INVALID_ARG;
    if (ws_bytes < fdas_batch_workspace_bytes(p, count)) return FDAS_ERR_WORKSPACE;
    for (int b = 0; b < count; ++b) {
        const fdas_batch_item &it = items[b];
        if (it.n < 1 || it.n > FDAS_MAX_N || it.ld < it.n) return FDAS_ERR_INVALID_ARG;
        if (!it.d_plane || !it.d_cands || !it.d_counts) return FDAS_ERR_INVALID_ARG;
        if (with_spec && (!it.d_spec || !aligned(it.d_spec, 16))) return FDAS_ERR_INVALID_ARG;
        if (!aligned(it.d_plane, 16) || !aligned(it.d_cands, 4) || !aligned(it.d_counts, 4) || !aligned(it.d_peaks, 4))
            return FDAS_ERR_INVALID_ARG;
    }
    return FDAS_OK;
}

// Tables of one batch; the convolution and harmonic-sum kernels receive them as parameters.
struct Tables {
    ConvBatch conv;
    HsBatch hs;
    int total_16k;  // harmonic-sum CTAs of all spectra in launches of 16384, 12288 and 4096 columns
    int total_12k;
    int total_4k;
};

void build_tables(const fdas_params &p, const fdas_batch_item *items, int count, void *d_ws, int templates_per_item,
                  Tables *t) {
    const fdas::Geometry g = fdas::geometry(p);
    const size_t stride = hs_ws_stride(p);
    t->conv.count = t->hs.count = count;
    int item = 0, blk = 0, blk1 = 0, blk2 = 0;
    for (int b = 0; b < count; ++b) {
        const fdas_batch_item &it = items[b];
        fdas::ConvJob &cj = t->conv.job[b];
        cj.spec = static_cast<const float2 *>(it.d_spec);
        cj.plane = it.d_plane;
        cj.ld = it.ld;
        cj.n = (int)it.n;
        cj.item0 = item;
        item += fdas::convolve_items(g, it.n, templates_per_item);
        fdas::HsJob &hj = t->hs.job[b];
        hj.plane = it.d_plane;
        hj.ld = it.ld;
        hj.n = (int)it.n;
        hj.blk0 = blk;
        hj.blk1 = blk1;
        hj.blk2 = blk2;
        int bk2, bk, bk1;
        fdas::harmonic_blocks(p, it.n, &bk2, &bk, &bk1);
        blk += bk;
        blk1 += bk1;
        blk2 += bk2;
        const fdas::HsWorkspace ws = fdas::hs_workspace(static_cast<char *>(d_ws) + (size_t)b * stride, p.n_harm);
        hj.counters = cj.counters = ws.counters;
        hj.peaks = cj.peaks = ws.peaks;
        hj.raw = cj.raw = ws.raw;
        hj.cands = it.d_cands;
        hj.counts = it.d_counts;
        hj.peak_out = it.d_peaks;
    }
    t->conv.total_items = item;
    t->total_16k = blk2;
    t->total_12k = blk;
    t->total_4k = blk1;
}

cudaError_t sm_count(int *sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
}

cudaError_t prepare() {
    cudaError_t e = fdas::prepare_convolve_batch();
    if (e != cudaSuccess) return e;
    return fdas::prepare_harmonic_batch();
}

// Enqueue the batch: one persistent convolution over every segment of every spectrum, then the
// harmonic sum (reset, one launch per group of rows, finalize) over every spectrum.
cudaError_t launch_batch(const fdas_params &p, const Tables &t, const void *d_tmpl, const float *d_thresh, int sms,
                         const fdas_launch_config &cfg, cudaStream_t s, bool conv_only = false) {
    const fdas::Geometry g = fdas::geometry(p);
    const int max_ctas = fdas::convolve_ctas_per_sm(g);  // resident CTAs per SM
    const int ctas = cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < max_ctas ? cfg.ctas_per_sm : max_ctas;
    const int grid = t.conv.total_items < ctas * sms ? t.conv.total_items : ctas * sms;
    const float2 *tmpl = static_cast<const float2 *>(d_tmpl);
    // FP32 with fundamental indexing: the convolution takes HP_1 of the single-plane rows, as in
    // fdas_search; the workspaces are reset before it and the harmonic sum skips those rows.
    const bool hp1 = !conv_only && g.precision == FDAS_FP32 && p.harm_index == FDAS_INDEX_FUNDAMENTAL;
    cudaError_t e = cudaSuccess;
    if (hp1) {
        e = fdas::launch_hs_reset_batch(p, t.hs, s);
        if (e == cudaSuccess)
            e = fdas::launch_convolve_batch_hp1(g, t.conv, tmpl, grid, cfg.templates_per_item, d_thresh, p.harm_mask,
                                                p.n_harm, s);
    } else {
        e = fdas::launch_convolve_batch(g, t.conv, tmpl, grid, cfg.templates_per_item, s);
    }
    if (e != cudaSuccess || conv_only) return e;
    return fdas::launch_harmonic_batch(p, t.hs, t.total_16k, t.total_12k, t.total_4k, d_thresh, s, hp1);
}

}  // namespace

struct fdas_batch_plan {
    fdas_params p;
    const void *d_tmpl;
    const float *d_thresh;
    void *d_ws;
    int count;
    int sms;
    fdas_launch_config cfg;
    fdas_batch_item items[FDAS_MAX_BATCH];
    Tables tables;
    cudaStream_t cap;  // private stream the graph is captured on (its auxiliary streams are made
                       // before each capture begins)
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

size_t fdas_batch_workspace_bytes(const fdas_params *p, int count) {
    if (fdas_check_params(p) == FDAS_ERR_INVALID_ARG || count < 1 || count > FDAS_MAX_BATCH) return 0;
    return (size_t)count * hs_ws_stride(*p);
}

fdas_status fdas_search_batch(const fdas_params *p, const fdas_batch_item *items, int count, const void *d_tmpl,
                              const float *d_thresh, void *d_ws, size_t ws_bytes, const fdas_launch_config *cfg,
                              fdas_stream_t stream) {
    fdas_status st = check_items(p, items, count, d_tmpl, d_thresh, d_ws, ws_bytes);
    if (st != FDAS_OK) return st;
    const fdas_launch_config c = cfg ? *cfg : fdas_launch_config{0, 0};
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 3 || c.templates_per_item < 0) return FDAS_ERR_INVALID_ARG;
    Tables *t = new (std::nothrow) Tables;  // about 30 KB, kept off the stack
    if (!t) return FDAS_ERR_INVALID_ARG;
    build_tables(*p, items, count, d_ws, c.templates_per_item, t);
    int sms = 0;
    cudaError_t e = sm_count(&sms);
    if (e == cudaSuccess) e = prepare();
    if (e == cudaSuccess) e = launch_batch(*p, *t, d_tmpl, d_thresh, sms, c, stream);
    delete t;
    return FDAS_STATUS(e);
}

fdas_status fdas_harmonic_sum_batch(const fdas_params *p, const fdas_batch_item *items, int count,
                                    const float *d_thresh, void *d_ws, size_t ws_bytes, fdas_stream_t stream) {
    fdas_status st = check_items(p, items, count, nullptr, d_thresh, d_ws, ws_bytes, false);
    if (st != FDAS_OK) return st;
    Tables *t = new (std::nothrow) Tables;
    if (!t) return FDAS_ERR_INVALID_ARG;
    build_tables(*p, items, count, d_ws, 0, t);
    cudaError_t e = fdas::prepare_harmonic_batch();
    if (e == cudaSuccess)
        e = fdas::launch_harmonic_batch(*p, t->hs, t->total_16k, t->total_12k, t->total_4k, d_thresh, stream, false);
    delete t;
    return FDAS_STATUS(e);
}

fdas_status fdas_batch_plan_create(const fdas_params *p, const fdas_batch_item *items, int count, const void *d_tmpl,
                                   const float *d_thresh, void *d_ws, size_t ws_bytes, fdas_batch_plan **out) {
    if (!out) return FDAS_ERR_INVALID_ARG;
    *out = nullptr;
    fdas_status st = check_items(p, items, count, d_tmpl, d_thresh, d_ws, ws_bytes);
    if (st != FDAS_OK) return st;
    fdas_batch_plan *plan = new (std::nothrow) fdas_batch_plan;
    if (!plan) return FDAS_ERR_INVALID_ARG;
    std::memset(plan, 0, sizeof(*plan));
    plan->p = *p;
    plan->d_tmpl = d_tmpl;
    plan->d_thresh = d_thresh;
    plan->d_ws = d_ws;
    plan->count = count;
    std::memcpy(plan->items, items, sizeof(fdas_batch_item) * (size_t)count);
    if (sm_count(&plan->sms) != cudaSuccess || prepare() != cudaSuccess ||
        cudaStreamCreateWithFlags(&plan->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete plan;
        return FDAS_ERR_CUDA;
    }
    build_tables(*p, items, count, d_ws, 0, &plan->tables);
    *out = plan;
    return FDAS_OK;
}

static void drop_graph(fdas_batch_plan *plan) {
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    plan->exec = nullptr;
    plan->graph = nullptr;
}

fdas_status fdas_batch_plan_launch(fdas_batch_plan *plan, fdas_stream_t stream) {
    if (!plan) return FDAS_ERR_INVALID_ARG;
    if (!plan->exec) {
        // Capture the batch once on the plan's private stream, then replay it on the caller's
        // streams. The capture is thread-local, and the auxiliary streams it forks into belong to
        // this thread and this private stream, so searches that other threads run meanwhile neither
        // join the graph nor break the capture.
        cudaStream_t cap = plan->cap;
        cudaError_t e = FDAS_NOTE(fdas::prepare_streams(cap));
        if (e != cudaSuccess) return FDAS_STATUS(e);
        e = FDAS_NOTE(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            const cudaError_t le = FDAS_NOTE(launch_batch(plan->p, plan->tables, plan->d_tmpl, plan->d_thresh,
                                                          plan->sms, plan->cfg, cap));
            e = FDAS_NOTE(cudaStreamEndCapture(cap, &plan->graph));
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = FDAS_NOTE(cudaGraphInstantiate(&plan->exec, plan->graph, 0));
        if (e != cudaSuccess) {
            drop_graph(plan);
            return FDAS_STATUS(e);
        }
    }
    return FDAS_STATUS(cudaGraphLaunch(plan->exec, stream));
}

fdas_status fdas_batch_plan_tune(fdas_batch_plan *plan, fdas_stream_t stream, fdas_launch_config *chosen,
                                 float *ms_per_batch) {
    if (!plan) return FDAS_ERR_INVALID_ARG;
    // Candidate launch shapes of the convolution, timed on the plan's own spectra with CUDA events.
    static const int kCtas[] = {0, 2};
    static const int kTpi[] = {0, 43, 29, 17};
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&b);
    if (ce != cudaSuccess) return FDAS_STATUS(ce);
    fdas_launch_config best{0, 0};
    float best_ms = -1.0f;
    Tables *t = new (std::nothrow) Tables;
    cudaError_t e = t ? cudaSuccess : cudaErrorMemoryAllocation;
    for (int ci = 0; ci < 2 && e == cudaSuccess; ++ci) {
        for (int ti = 0; ti < 4 && e == cudaSuccess; ++ti) {
            const fdas_launch_config cfg{kCtas[ci], kTpi[ti]};
            build_tables(plan->p, plan->items, plan->count, plan->d_ws, cfg.templates_per_item, t);
            e = launch_batch(plan->p, *t, plan->d_tmpl, plan->d_thresh, plan->sms, cfg, stream, true);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(a, stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                e = launch_batch(plan->p, *t, plan->d_tmpl, plan->d_thresh, plan->sms, cfg, stream, true);
            if (e == cudaSuccess) e = cudaEventRecord(b, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                best = cfg;
            }
        }
    }
    delete t;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return FDAS_STATUS(e);
    // The timed launches have finished: a kernel that gave up on a bounded wait shows in the status.
    unsigned flags[2] = {0u, 0u};
    e = fdas::device_status_async(flags, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return FDAS_STATUS(e);
    if ((flags[0] | flags[1]) & FDAS_DEV_WAIT_TIMEOUT) return FDAS_ERR_TIMEOUT;
    plan->cfg = best;
    build_tables(plan->p, plan->items, plan->count, plan->d_ws, best.templates_per_item, &plan->tables);
    drop_graph(plan);  // the next launch captures the new shape
    if (chosen) *chosen = best;
    if (ms_per_batch) *ms_per_batch = best_ms / 3.0f;
    return FDAS_OK;
}

void fdas_batch_plan_destroy(fdas_batch_plan *plan) {
    if (!plan) return;
    drop_graph(plan);
    if (plan->cap) cudaStreamDestroy(plan->cap);
    delete plan;
}

}  // extern "C"
