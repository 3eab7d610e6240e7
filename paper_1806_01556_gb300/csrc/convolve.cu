// FT convolution by overlap-save with fused power and discard (Sec. 2.1: OLS-FDFIR, AOLS-2048-P).
//
// For template t the plane row is P[t][j] = |sum_q X[j+q] conj(a_t[q])|^2. Overlap-save computes it
// per segment s of F = 2048 input points, w_s[n] = X[s*L - h + n] (zero outside [0, N)), as
//     u = IDFT(DFT(w_s) * T_t),   P[t][s*L + m] = |u[h + m]|^2,  m = 0..L-1,  L = F - n_tap + 1,
// where T_t = conj(DFT(wrapped taps)) comes from fdas_make_templates. As in the paper's AOLS
// kernel, the segment is transformed once and reused for every template. The F - L wrapped
// outputs are never stored, which fuses the "discard" of the FOP preparation (Sec. 3.2).
//
// GB300 mapping: one CTA of 128 threads owns one segment (and a range of templates). Each thread
// holds 16 complex points in registers. A 2048-point FFT is three Stockham passes, radix
// 16 x 16 x 8, with two shared-memory exchanges in a padded layout that is conflict-free for
// 64-bit accesses. After the forward FFT, thread tid holds frequency m = tid + 128 q in register
// q. This is exactly the input layout of the inverse FFT's first pass, so the product with the
// template needs no exchange. Each template (16 KB, from the 1.4 MB bank that stays in L2) is
// brought into a shared-memory double buffer by one TMA bulk copy, so the next template is in flight
// while the current one is transformed. After the inverse FFT, thread tid holds time index
// n = tid + 128 q, so the power stores of a warp are 32 consecutive columns, issued as predicated
// stores from one base pointer per template.
#include <utility>

#include "hs_keys.cuh"
#include "ols_common.cuh"

namespace fdas {
namespace {

// Two exchange buffers, two template buffers, the HP_1 thresholds of the first kTaShared rows, and two
// mbarriers for the template copies.
constexpr int kTaShared = 256;
constexpr size_t kSmemBytes =
    (2 * kPadded + 2 * kF) * sizeof(float2) + kTaShared * sizeof(float) + 2 * sizeof(unsigned long long);

// HP_1 detection fused into the convolution (fdas_search): HP_1(i, j) is the plane value itself
// (Algorithm 1 with k = 1), so for the rows that take part in no other plane (|i| > c/2) the
// candidates above TA(1, i) and the HP_1 peak are taken while the values are in registers, and the
// harmonic sum skips its single-plane launch. The row-group launches still take HP_1 of their rows.
struct Hp1 {
    const float *ta;  // TA(1, row) for every row; nullptr: no HP_1 candidates (bit 0 of harm_mask clear)
    unsigned long long *raw;
    unsigned long long *counters;
    unsigned long long *peaks;
    int c;            // zero-drift row
    int lo1;          // rows with |row - c| >= lo1 are the single-plane rows this kernel takes
};

// Rare path, kept out of line so that the hot loop stays small: emit the kept outputs of one row
// segment above ta, re-read from the plane (the calling warp must be converged: emit ballots).
__device__ __noinline__ void hp1_emit_row(const float *rowp, float ta, int t, int col, unsigned smask, Hp1 hp1) {
#pragma unroll 1
    for (int q = 0; q < 16; ++q) {
        const int o = 128 * (q >> 3) + 256 * (q & 7);
        const bool kept = (smask >> q) & 1u;
        const float pv = kept ? rowp[o] : -1.0f;
        emit(kept && pv > ta, pv, t, (unsigned)(col + o), 1, threadIdx.x & 31, hp1.counters, hp1.raw);
    }
}

// Column (as row << 24 | column) of the first kept output equal to best in one row segment.
__device__ __noinline__ unsigned hp1_best_loc(const float *rowp, float best, int t, int col, unsigned smask) {
    unsigned loc = 0xFFFFFFFFu;
#pragma unroll 1
    for (int q = 0; q < 16; ++q) {
        const int o = 128 * (q >> 3) + 256 * (q & 7);
        if (((smask >> q) & 1u) && rowp[o] == best) {
            const unsigned l = ((unsigned)t << 24) | (unsigned)(col + o);
            loc = l < loc ? l : loc;
        }
    }
    return loc;
}

template <bool HP1, class Jobs>
__global__ void __launch_bounds__(kThreads, 3)
    fdas_ols_fp32(Jobs jobs, const float2 *__restrict__ tmpl, int n_temp, int h, int keep, Hp1 hp1) {
    extern __shared__ __align__(128) float2 smem[];
    float2 *buf0 = smem;
    float2 *buf1 = smem + kPadded;
    float2 *tbuf = smem + 2 * kPadded;  // [2][kF], template values of the current and next template
    float *ta_s = reinterpret_cast<float *>(smem + 2 * kPadded + 2 * kF);  // HP1: TA(1, t) for t < kTaShared
    unsigned long long *tbar = reinterpret_cast<unsigned long long *>(ta_s + kTaShared);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&tbar[0]);
        mbar_init(&tbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (HP1)
        for (int t = tid; t < n_temp && t < kTaShared; t += kThreads)
            ta_s[t] = hp1.ta ? __ldg(&hp1.ta[t]) : __int_as_float(0x7f800000);
    __syncthreads();
    unsigned phase = 0u;  // bit b: parity of the next completion of template buffer b
    const float2 *wtab = tmpl + (size_t)n_temp * kF;  // exp(-2 pi i k / F)

    // Stockham twiddles of this thread, fixed for the whole kernel.
    float2 tw2[16], tw3a[8], tw3b[8];
    {
        const int k = tid & 15;
#pragma unroll
        for (int r = 0; r < 16; ++r) tw2[r] = __ldg(&wtab[8 * ((k * r) & 255)]);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            tw3a[r] = __ldg(&wtab[tid * r]);
            tw3b[r] = __ldg(&wtab[(tid + 128) * r]);
        }
    }
    // Output register (hh, r) holds segment time index m = tid + 128 hh + 256 r; it is a valid
    // (non-wrapped) overlap-save output iff h <= m < h + keep. Bit 8 hh + r of keep_mask.
    unsigned keep_mask = 0u;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int m = tid + 128 * hh + 256 * r;
            if (m >= h && m < h + keep) keep_mask |= 1u << (8 * hh + r);
        }
    const float scale = 1.0f / kF;
    const int n_items = jobs.total();

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Item it = jobs.get(item);
        const int n = it.n, s = it.s, t0 = it.t0, t1 = it.t1;
        Hp1 h1 = hp1;  // HP1: a batch item's own workspace replaces the kernel's
        if (HP1 && it.counters != nullptr) {
            h1.raw = it.raw;
            h1.counters = it.counters;
            h1.peaks = it.peaks;
        }
        const float2 *__restrict__ spec = it.spec;
        const int origin = s * keep - h;  // input index of segment point 0
        const int col0 = s * keep - h;    // column of segment time index 0
        // Outputs this thread stores for this segment: valid (keep_mask) and inside the spectrum.
        unsigned smask = keep_mask;
        if ((s + 1) * keep > n) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (col0 + tid + 128 * hh + 256 * r >= n) smask &= ~(1u << (8 * hh + r));
        }
        // Template t0 lands in buffer 0 while the forward FFT runs. Every earlier read of buffer 0
        // happened before a barrier that thread 0 has passed.
        if (tid == 0) tma_load(tbuf, tmpl + (size_t)t0 * kF, kF * sizeof(float2), &tbar[0]);

        // Forward FFT of the segment: W[q] = DFT(w_s)[tid + 128 q] / F.
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int idx = origin + tid + 128 * r;
            v[r] = (idx >= 0 && idx < n) ? __ldg(&spec[idx]) : make_float2(0.f, 0.f);
        }
        fft_passes_12<false>(v, buf0, buf1, tw2, tid, [] {});
        float best = -1.0f;  // HP1: this thread's largest single-plane-row output of the item, its template
        int best_t = -1;
        float2 W[16];
        {
            float2 u[8];
            fft_pass_3<false>(u, buf1, tw3a, tid);
#pragma unroll
            for (int r = 0; r < 8; ++r) W[2 * r] = make_float2(u[r].x * scale, u[r].y * scale);
            fft_pass_3<false>(u, buf1, tw3b, tid + 128);
#pragma unroll
            for (int r = 0; r < 8; ++r) W[2 * r + 1] = make_float2(u[r].x * scale, u[r].y * scale);
        }

        for (int t = t0; t < t1; ++t) {
            const int slot = (t - t0) & 1;
            mbar_wait(&tbar[slot], (phase >> slot) & 1u);  // template t is in buffer slot
            phase ^= 1u << slot;
            const float2 *T = tbuf + slot * kF + tid;
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = cmul(W[q], T[128 * q]);
            // After the first barrier of this FFT every thread has read buffer slot^1 for the last
            // time (in the previous template), so thread 0 refills it with template t + 1.
            fft_passes_12<true>(v, buf0, buf1, tw2, tid, [&] {
                if (tid == 0 && t + 1 < t1)
                    tma_load(tbuf + (slot ^ 1) * kF, tmpl + (size_t)(t + 1) * kF, kF * sizeof(float2),
                             &tbar[slot ^ 1]);
            });
            // Column col0 + b + 256 r of row t, for b = tid + 128 hh: one base pointer per half, then
            // constant offsets; a plain predicated store per output.
            float *const dst = it.plane + (size_t)t * it.ld + col0 + tid;
            const bool k1row = HP1 && abs(t - hp1.c) >= hp1.lo1;  // CTA-uniform
            float mx = -1.0f;  // HP1: largest kept output of this template
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float2 u[8];
                fft_pass_3<true>(u, buf1, hh ? tw3b : tw3a, tid + 128 * hh);
                const unsigned m8 = smask >> (8 * hh);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float pw = fmaf(u[r].x, u[r].x, u[r].y * u[r].y);
                    if ((m8 >> r) & 1u) {
                        dst[128 * hh + 256 * r] = pw;
                        if (k1row) mx = fmaxf(mx, pw);
                    }
                }
            }
            if (k1row) {
                const float ta = t < kTaShared ? ta_s[t] : hp1.ta ? __ldg(&hp1.ta[t]) : __int_as_float(0x7f800000);
                if (__any_sync(0xFFFFFFFFu, mx > ta)) hp1_emit_row(dst, ta, t, col0 + tid, smask, h1);  // rare
                if (mx > best) {  // strict: the first template wins ties, as in the canonical order
                    best = mx;
                    best_t = t;
                }
            }
        }
        if (HP1) {
            // The HP_1 peak of the item's single-plane rows: the column of this thread's best
            // (re-read from its row), then the warp's largest key, one atomicMax per warp. Peak
            // keys only grow, so a warp whose best power is below the peak found so far skips this.
            const unsigned wmax = __reduce_max_sync(0xFFFFFFFFu, best >= 0.0f ? __float_as_uint(best) : 0u);
            const unsigned cur = (unsigned)(*(volatile unsigned long long *)&h1.peaks[0] >> 32);
            if (wmax >= cur) {  // warp-uniform
                const unsigned loc = best_t >= 0 ? hp1_best_loc(it.plane + (size_t)best_t * it.ld + col0 + tid, best,
                                                                best_t, col0 + tid, smask)
                                                 : 0xFFFFFFFFu;
                const unsigned long long key = warp_peak_key_loc(best, loc);
                if ((tid & 31) == 0 && key != 0ull) atomicMax(&h1.peaks[0], key);
            }
        }
    }
}

}  // namespace

static void chunking(const Geometry &g, int templates_per_item, int *t_chunk, int *n_tchunk) {
    if (templates_per_item <= 0 && g.precision != FDAS_FP32) templates_per_item = kTcDefaultTemplatesPerItem;
    *t_chunk = (templates_per_item > 0 && templates_per_item < g.n_temp) ? templates_per_item : g.n_temp;
    *n_tchunk = (g.n_temp + *t_chunk - 1) / *t_chunk;
}

static cudaError_t persistent_grid(int n_items, int ctas_per_sm, int *grid) {
    *grid = n_items;
    if (ctas_per_sm <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = n_items < ctas_per_sm * sms ? n_items : ctas_per_sm * sms;
    return cudaSuccess;
}

cudaError_t launch_convolve_fp32(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                                 size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s) {
    // A work item is one segment with t_chunk templates; the segment's forward FFT is done once per item.
    SingleJobs jobs;
    jobs.spec = spec;
    jobs.plane = plane;
    jobs.ld = ld;
    jobs.n = (int)n;
    jobs.n_seg = (int)((n + g.keep - 1) / g.keep);
    jobs.n_temp = g.n_temp;
    chunking(g, templates_per_item, &jobs.t_chunk, &jobs.n_tchunk);
    int grid = 0;
    cudaError_t e = persistent_grid(jobs.n_seg * jobs.n_tchunk, ctas_per_sm, &grid);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fdas_ols_fp32<false, SingleJobs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    fdas_ols_fp32<false><<<grid, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep, Hp1{});
    return cudaGetLastError();
}

namespace {
__device__ unsigned g_wait_check_ok;

// One thread waits on an mbarrier that nothing will ever complete, through the same bounded wait
// the convolution kernels use. The wait gives up after about one second, records it in the
// status word and returns; g_wait_check_ok receives 0 then (1 would mean the phase completed).
__global__ void fdas_wait_timeout_check() {
    __shared__ unsigned long long bar;
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    g_wait_check_ok = mbar_wait(&bar, 0u) ? 1u : 0u;
}
}  // namespace

cudaError_t check_wait_timeout(unsigned *flags) {
    unsigned h_ok = 1u;
    cudaError_t e = device_status(flags, true);  // start from a clear word
    if (e == cudaSuccess) {
        fdas_wait_timeout_check<<<1, 1>>>();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&h_ok, g_wait_check_ok, sizeof(unsigned));
    if (e == cudaSuccess) e = device_status(flags, true);
    if (e == cudaSuccess && h_ok != 0u) *flags = 0u;  // the phase cannot complete: report no timeout seen
    return e;
}

cudaError_t launch_convolve_hp1(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                                size_t ld, const float *thresh, unsigned harm_mask, int n_harm, const HsWorkspace &ws,
                                cudaStream_t s) {
    SingleJobs jobs;
    jobs.spec = spec;
    jobs.plane = plane;
    jobs.ld = ld;
    jobs.n = (int)n;
    jobs.n_seg = (int)((n + g.keep - 1) / g.keep);
    jobs.n_temp = g.n_temp;
    chunking(g, 0, &jobs.t_chunk, &jobs.n_tchunk);
    cudaError_t e = cudaFuncSetAttribute(fdas_ols_fp32<true, SingleJobs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // The single-plane rows: |i| > c/2 with two or more planes, every row with one.
    const Hp1 hp1{(harm_mask & 1u) ? thresh : nullptr, ws.raw, ws.counters, ws.peaks, g.c, n_harm >= 2 ? g.c / 2 + 1 : 0};
    fdas_ols_fp32<true><<<jobs.n_seg * jobs.n_tchunk, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep,
                                                                                hp1);
    return cudaGetLastError();
}

cudaError_t launch_convolve(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                            size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s) {
    if (g.precision == FDAS_FP32)
        return launch_convolve_fp32(g, spec, n, tmpl, plane, ld, ctas_per_sm, templates_per_item, s);
    return launch_convolve_tc(g, spec, n, tmpl, plane, ld, ctas_per_sm, templates_per_item, s);
}

cudaError_t device_status(unsigned *flags, bool clear) {
    unsigned tc_flags = 0u;
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_device_status, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
    }
    if (e == cudaSuccess) e = device_status_tc(&tc_flags, clear);
    if (e == cudaSuccess) *flags |= tc_flags;
    return e;
}

cudaError_t device_status_async(unsigned *h_flags2, cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(&h_flags2[0], g_device_status, sizeof(unsigned), 0,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = device_status_tc_async(&h_flags2[1], s);
    return e;
}

cudaError_t set_device_status(unsigned flags) {
    cudaError_t e = cudaMemcpyToSymbol(g_device_status, &flags, sizeof(unsigned));
    unsigned tc = 0u;
    if (e == cudaSuccess) e = device_status_tc(&tc, true);  // one word holds the new state
    return e;
}

cudaError_t prepare_convolve_batch() {
    cudaError_t e = cudaFuncSetAttribute(fdas_ols_fp32<false, BatchJobs>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fdas_ols_fp32<true, BatchJobs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
    if (e == cudaSuccess) e = prepare_convolve_batch_tc();
    return e;
}

int convolve_items(const Geometry &g, size_t n, int templates_per_item) {
    int t_chunk, n_tchunk;
    chunking(g, templates_per_item, &t_chunk, &n_tchunk);
    return (int)((n + g.keep - 1) / g.keep) * n_tchunk;
}

cudaError_t launch_convolve_batch_hp1(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                      int templates_per_item, const float *thresh, unsigned harm_mask, int n_harm,
                                      cudaStream_t s) {
    BatchJobs jobs;
    jobs.batch = batch;
    jobs.n_temp = g.n_temp;
    chunking(g, templates_per_item, &jobs.t_chunk, &jobs.n_tchunk);
    // The workspace pointers come from each item; the single-plane rows as in launch_convolve_hp1.
    const Hp1 hp1{(harm_mask & 1u) ? thresh : nullptr, nullptr, nullptr, nullptr, g.c,
                  n_harm >= 2 ? g.c / 2 + 1 : 0};
    fdas_ols_fp32<true><<<grid, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep, hp1);
    return cudaGetLastError();
}

cudaError_t launch_convolve_batch(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                  int templates_per_item, cudaStream_t s) {
    if (g.precision != FDAS_FP32) return launch_convolve_batch_tc(g, batch, tmpl, grid, templates_per_item, s);
    BatchJobs jobs;
    jobs.batch = batch;
    jobs.n_temp = g.n_temp;
    chunking(g, templates_per_item, &jobs.t_chunk, &jobs.n_tchunk);
    fdas_ols_fp32<false><<<grid, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep, Hp1{});
    return cudaGetLastError();
}

}  // namespace fdas
