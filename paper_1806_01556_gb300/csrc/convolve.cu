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

#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kF = 2048;
constexpr int kThreads = 128;
constexpr int kPadded = kF + kF / 16;  // one pad element after every 16

__device__ __forceinline__ int pad(int e) { return e + (e >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
template <bool INV>
__device__ __forceinline__ float2 twiddle(float2 v, float2 w) {  // w = exp(-2 pi i x); INV uses conj(w)
    return INV ? cmul_conj(v, w) : cmul(v, w);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Status bits set on the device (read with fdas_device_status): a bounded wait gave up.
__device__ unsigned int g_device_status;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// One-dimensional TMA bulk copy global -> shared, completing on an mbarrier (transaction count in bytes).
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Wait for phase `parity` of the mbarrier, for at most about 2^31 SM cycles (about one second). On
// time-out the status word records it; the caller carries on, so the launch always ends.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const long long start = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - start > (1ll << 31)) {
            atomicOr(&g_device_status, 1u);
            return false;
        }
    }
}

// In-place 4-point DFT of (a, b, c, d) with sign exp(-+2 pi i / 4); outputs in natural order.
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
    a = cadd(s0, s2);
    c = csub(s0, s2);
    if (!INV) {
        b = make_float2(s1.x + s3.y, s1.y - s3.x);  // s1 - i s3
        d = make_float2(s1.x - s3.y, s1.y + s3.x);  // s1 + i s3
    } else {
        b = make_float2(s1.x - s3.y, s1.y + s3.x);
        d = make_float2(s1.x + s3.y, s1.y - s3.x);
    }
}

// Multiply by exp(-+2 pi i m / 16) for the constant m (0 < m < 16).
template <bool INV, int M>
__device__ __forceinline__ float2 w16(float2 v) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r = 0.70710678118654752f;
    constexpr int m = M & 15;
    constexpr float wr = m == 0 ? 1.f : m == 1 ? c1 : m == 2 ? r : m == 3 ? s1 : m == 4 ? 0.f : m == 5 ? -s1
                       : m == 6 ? -r : m == 7 ? -c1 : m == 8 ? -1.f : m == 9 ? -c1 : m == 10 ? -r : m == 11 ? -s1
                       : m == 12 ? 0.f : m == 13 ? s1 : m == 14 ? r : c1;
    constexpr float wi0 = m == 0 ? 0.f : m == 1 ? -s1 : m == 2 ? -r : m == 3 ? -c1 : m == 4 ? -1.f : m == 5 ? -c1
                        : m == 6 ? -r : m == 7 ? -s1 : m == 8 ? 0.f : m == 9 ? s1 : m == 10 ? r : m == 11 ? c1
                        : m == 12 ? 1.f : m == 13 ? c1 : m == 14 ? r : s1;
    constexpr float wi = INV ? -wi0 : wi0;
    if (m == 4) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    return make_float2(fmaf(v.x, wr, -v.y * wi), fmaf(v.x, wi, v.y * wr));
}

// 16-point DFT in registers, natural order in and out: radix 4 x 4 with internal twiddles.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // v[4 k1 + n2] *= W16^(n2 k1)
    v[5] = w16<INV, 1>(v[5]);
    v[6] = w16<INV, 2>(v[6]);
    v[7] = w16<INV, 3>(v[7]);
    v[9] = w16<INV, 2>(v[9]);
    v[10] = w16<INV, 4>(v[10]);
    v[11] = w16<INV, 6>(v[11]);
    v[13] = w16<INV, 3>(v[13]);
    v[14] = w16<INV, 6>(v[14]);
    v[15] = w16<INV, 9>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 register block.
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// 8-point DFT in registers, natural order in and out: radix 4 x 2.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    v[3] = w16<INV, 2>(v[3]);  // W8^1
    v[5] = w16<INV, 4>(v[5]);  // W8^2
    v[7] = w16<INV, 6>(v[7]);  // W8^3
    float2 t[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        t[k1] = cadd(v[2 * k1], v[2 * k1 + 1]);
        t[k1 + 4] = csub(v[2 * k1], v[2 * k1 + 1]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = t[i];
}

// Passes 1 and 2 of the Stockham FFT: registers (A[tid + 128 r]) -> pass 1 -> buf0 -> pass 2 -> buf1.
template <bool INV, class AfterFirstBarrier>
__device__ __forceinline__ void fft_passes_12(float2 (&v)[16], float2 *buf0, float2 *buf1, const float2 (&tw2)[16],
                                              int tid, AfterFirstBarrier after_first_barrier) {
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf0[pad(16 * tid + r)] = v[r];
    __syncthreads();
    after_first_barrier();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf0[pad(tid + 128 * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twiddle<INV>(v[r], tw2[r]);
    dft16<INV>(v);
    const int base = (tid >> 4) * 256 + (tid & 15);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf1[pad(base + 16 * r)] = v[r];
    __syncthreads();
}

// Pass 3 for butterfly b = tid + 128 hh: reads buf1[b + 256 r], returns index b + 256 r in u[r].
template <bool INV>
__device__ __forceinline__ void fft_pass_3(float2 (&u)[8], const float2 *buf1, const float2 (&tw3)[8], int b) {
#pragma unroll
    for (int r = 0; r < 8; ++r) u[r] = buf1[pad(b + 256 * r)];
#pragma unroll
    for (int r = 1; r < 8; ++r) u[r] = twiddle<INV>(u[r], tw3[r]);
    dft8<INV>(u);
}

// Two exchange buffers, two template buffers, and two mbarriers for the template copies.
constexpr size_t kSmemBytes = (2 * kPadded + 2 * kF) * sizeof(float2) + 2 * sizeof(unsigned long long);

// One work item: segment s of one spectrum with templates [t0, t1).
struct Item {
    const float2 *spec;
    float *plane;
    size_t ld;
    int n;
    int s;
    int t0;
    int t1;
};

// Work items of a single spectrum: item = s * n_tchunk + chunk.
struct SingleJobs {
    const float2 *spec;
    float *plane;
    size_t ld;
    int n;
    int n_seg;
    int t_chunk;
    int n_tchunk;
    int n_temp;
    __device__ int total() const { return n_seg * n_tchunk; }
    __device__ Item get(int item) const {
        const int s = item / n_tchunk;
        const int t0 = (item - s * n_tchunk) * t_chunk;
        return Item{spec, plane, ld, n, s, t0, min(t0 + t_chunk, n_temp)};
    }
};

// Work items of a batch (a kernel parameter): the items of spectrum b are
// [job[b].item0, job[b].item0 + n_seg_b * n_tchunk).
struct BatchJobs {
    ConvBatch batch;
    int t_chunk;
    int n_tchunk;
    int n_temp;
    __device__ int total() const { return batch.total_items; }
    __device__ Item get(int item) const {
        int lo = 0, hi = batch.count - 1;  // last job with item0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (batch.job[mid].item0 <= item) lo = mid; else hi = mid - 1;
        }
        const ConvJob &J = batch.job[lo];
        const int local = item - J.item0;
        const int s = local / n_tchunk;
        const int t0 = (local - s * n_tchunk) * t_chunk;
        return Item{J.spec, J.plane, (size_t)J.ld, J.n, s, t0, min(t0 + t_chunk, n_temp)};
    }
};

template <class Jobs>
__global__ void __launch_bounds__(kThreads, 3)
    fdas_ols_fp32(Jobs jobs, const float2 *__restrict__ tmpl, int n_temp, int h, int keep) {
    extern __shared__ __align__(128) float2 smem[];
    float2 *buf0 = smem;
    float2 *buf1 = smem + kPadded;
    float2 *tbuf = smem + 2 * kPadded;  // [2][kF], template values of the current and next template
    unsigned long long *tbar = reinterpret_cast<unsigned long long *>(smem + 2 * kPadded + 2 * kF);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&tbar[0]);
        mbar_init(&tbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
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
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                float2 u[8];
                fft_pass_3<true>(u, buf1, hh ? tw3b : tw3a, tid + 128 * hh);
                const unsigned m8 = smask >> (8 * hh);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float pw = fmaf(u[r].x, u[r].x, u[r].y * u[r].y);
                    if ((m8 >> r) & 1u) dst[128 * hh + 256 * r] = pw;
                }
            }
        }
    }
}

}  // namespace

static void chunking(const Geometry &g, int templates_per_item, int *t_chunk, int *n_tchunk) {
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
    e = cudaFuncSetAttribute(fdas_ols_fp32<SingleJobs>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    fdas_ols_fp32<<<grid, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    return cudaGetLastError();
}

cudaError_t device_status(unsigned *flags, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_device_status, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
    }
    return e;
}

cudaError_t prepare_convolve_batch() {
    return cudaFuncSetAttribute(fdas_ols_fp32<BatchJobs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes);
}

int convolve_items(const Geometry &g, size_t n, int templates_per_item) {
    int t_chunk, n_tchunk;
    chunking(g, templates_per_item, &t_chunk, &n_tchunk);
    return (int)((n + g.keep - 1) / g.keep) * n_tchunk;
}

cudaError_t launch_convolve_batch(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                  int templates_per_item, cudaStream_t s) {
    BatchJobs jobs;
    jobs.batch = batch;
    jobs.n_temp = g.n_temp;
    chunking(g, templates_per_item, &jobs.t_chunk, &jobs.n_tchunk);
    fdas_ols_fp32<<<grid, kThreads, kSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    return cudaGetLastError();
}

}  // namespace fdas
