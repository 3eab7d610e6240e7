// Pieces shared by the overlap-save convolution kernels (FP32 and tensor-core forms): the
// 2048-point FFT in registers (radix 16 x 16 x 8 Stockham passes through a padded shared-memory
// buffer; the butterflies' complex sums as packed FP32x2 instructions, two lanes per issue slot),
// the TMA bulk copy with its bounded mbarrier wait, and the work-item decomposition (segment s of a
// spectrum with a range of templates). Everything here has internal linkage, so
// each translation unit that includes it has its own copy, including its own status word.
#pragma once
#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kF = 2048;
constexpr int kThreads = 128;
constexpr int kPadded = kF + kF / 16;  // one pad element after every 16

// Padded position of element e of an exchange buffer (one pad element after every 16), conflict-free
// for 64-bit accesses. The exchanges below address it as one base pointer per thread plus constant
// offsets (the comments give the pad() expression each one implements).
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
// The same sums as single packed FP32x2 instructions (two lanes per issue slot).
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) {
    unsigned long long x, y, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}

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
// time-out the status word records it; the caller carries on, so the launch always ends. Each
// try_wait may suspend the thread until the phase completes, for at most 1 ms (the hint, in ns),
// so a waiting warp takes few issue slots from the others.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const long long start = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
            : "memory");
        if (ok) return true;
        if (clock64() - start > (1ll << 31)) {
            atomicOr(&g_device_status, 1u);
            return false;
        }
    }
}

// In-place 4-point DFT of (a, b, c, d) with sign exp(-+2 pi i / 4); outputs in natural order.
// PACKED: the complex sums as packed FP32x2 instructions (the +-i s3 terms stay scalar).
template <bool INV, bool PACKED = true>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 s0 = PACKED ? cadd2(a, c) : cadd(a, c), s1 = PACKED ? csub2(a, c) : csub(a, c),
                 s2 = PACKED ? cadd2(b, d) : cadd(b, d), s3 = PACKED ? csub2(b, d) : csub(b, d);
    a = PACKED ? cadd2(s0, s2) : cadd(s0, s2);
    c = PACKED ? csub2(s0, s2) : csub(s0, s2);
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

// 8-point DFT in registers, natural order in and out: radix 4 x 2.
template <bool INV, bool PACKED = true>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    dft4<INV, PACKED>(v[0], v[2], v[4], v[6]);
    dft4<INV, PACKED>(v[1], v[3], v[5], v[7]);
    v[3] = w16<INV, 2>(v[3]);  // W8^1
    v[5] = w16<INV, 4>(v[5]);  // W8^2
    v[7] = w16<INV, 6>(v[7]);  // W8^3
    float2 t[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        t[k1] = PACKED ? cadd2(v[2 * k1], v[2 * k1 + 1]) : cadd(v[2 * k1], v[2 * k1 + 1]);
        t[k1 + 4] = PACKED ? csub2(v[2 * k1], v[2 * k1 + 1]) : csub(v[2 * k1], v[2 * k1 + 1]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = t[i];
}

// ---- Constant twiddles folded into the butterflies (FMA form) ----
//
// A twiddle w with Re w != 0 is w = s (1 + i t), s = Re w, t = Im w / s. The factor (1 + i t) costs
// two FMAs, (x.r - t x.i, x.i + t x.r), and the real s rides on the FMA that adds the product into a
// butterfly sum: a radix-4 butterfly whose first input carries no twiddle takes 22 FP32 instructions
// instead of 28 (three complex products and 16 additions). The inverse transform uses
// conj(w) = s (1 - i t). Used for the constant twiddles W16^m of the 16-point DFTs, whose s and t are
// compile-time constants.

// x (1 + i t) (forward) or x (1 - i t) (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_1it(float2 x, float t) {
    const float u = INV ? -t : t;
    return make_float2(fmaf(-u, x.y, x.x), fmaf(u, x.x, x.y));
}
// x W4: -i x (forward) or +i x (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 x) {
    return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
}

// 4-point DFT of (a, sb b, sc c, sb mu d) in place, natural order: 16 FMAs.
template <bool INV>
__device__ __forceinline__ void r4_scaled(float2 &a, float2 &b, float2 &c, float2 &d, float sc, float mu, float sb) {
    const float2 s0 = make_float2(fmaf(sc, c.x, a.x), fmaf(sc, c.y, a.y));
    const float2 s1 = make_float2(fmaf(-sc, c.x, a.x), fmaf(-sc, c.y, a.y));
    const float2 q = make_float2(fmaf(mu, d.x, b.x), fmaf(mu, d.y, b.y));
    const float2 p = mul_w4<INV>(make_float2(fmaf(-mu, d.x, b.x), fmaf(-mu, d.y, b.y)));
    a = make_float2(fmaf(sb, q.x, s0.x), fmaf(sb, q.y, s0.y));
    c = make_float2(fmaf(-sb, q.x, s0.x), fmaf(-sb, q.y, s0.y));
    b = make_float2(fmaf(sb, p.x, s1.x), fmaf(sb, p.y, s1.y));
    d = make_float2(fmaf(-sb, p.x, s1.x), fmaf(-sb, p.y, s1.y));
}

// cos(2 pi m / 16) and tan(2 pi m / 16) for the constant m (cos != 0).
template <int M>
__device__ __forceinline__ constexpr float cos16() {
    constexpr int m = M & 15;
    static_assert(m != 4 && m != 12, "W16^4 and W16^12 are rotations");
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r = 0.70710678118654752f;
    return m == 0 ? 1.f : m == 1 ? c1 : m == 2 ? r : m == 3 ? s1 : m == 5 ? -s1 : m == 6 ? -r : m == 7 ? -c1
         : m == 8 ? -1.f : m == 9 ? -c1 : m == 10 ? -r : m == 11 ? -s1 : m == 13 ? s1 : m == 14 ? r : c1;
}
template <int M>
__device__ __forceinline__ constexpr float tan16() {
    constexpr int m = M & 15;
    static_assert(m != 4 && m != 12, "W16^4 and W16^12 are rotations");
    constexpr float t1 = 0.41421356237309505f, t3 = 2.4142135623730950f;
    return (m & 7) == 0 ? 0.f : (m & 7) == 1 ? t1 : (m & 7) == 2 ? 1.f : (m & 7) == 3 ? t3 : (m & 7) == 5 ? -t3
         : (m & 7) == 6 ? -1.f : -t1;
}

// 16-point DFT in registers, natural order in and out: the first radix-4 layer and the untwiddled
// row of the second with packed sums, the three rows with constant twiddles W16^m in FMA form (about
// the same issue slots as complex products followed by packed sums, 6 fewer FP32 pipe operations
// per twiddled row).
template <bool INV>
__device__ __forceinline__ void dft16_hyb(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    dft4<INV>(v[0], v[1], v[2], v[3]);
    constexpr float c1 = cos16<1>(), c2 = cos16<2>(), c3 = cos16<3>(), c6 = cos16<6>(), c9 = cos16<9>();
    {
        v[5] = mul_1it<INV>(v[5], -tan16<1>());
        v[6] = mul_1it<INV>(v[6], -tan16<2>());
        v[7] = mul_1it<INV>(v[7], -tan16<3>());
        r4_scaled<INV>(v[4], v[5], v[6], v[7], c2, c3 / c1, c1);
    }
    {
        v[9] = mul_1it<INV>(v[9], -tan16<2>());
        v[10] = mul_w4<INV>(v[10]);
        v[11] = mul_1it<INV>(v[11], -tan16<6>());
        r4_scaled<INV>(v[8], v[9], v[10], v[11], 1.f, c6 / c2, c2);
    }
    {
        v[13] = mul_1it<INV>(v[13], -tan16<3>());
        v[14] = mul_1it<INV>(v[14], -tan16<6>());
        v[15] = mul_1it<INV>(v[15], -tan16<9>());
        r4_scaled<INV>(v[12], v[13], v[14], v[15], c6, c9 / c3, c3);
    }
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// Passes 1 and 2 of the Stockham FFT: registers (A[tid + 128 r]) -> pass 1 -> buf0 -> pass 2 -> buf1.
// `sync` synchronises the 128 threads that run the FFT (the whole CTA by default).
template <bool INV, class AfterFirstBarrier, class Sync>
__device__ __forceinline__ void fft_passes_12(float2 (&v)[16], float2 *buf0, float2 *buf1, const float2 (&tw2)[16],
                                              int tid, AfterFirstBarrier after_first_barrier, Sync sync) {
    dft16_hyb<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) (buf0 + 17 * tid)[r] = v[r];  // pad(16 tid + r)
    sync();
    after_first_barrier();
    const float2 *src = buf0 + tid + (tid >> 4);  // pad(tid + 128 r) = tid + tid / 16 + 136 r
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = src[136 * r];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = twiddle<INV>(v[r], tw2[r]);
    dft16_hyb<INV>(v);
    float2 *dst = buf1 + (tid >> 4) * 272 + (tid & 15);  // pad(256 (tid / 16) + tid % 16 + 16 r)
#pragma unroll
    for (int r = 0; r < 16; ++r) dst[17 * r] = v[r];
    sync();
}
template <bool INV, class AfterFirstBarrier>
__device__ __forceinline__ void fft_passes_12(float2 (&v)[16], float2 *buf0, float2 *buf1, const float2 (&tw2)[16],
                                              int tid, AfterFirstBarrier after_first_barrier) {
    fft_passes_12<INV>(v, buf0, buf1, tw2, tid, after_first_barrier, [] { __syncthreads(); });
}

// Pass 3 for butterfly b = tid + 128 hh: reads buf1[b + 256 r], returns index b + 256 r in u[r].
template <bool INV>
__device__ __forceinline__ void fft_pass_3(float2 (&u)[8], const float2 *buf1, const float2 (&tw3)[8], int b) {
#pragma unroll
    for (int r = 0; r < 8; ++r) u[r] = (buf1 + b + (b >> 4))[272 * r];  // pad(b + 256 r)
#pragma unroll
    for (int r = 1; r < 8; ++r) u[r] = twiddle<INV>(u[r], tw3[r]);
    dft8<INV>(u);
}

// One work item: segment s of one spectrum with templates [t0, t1).
struct Item {
    const float2 *spec;
    float *plane;
    size_t ld;
    int n;
    int s;
    int t0;
    int t1;
    // The spectrum's harmonic-sum workspace in a batch (nullptr for a single spectrum, whose
    // workspace the kernel gets as a parameter).
    unsigned long long *counters;
    unsigned long long *peaks;
    unsigned long long *raw;
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
        return Item{spec, plane, ld, n, s, t0, min(t0 + t_chunk, n_temp), nullptr, nullptr, nullptr};
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
        return Item{J.spec, J.plane, (size_t)J.ld, J.n, s, t0, min(t0 + t_chunk, n_temp), J.counters, J.peaks, J.raw};
    }
};

}  // namespace
}  // namespace fdas
