// FT convolution on the tensor cores: precisions FDAS_BF16X3 and FDAS_FP16S.
//
// The overlap-save steps are those of the FP32 kernel (Sec. 2.1): segment s of F = 2048 input
// points is transformed once (FP32 FFT in registers), multiplied by each template T_t, transformed
// back, and |u|^2 of the L = F - n_tap + 1 valid outputs is stored. Here the inverse transform,
// 85 per segment, runs as dense GEMMs on the fifth-generation tensor cores (tcgen05.mma, FP32
// accumulation in Tensor Memory). The 2048-point inverse DFT is factored in four steps with
// F = 32 x 64, m = m1 + 32 m2 and n = 64 n1 + n2:
//
//   D1[n2; t, m1] = sum_m2 e^{2 pi i m2 n2 / 64} U_t[m1 + 32 m2]           (GEMM, K = 64 complex)
//   V [n2; t, m1] = e^{2 pi i m1 n2 / 2048} D1[n2; t, m1]                   (CUDA cores)
//   u_t[64 n1 + n2] = sum_m1 e^{2 pi i m1 n1 / 32} V[n2; t, m1]             (GEMM, K = 32 complex)
//
// Complex products are written in real form, [re; im] = [[c, -s], [s, c]] [re; im], so each GEMM
// is a real GEMM of twice the size. The tensor cores take 16-bit operands, so each operand x is
// split into x = hi + lo with hi = round16(x), lo = round16(x - hi), and a product A B is
// accumulated as A_lo B_hi + A_hi B_lo + A_hi B_hi (the A_lo B_lo term is below FP32 rounding of
// the result). With BF16 halves this keeps about 16 significant bits per operand; with FP16 halves
// (FDAS_FP16S) about 22 bits, but FP16's range needs scaling: the product U = W * T_t is scaled
// by 2^k per segment, chosen from the largest component of W so that |U| < 2^14.5 (|T_t| is at
// most sqrt(n_tap) <= 32 because the taps have unit energy), and the mid-stage twiddles carry a
// factor 2^-6 so that the 64-term sums D1 stay in range. The power is rescaled by 2^(12 - 2k).
//
// Per CTA (128 threads, two CTAs per SM) the constant operands are set up once: the real-form
// 64-point DFT matrix (both halves) in Tensor Memory as the A operand of step 1, the real-form
// 32-point DFT matrix in shared memory as the B operand of step 3, and a table of the mid-stage
// twiddles. Templates are processed in pairs:
//   prep  (CUDA cores)  U = W * T_t for both templates, split, stored as step 1's B operand;
//   MMA1  (one thread)  24 MMAs, M = 128 (n2, re/im), N = 64 (two templates x 32 m1), K = 128;
//   mid   (CUDA cores)  D1 from TMEM, partner component by shuffle, twiddle, split, stored as
//                       step 3's A operand (rows: two templates x 64 n2);
//   MMA3  (one thread)  12 MMAs, M = 128, N = 64 (n1, re/im), K = 64;
//   out   (CUDA cores)  D3 from TMEM, |u|^2 of the kept outputs, coalesced stores.
// The other CTA on the SM overlaps its CUDA-core stages with this CTA's MMAs. Every wait (template
// copies, MMA completion) is bounded; a wait that gives up sets the device status word, and the
// CTA stops issuing work, waits once more (bounded) for what it issued and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ols_common.cuh"
#include "tc_ops.cuh"

namespace fdas {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTmemCols = 256;  // R64 hi [0,64), R64 lo [64,128), D1 [128,192), D3 [192,256)

// Shared memory (bytes). Region X holds the forward FFT's exchange buffers, later step 1's B
// operand (2 x 16 KB) and then step 3's A operand (2 x 16 KB); their lifetimes do not overlap.
constexpr int kXBytes = 2 * kPadded * 8;             // 34816
constexpr int kB1Term = 64 * 128 * 2;                // rows (t, m1) x K (m2, re/im), 16-bit
constexpr int kA3Term = 128 * 64 * 2;                // rows (t, n2) x K (re/im, m1)
constexpr int kB3Term = 64 * 64 * 2;                 // rows (n1, re/im) x K (re/im, m1)
constexpr int kTwRow = 32 * 8 + 16;                  // 32 twiddles per n2 row, padded by 16 bytes
constexpr int kOffT = kXBytes;                       // two templates, FP32 complex
constexpr int kOffB3 = kOffT + 2 * kF * 8;
constexpr int kOffTw = kOffB3 + 2 * kB3Term;
constexpr int kOffBar = kOffTw + 64 * kTwRow;
constexpr int kTcSmemBytes = kOffBar + 64;
static_assert(2 * kB1Term <= kXBytes && 2 * kA3Term <= kXBytes, "operands fit in the exchange region");
static_assert(kOffT % 128 == 0 && kOffB3 % 1024 == 0 && kOffTw % 16 == 0 && kOffBar % 8 == 0, "alignment");

// Byte offset of element (row, k) in a K-major operand without swizzle: 8 x 8 core matrices of
// 128 bytes, K-adjacent core matrices 128 bytes apart, row groups `sbo` bytes apart.
__host__ __device__ constexpr int kmajor_off(int row, int k, int sbo) {
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// x = hi + lo in two 16-bit halves (BF16 or FP16), two values per 32-bit word (a low, b high).
template <bool HALF>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    if (HALF) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}
template <bool HALF>
__device__ __forceinline__ void split1(float a, uint16_t &hi, uint16_t &lo) {
    uint32_t h, l;
    split2<HALF>(a, 0.f, h, l);
    hi = (uint16_t)(h & 0xFFFFu);
    lo = (uint16_t)(l & 0xFFFFu);
}

// Bounded mbarrier wait that also gives up at once when the CTA has already aborted.
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity, volatile int *aborted) {
    if (*aborted) return false;
    if (mbar_wait(bar, parity)) return true;
    *aborted = 1;
    return false;
}

// Expect `bytes` on the mbarrier, then copy `count` consecutive templates into shared memory.
__device__ __forceinline__ void load_templates(float2 *dst, const float2 *src, int count, unsigned long long *bar) {
    const unsigned bytes = (unsigned)(count * kF * sizeof(float2));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    for (int i = 0; i < count; ++i)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_u32(dst + i * kF)),
            "l"(src + (size_t)i * kF), "r"((unsigned)(kF * sizeof(float2))), "r"(smem_u32(bar))
            : "memory");
}

template <bool HALF, class Jobs>
__global__ void __launch_bounds__(kTcThreads, 2)
    fdas_ols_tc(Jobs jobs, const float2 *__restrict__ tmpl, int n_temp, int h, int keep) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *buf0 = reinterpret_cast<float2 *>(smem);
    float2 *buf1 = buf0 + kPadded;
    unsigned char *const opx = smem;  // step 1's B operand, then step 3's A operand (hi, then lo)
    float2 *tbuf = reinterpret_cast<float2 *>(smem + kOffT);
    unsigned char *const b3 = smem + kOffB3;
    unsigned char *const twt = smem + kOffTw;
    unsigned long long *tbar = reinterpret_cast<unsigned long long *>(smem + kOffBar);
    unsigned long long *mbar = tbar + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tbar + 2);
    volatile int *aborted = reinterpret_cast<volatile int *>(tbar + 3);
    unsigned *red = reinterpret_cast<unsigned *>(tbar + 4);  // [4] per-warp maxima

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const float2 *wtab = tmpl + (size_t)n_temp * kF;  // exp(-2 pi i k / F)
    constexpr uint32_t kIdesc = tc::idesc_f16(128, 64, !HALF);

    if (tid == 0) {
        mbar_init(tbar);
        mbar_init(mbar);
        *aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (w == 0) tc::tmem_alloc(tslot, kTmemCols);

    // Step 3's B operand: rows nu = 2 n1 + c, K index k3 = 32 c' + m1, entries of the real form of
    // e^{2 pi i m1 n1 / 32}. Both halves.
    for (int i = tid; i < 64 * 64; i += kTcThreads) {
        const int nu = i >> 6, k3 = i & 63;
        const int n1 = nu >> 1, c = nu & 1, cp = k3 >> 5, m1 = k3 & 31;
        const float2 e0 = __ldg(&wtab[64 * ((m1 * n1) & 31)]);
        const float er = e0.x, ei = -e0.y;  // conj: e^{+2 pi i m1 n1 / 32}
        const float v = c == 0 ? (cp == 0 ? er : -ei) : (cp == 0 ? ei : er);
        uint16_t hi, lo;
        split1<HALF>(v, hi, lo);
        const int o = kmajor_off(nu, k3, 1024);
        *reinterpret_cast<uint16_t *>(b3 + o) = hi;
        *reinterpret_cast<uint16_t *>(b3 + kB3Term + o) = lo;
    }
    // Mid-stage twiddles e^{2 pi i m1 n2 / 2048} (times 2^-6 for FP16), row n2, column m1.
    for (int i = tid; i < 64 * 32; i += kTcThreads) {
        const int n2 = i >> 5, m1 = i & 31;
        const float2 e0 = __ldg(&wtab[m1 * n2]);
        const float s2 = HALF ? 0.015625f : 1.f;
        *reinterpret_cast<float2 *>(twt + n2 * kTwRow + m1 * 8) = make_float2(e0.x * s2, -e0.y * s2);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;
    const uint32_t t_ahi = tm, t_alo = tm + 64, t_d1 = tm + 128, t_d3 = tm + 192;
    const uint32_t lane_base = (uint32_t)(32 * w) << 16;

    // Step 1's A operand into TMEM: this thread's lane l = tid is output row (n2, c) with
    // n2 = 16 w + (lane & 15), c = lane >> 4; K index k = 32 wq + 2 q + c' is input (m2 = wq + 4 q, c').
    {
        const int n2 = 16 * w + (lane & 15), c = lane >> 4;
#pragma unroll 1
        for (int j0 = 0; j0 < 64; j0 += 16) {
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float v2[2];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int k = 2 * (j0 + j) + b;
                    const int m2 = (k >> 5) + 4 * ((k & 31) >> 1), cp = k & 1;
                    const float2 e0 = __ldg(&wtab[32 * ((m2 * n2) & 63)]);
                    const float er = e0.x, ei = -e0.y;  // e^{+2 pi i m2 n2 / 64}
                    v2[b] = c == 0 ? (cp == 0 ? er : -ei) : (cp == 0 ? ei : er);
                }
                split2<HALF>(v2[0], v2[1], hw[j], lw[j]);
            }
            tc::tmem_st16(t_ahi + lane_base + j0, hw);
            tc::tmem_st16(t_alo + lane_base + j0, lw);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    // Forward-FFT twiddles of this thread (as in the FP32 kernel).
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

    unsigned tphase = 0u, mphase = 0u;
    bool t_pending = false;  // a template copy was issued and not yet waited for
    const float inv_f = 1.0f / kF;
    const int n_items = jobs.total();
    // Out stage: this thread's TMEM lane 32 w + lane is output row (t_local, n2).
    const int o_tl = w >> 1, o_n2 = 32 * (w & 1) + lane;
    // Mid stage: partner sign of the twiddle product (see below).
    const float msign = (lane >> 4) ? 1.f : -1.f;
    const int m_n2 = 16 * w + (lane & 15), m_c = lane >> 4;

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Item it = jobs.get(item);
        const int n = it.n, s = it.s, t0 = it.t0, t1 = it.t1;
        const float2 *__restrict__ spec = it.spec;
        const int origin = s * keep - h;
        const int col0 = s * keep - h;
        // Outputs n = 64 n1 + o_n2 this thread stores: kept (h <= n < h + keep) and inside the spectrum.
        uint32_t omask = 0u;
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const int m = 64 * n1 + o_n2;
            if (m >= h && m < h + keep && col0 + m < n) omask |= 1u << n1;
        }
        if (tid == 0 && !*aborted) load_templates(tbuf, tmpl + (size_t)t0 * kF, min(2, t1 - t0), tbar);
        t_pending = true;

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
            for (int r = 0; r < 8; ++r) W[2 * r] = make_float2(u[r].x * inv_f, u[r].y * inv_f);
            fft_pass_3<false>(u, buf1, tw3b, tid + 128);
#pragma unroll
            for (int r = 0; r < 8; ++r) W[2 * r + 1] = make_float2(u[r].x * inv_f, u[r].y * inv_f);
        }
        float pscale = 1.f;
        if (HALF) {
            float mx = 0.f;
#pragma unroll
            for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fmaxf(fabsf(W[q].x), fabsf(W[q].y)));
            const unsigned mb = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(mx));
            if (lane == 0) red[w] = mb;
            __syncthreads();  // also ends every thread's reads of buf1 before region X is reused
            const unsigned mall = max(max(red[0], red[1]), max(red[2], red[3]));
            // 2^k with k = 8 - exponent(max component), so that |U| 2^k < 2^14.5.
            int k = mall ? 8 - ((int)((mall >> 23) & 0xFF) - 127) : 0;
            k = max(-40, min(40, k));
            const float s1 = __uint_as_float((unsigned)(k + 127) << 23);
#pragma unroll
            for (int q = 0; q < 16; ++q) W[q] = make_float2(W[q].x * s1, W[q].y * s1);
            pscale = __uint_as_float((unsigned)(12 - 2 * k + 127) << 23);
        } else {
            __syncthreads();  // every thread's reads of buf1 end before region X is reused
        }

        for (int t = t0; t < t1; t += 2) {
            const int tb = min(2, t1 - t);
            tc_wait(tbar, tphase, aborted);
            tphase ^= 1u;
            t_pending = false;
            // prep: U = W T_t; B1 row 32 tl + lane, K chunk 4 w + i holds q = 4 i .. 4 i + 3.
#pragma unroll
            for (int tl = 0; tl < 2; ++tl) {
                uint32_t hw[16], lw[16];
                const float2 *T = tbuf + tl * kF + tid;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float2 u = tl < tb ? cmul(W[q], T[128 * q]) : make_float2(0.f, 0.f);
                    split2<HALF>(u.x, u.y, hw[q], lw[q]);
                }
                unsigned char *row = opx + kmajor_off(32 * tl + lane, 32 * w, 2048);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    *reinterpret_cast<uint4 *>(row + 128 * i) = make_uint4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
                    *reinterpret_cast<uint4 *>(row + kB1Term + 128 * i) =
                        make_uint4(lw[4 * i], lw[4 * i + 1], lw[4 * i + 2], lw[4 * i + 3]);
                }
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0 && !*aborted) {
                // Every thread has read the template buffer: bring in the next pair.
                if (t + 2 < t1) load_templates(tbuf, tmpl + (size_t)(t + 2) * kF, min(2, t1 - t - 2), tbar);
                tc::fence_after_sync();
                const uint32_t b1 = smem_u32(opx);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const uint64_t bh = tc::desc_kmajor(b1 + 256 * kk, 128, 2048);
                    const uint64_t bl = tc::desc_kmajor(b1 + kB1Term + 256 * kk, 128, 2048);
                    tc::mma_ts(t_d1, t_alo + 8 * kk, bh, kIdesc, kk > 0);
                    tc::mma_ts(t_d1, t_ahi + 8 * kk, bl, kIdesc, 1u);
                    tc::mma_ts(t_d1, t_ahi + 8 * kk, bh, kIdesc, 1u);
                }
                tc::commit(reinterpret_cast<uint64_t *>(mbar));
            }
            if (t + 2 < t1) t_pending = true;
            tc_wait(mbar, mphase, aborted);
            mphase ^= 1u;
            tc::fence_after_sync();

            // mid: this thread holds component c of D1 at (n2, t, m1); the partner lane (lane ^ 16)
            // holds the other. Own component of V = D1 e^{2 pi i m1 n2 / F}: x wr + sign p wi with
            // sign -1 for the real part, +1 for the imaginary part.
#pragma unroll
            for (int tl = 0; tl < 2; ++tl) {
                uint32_t x[32];
                tc::tmem_ld32(t_d1 + lane_base + 32 * tl, x);
                uint32_t hw[16], lw[16];
                const unsigned char *trow = twt + m_n2 * kTwRow;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float4 tw = *reinterpret_cast<const float4 *>(trow + 16 * j);
                    const float xa = __uint_as_float(x[2 * j]), xb = __uint_as_float(x[2 * j + 1]);
                    const float pa = __shfl_xor_sync(0xFFFFFFFFu, xa, 16);
                    const float pb = __shfl_xor_sync(0xFFFFFFFFu, xb, 16);
                    const float va = fmaf(xa, tw.x, msign * pa * tw.y);
                    const float vb = fmaf(xb, tw.z, msign * pb * tw.w);
                    split2<HALF>(va, vb, hw[j], lw[j]);
                }
                unsigned char *row = opx + kmajor_off(64 * tl + m_n2, 32 * m_c, 1024);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    *reinterpret_cast<uint4 *>(row + 128 * i) = make_uint4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
                    *reinterpret_cast<uint4 *>(row + kA3Term + 128 * i) =
                        make_uint4(lw[4 * i], lw[4 * i + 1], lw[4 * i + 2], lw[4 * i + 3]);
                }
            }
            tc::fence_before_sync();
            tc::fence_proxy_async();
            __syncthreads();
            if (tid == 0 && !*aborted) {
                tc::fence_after_sync();
                const uint32_t a3 = smem_u32(opx), bb = smem_u32(b3);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ah = tc::desc_kmajor(a3 + 256 * kk, 128, 1024);
                    const uint64_t al = tc::desc_kmajor(a3 + kA3Term + 256 * kk, 128, 1024);
                    const uint64_t bh = tc::desc_kmajor(bb + 256 * kk, 128, 1024);
                    const uint64_t bl = tc::desc_kmajor(bb + kB3Term + 256 * kk, 128, 1024);
                    tc::mma_ss(t_d3, al, bh, kIdesc, kk > 0);
                    tc::mma_ss(t_d3, ah, bl, kIdesc, 1u);
                    tc::mma_ss(t_d3, ah, bh, kIdesc, 1u);
                }
                tc::commit(reinterpret_cast<uint64_t *>(mbar));
            }
            tc_wait(mbar, mphase, aborted);
            mphase ^= 1u;
            tc::fence_after_sync();

            // out: columns 2 n1 + c of this thread's lane hold (re, im) of u[64 n1 + o_n2].
            if (o_tl < tb) {
                float *const dst = it.plane + (size_t)(t + o_tl) * it.ld + col0 + o_n2;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t y[32];
                    tc::tmem_ld32(t_d3 + lane_base + 32 * hh, y);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int n1 = 16 * hh + i;
                        const float re = __uint_as_float(y[2 * i]), im = __uint_as_float(y[2 * i + 1]);
                        const float pw = fmaf(re, re, im * im) * pscale;
                        if ((omask >> n1) & 1u) dst[64 * n1] = pw;
                    }
                }
            }
            tc::fence_before_sync();
        }
    }

    // Teardown: nothing of this CTA may be in flight when its TMEM is freed.
    __syncthreads();
    if (t_pending) mbar_wait(tbar, tphase);
    if (tid == 0) tc::commit(reinterpret_cast<uint64_t *>(mbar));
    mbar_wait(mbar, mphase);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (w == 0) tc::tmem_dealloc(tm, kTmemCols);
}

template <bool HALF, class Jobs>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(fdas_ols_tc<HALF, Jobs>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
}

}  // namespace

cudaError_t launch_convolve_tc(const Geometry &g, const float2 *spec, size_t n, const float2 *tmpl, float *plane,
                               size_t ld, int ctas_per_sm, int templates_per_item, cudaStream_t s) {
    SingleJobs jobs;
    jobs.spec = spec;
    jobs.plane = plane;
    jobs.ld = ld;
    jobs.n = (int)n;
    jobs.n_seg = (int)((n + g.keep - 1) / g.keep);
    jobs.n_temp = g.n_temp;
    const int tpi = templates_per_item > 0 ? templates_per_item : kTcDefaultTemplatesPerItem;
    jobs.t_chunk = tpi < g.n_temp ? tpi : g.n_temp;
    jobs.n_tchunk = (g.n_temp + jobs.t_chunk - 1) / jobs.t_chunk;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int ctas = ctas_per_sm > 0 && ctas_per_sm < kTcMaxCtasPerSm ? ctas_per_sm : kTcMaxCtasPerSm;
    const int items = jobs.n_seg * jobs.n_tchunk;
    const int grid = items < ctas * sms ? items : ctas * sms;
    const bool half = g.precision == FDAS_FP16S;
    e = half ? set_smem<true, SingleJobs>() : set_smem<false, SingleJobs>();
    if (e != cudaSuccess) return e;
    if (half)
        fdas_ols_tc<true><<<grid, kTcThreads, kTcSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    else
        fdas_ols_tc<false><<<grid, kTcThreads, kTcSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    return cudaGetLastError();
}

cudaError_t prepare_convolve_batch_tc() {
    cudaError_t e = set_smem<true, BatchJobs>();
    if (e == cudaSuccess) e = set_smem<false, BatchJobs>();
    return e;
}

cudaError_t launch_convolve_batch_tc(const Geometry &g, const ConvBatch &batch, const float2 *tmpl, int grid,
                                     int templates_per_item, cudaStream_t s) {
    BatchJobs jobs;
    jobs.batch = batch;
    jobs.n_temp = g.n_temp;
    const int tpi = templates_per_item > 0 ? templates_per_item : kTcDefaultTemplatesPerItem;
    jobs.t_chunk = tpi < g.n_temp ? tpi : g.n_temp;
    jobs.n_tchunk = (g.n_temp + jobs.t_chunk - 1) / jobs.t_chunk;
    if (g.precision == FDAS_FP16S)
        fdas_ols_tc<true><<<grid, kTcThreads, kTcSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    else
        fdas_ols_tc<false><<<grid, kTcThreads, kTcSmemBytes, s>>>(jobs, tmpl, g.n_temp, g.h, g.keep);
    return cudaGetLastError();
}

cudaError_t device_status_tc(unsigned *flags, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_device_status, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof(unsigned));
    }
    return e;
}

}  // namespace fdas
