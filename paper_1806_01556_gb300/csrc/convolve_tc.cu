// FT convolution with the tensor cores: precisions FDAS_BF16X3 and FDAS_FP16S.
//
// The overlap-save steps are those of the FP32 kernel (Sec. 2.1): segment s of F = 2048 input
// points is transformed once (FP32 FFT in registers), multiplied by each template T_t, transformed
// back, and |u|^2 of the L = F - n_tap + 1 valid outputs is stored. The inverse transform, 85 per
// segment, is factored in four steps with F = 32 x 64, m = m1 + 32 m2 and n = 64 n1 + n2:
//
//   D1[n2; t, m1] = sum_m2 e^{2 pi i m2 n2 / 64} U_t[m1 + 32 m2]   (tensor cores, two thirds of the work)
//   V [n2; t, m1] = e^{2 pi i m1 n2 / 2048} D1[n2; t, m1]           (CUDA cores, FP32)
//   u_t[64 n1 + n2] = sum_m1 e^{2 pi i m1 n1 / 32} V[n2; t, m1]     (CUDA cores, FP32, in registers)
//
// The first step is a dense GEMM on the fifth-generation tensor cores (tcgen05.mma, FP32
// accumulation in Tensor Memory), in real form: [re; im] = [[c, -s], [s, c]] [re; im], so it is a
// real GEMM with M = 128 (n2, re/im), K = 128 (m2, re/im), N = 32 m1 per template. The tensor cores
// take 16-bit operands, so each operand x is split into x = hi + lo with hi = round16(x),
// lo = round16(x - hi), and a product A B is accumulated as A_lo B_hi + A_hi B_lo + A_hi B_hi (the
// A_lo B_lo term is below FP32 rounding of the result). With BF16 halves (FDAS_BF16X3) this keeps
// about 16 significant bits per operand; with FP16 halves (FDAS_FP16S) about 22 bits, but FP16's
// range needs scaling: the product U = W * T_t is scaled by 2^k per segment, chosen from the
// largest component of W so that |U| < 2^14.5 (|T_t| is at most sqrt(n_tap) <= 32 because the taps
// have unit energy); the 64-term sums D1 are FP32 and the twiddles carry a factor 2^-6 that the
// power rescaling 2^(12 - 2k) undoes.
//
// One persistent CTA per SM runs three independent worker groups of 4 warps; each group owns a
// stream of work items (a segment with a range of templates) and its own shared-memory operand
// and TMEM accumulator, and is served by its own MMA-issue warp:
//   prep  (group)       forward FFT of the segment (W kept in shared memory); per pair of templates
//                       U = W * T_t (templates read from L2), split, stored as the GEMM's B operand
//                       (rows: 2 templates x 32 m1, K: 64 m2 x re/im);
//   MMA   (warp 12 + g) one thread issues 24 MMAs per pair (M = 128, N = 64, K = 128; A = the
//                       real-form 64-point DFT matrix, both halves, resident in Tensor Memory);
//   mid   (group)       D1 from TMEM (each thread holds the real or the imaginary row of one n2; the
//                       partner lane 16 away holds the other), the twiddle product, a 32-point DFT
//                       in registers (radix 4 x 8), |u|^2 of the kept outputs, coalesced stores.
// While one group waits for its GEMM the other two keep the CUDA cores busy, and the tensor cores
// take the three groups' GEMMs in turn. Every wait is bounded: a wait that gives up sets the device
// status word and an abort flag, after which no role issues work or waits again; before freeing its
// TMEM the CTA waits once more, bounded, for whatever it had issued.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ols_common.cuh"
#include "tc_ops.cuh"

namespace fdas {
namespace {

constexpr int kGroups = 3;                            // worker groups of 4 warps
constexpr int kMmaWarp0 = 4 * kGroups;                // MMA-issue warps 12, 13, 14
constexpr int kTcThreads = (4 * kGroups + kGroups) * 32;
constexpr uint32_t kTmemCols = 512;
// Tensor Memory columns: the DFT matrix (hi, lo), then one D1 per group.
constexpr uint32_t kColAhi = 0, kColAlo = 64, kColD1 = 128;

// Shared memory (bytes), per group: region X (the forward FFT's exchange buffers, then the GEMM's
// B operand, hi and lo) and W; then the twiddle table, barriers and small state.
constexpr int kB1Term = 64 * 128 * 2;                 // rows (t_local, m1) x K (m2, re/im), 16-bit
constexpr int kXBytes = 2 * kPadded * 8;
constexpr int kGroupBytes = kXBytes + kF * 8;         // region X + W
constexpr int kTwRow = 32 * 8 + 16;                   // 32 twiddles per n2 row, padded by 16 bytes
constexpr int kOffTw = kGroups * kGroupBytes;
constexpr int kOffBar = kOffTw + 64 * kTwRow;
constexpr int kNumBars = 2 * kGroups + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kTcSmemBytes = kOffMisc + 16 + 16 * kGroups + 64 * kGroups;
static_assert(2 * kB1Term <= kXBytes, "the operand fits in the FFT's region");
static_assert(kGroupBytes % 1024 == 0 && kOffTw % 16 == 0 && kOffBar % 8 == 0, "alignment");
static_assert(kTcSmemBytes <= 227 * 1024, "shared memory per CTA");

// Byte offset of element (row, k) in a K-major operand without swizzle: 8 x 8 core matrices of
// 128 bytes, K-adjacent core matrices 128 bytes apart, row groups `sbo` bytes apart.
__host__ __device__ constexpr int kmajor_off(int row, int k, int sbo) {
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

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

// Bounded mbarrier wait that also gives up at once when the CTA has already aborted.
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity, volatile int *aborted) {
    if (*aborted) return false;
    if (mbar_wait(bar, parity)) return true;
    *aborted = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_n(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// v * e^{2 pi i k / 32} for k known at compile time after unrolling.
__device__ __forceinline__ float2 w32(float2 v, int k) {
    constexpr float C[9] = {1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                            0.70710678118654752f, 0.55557023301960218f, 0.38268343236508977f,
                            0.19509032201612825f, 0.f};  // cos(2 pi j / 32), j = 0..8
    k &= 31;
    if (k == 0) return v;
    if (k == 8) return make_float2(-v.y, v.x);
    if (k == 16) return make_float2(-v.x, -v.y);
    if (k == 24) return make_float2(v.y, -v.x);
    const float c = k <= 8 ? C[k] : k <= 16 ? -C[16 - k] : k <= 24 ? -C[k - 16] : C[32 - k];
    const float sn = k <= 8 ? C[8 - k] : k <= 16 ? C[k - 8] : k <= 24 ? -C[24 - k] : -C[k - 24];
    return make_float2(fmaf(v.x, c, -v.y * sn), fmaf(v.x, sn, v.y * c));
}

// In-place inverse 32-point DFT, natural order: u[n] = sum_m v[m] e^{2 pi i m n / 32}. Radix 4 x 8:
// m = a + 8 b, n = 4 c + d: 4-point DFTs over b, twiddles e^{2 pi i a d / 32}, 8-point DFTs over a.
// Scalar sums here: the packed FP32x2 form measured slightly slower in this kernel.
__device__ __forceinline__ void idft32(float2 (&v)[32]) {
#pragma unroll
    for (int a = 0; a < 8; ++a) dft4<true, false>(v[a], v[a + 8], v[a + 16], v[a + 24]);
#pragma unroll
    for (int a = 1; a < 8; ++a)
#pragma unroll
        for (int d = 1; d < 4; ++d) v[a + 8 * d] = w32(v[a + 8 * d], a * d);
    float2 u[32];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        float2 x[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) x[a] = v[a + 8 * d];
        dft8<true, false>(x);
#pragma unroll
        for (int c = 0; c < 8; ++c) u[4 * c + d] = x[c];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = u[i];
}

// Barrier indices: per group g, B1 full (4 warp arrivals) and D1 full (MMA commit).
__device__ __forceinline__ int bar_b1full(int g) { return 2 * g; }
__device__ __forceinline__ int bar_d1full(int g) { return 2 * g + 1; }
constexpr int kBarFin = 2 * kGroups;

// Named barrier of group g's four warps (ids 1..kGroups).
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;\n" ::"r"(g + 1) : "memory"); }

template <bool HALF, class Jobs>
__global__ void __launch_bounds__(kTcThreads, 1)
    fdas_ols_tc(Jobs jobs, const float2 *__restrict__ tmpl, int n_temp, int h, int keep) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *const twt = smem + kOffTw;
    unsigned long long *const bars = reinterpret_cast<unsigned long long *>(smem + kOffBar);
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *const aborted = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const float2 *wtab = tmpl + (size_t)n_temp * kF;  // exp(-2 pi i k / F)
    const int n_items = jobs.total();
    const int n_virt = gridDim.x * kGroups;  // worker groups across the grid

    if (tid == 0) {
        for (int g = 0; g < kGroups; ++g) {
            mbar_init_n(&bars[bar_b1full(g)], 4);
            mbar_init_n(&bars[bar_d1full(g)], 1);
        }
        mbar_init_n(&bars[kBarFin], 1);
        *aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (w == 0) tc::tmem_alloc(tslot, kTmemCols);

    // Mid-stage twiddles e^{2 pi i m1 n2 / 2048} (times 2^-6 for FP16), row n2, column m1.
    for (int i = tid; i < 64 * 32; i += kTcThreads) {
        const int n2 = i >> 5, m1 = i & 31;
        const float2 e0 = __ldg(&wtab[m1 * n2]);
        const float s2 = HALF ? 0.015625f : 1.f;
        *reinterpret_cast<float2 *>(twt + n2 * kTwRow + m1 * 8) = make_float2(e0.x * s2, -e0.y * s2);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tslot;
    const uint32_t lane_base = (uint32_t)(32 * (w & 3)) << 16;

    // The GEMM's A operand into TMEM (warps 0-3, one lane each): lane l is output row (n2, c) with
    // n2 = 16 (l >> 5) + (l & 15), c = (l >> 4) & 1; K index k = 32 wq + 2 q + c' is input
    // (m2 = wq + 4 q, c').
    if (w < 4) {
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
            tc::tmem_st16(tm + kColAhi + lane_base + j0, hw);
            tc::tmem_st16(tm + kColAlo + lane_base + j0, lw);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    if (w < kMmaWarp0) {
        // ------------------------------------------------------------------ worker group g
        const int g = w >> 2, gt = tid & 127;  // group and thread index within the group
        unsigned char *const region = smem + g * kGroupBytes;  // FFT buffers, then B1 (hi, lo)
        float2 *const Ws = reinterpret_cast<float2 *>(region + kXBytes);
        float2 *buf0 = reinterpret_cast<float2 *>(region);
        float2 *buf1 = buf0 + kPadded;
        unsigned *const red = reinterpret_cast<unsigned *>(smem + kOffMisc + 16 + 16 * g);  // [4]
        const uint32_t d1 = tm + kColD1 + 64 * g + lane_base;
        // Mid role: TMEM lane 32 (w & 3) + lane is D1 row (n2, c). The even lane (c = 0) finishes
        // template 0 of the pair (it needs the imaginary part from its partner), the odd lane
        // template 1 (it needs the real part).
        const int n2 = 16 * (w & 3) + (lane & 15);
        const int tlm = lane >> 4;
        const bool odd = tlm != 0;
        const unsigned char *trow = twt + n2 * kTwRow;
        const float inv_f = 1.0f / kF;
        int p = 0;  // pair counter of this group
        for (int item = blockIdx.x * kGroups + g; item < n_items; item += n_virt) {
            const Item it = jobs.get(item);
            const int n = it.n, t0 = it.t0, t1 = it.t1;
            const int origin = it.s * keep - h;
            const int col0 = it.s * keep - h;
            // Forward FFT of the segment: W[q] = DFT(w_s)[gt + 128 q] / F, kept in shared memory
            // (each thread reads back only what it wrote). Region X is free: this group's last
            // GEMM has completed (its D1 was read).
            float pscale = 1.f;
            {
                float2 v[16];
                {
                    float2 tw2[16];
                    const int k = gt & 15;
#pragma unroll
                    for (int q = 0; q < 16; ++q) tw2[q] = __ldg(&wtab[8 * ((k * q) & 255)]);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int idx = origin + gt + 128 * q;
                        v[q] = (idx >= 0 && idx < n) ? __ldg(&it.spec[idx]) : make_float2(0.f, 0.f);
                    }
                    fft_passes_12<false>(v, buf0, buf1, tw2, gt, [] {}, [g] { group_sync(g); });
                }
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    float2 tw3[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) tw3[q] = __ldg(&wtab[(gt + 128 * hh) * q]);
                    float2 u[8];
                    fft_pass_3<false>(u, buf1, tw3, gt + 128 * hh);
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[2 * q + hh] = make_float2(u[q].x * inv_f, u[q].y * inv_f);
                }
                if (HALF) {
                    float mx = 0.f;
#pragma unroll
                    for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
                    const unsigned mb = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(mx));
                    if (lane == 0) red[w & 3] = mb;
                    group_sync(g);
                    const unsigned mall = max(max(red[0], red[1]), max(red[2], red[3]));
                    // 2^k with k = 8 - exponent(max component), so that |U| 2^k < 2^14.5.
                    int k = mall ? 8 - ((int)((mall >> 23) & 0xFF) - 127) : 0;
                    k = max(-40, min(40, k));
                    const float s1 = __uint_as_float((unsigned)(k + 127) << 23);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = make_float2(v[q].x * s1, v[q].y * s1);
                    pscale = __uint_as_float((unsigned)(12 - 2 * k + 127) << 23);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) Ws[gt + 128 * q] = v[q];
            }
            group_sync(g);  // every thread of the group is done with the FFT buffers (and red[])
            uint32_t omask = 0u;  // outputs n = 64 n1 + n2 kept (h <= n < h + keep) and inside the spectrum
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) {
                const int m = 64 * n1 + n2;
                if (m >= h && m < h + keep && col0 + m < n) omask |= 1u << n1;
            }

            for (int t = t0; t < t1; t += 2, ++p) {
                const int tb = min(2, t1 - t);
                // prep: U = W T_t; B1 row 32 tl + lane, K chunk 4 (w & 3) + i holds q = 4 i .. 4 i + 3.
                for (int tl = 0; tl < tb; ++tl) {
                    const float2 *T = tmpl + (size_t)(t + tl) * kF + gt;
                    float2 tv[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) tv[q] = __ldg(&T[128 * q]);
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float2 u = cmul(Ws[gt + 128 * q], tv[q]);
                        split2<HALF>(u.x, u.y, hw[q], lw[q]);
                    }
                    unsigned char *row = region + kmajor_off(32 * tl + lane, 32 * (w & 3), 2048);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        *reinterpret_cast<uint4 *>(row + 128 * i) =
                            make_uint4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
                        *reinterpret_cast<uint4 *>(row + kB1Term + 128 * i) =
                            make_uint4(lw[4 * i], lw[4 * i + 1], lw[4 * i + 2], lw[4 * i + 3]);
                    }
                }
                tc::fence_before_sync();  // this warp's reads of D1 (previous pair) are done
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[bar_b1full(g)]);

                // mid: wait for the GEMM, then finish both templates of the pair.
                tc_wait(&bars[bar_d1full(g)], p & 1, aborted);
                tc::fence_after_sync();
                float2 v[32];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t xe[16], xo[16];  // own component (re if even lane, im if odd) of templates 0, 1
                    tc::tmem_ld16x2(d1 + 16 * hh, xe, d1 + 32 + 16 * hh, xo);
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const int m1 = 16 * hh + i;
                        const float ga = __shfl_xor_sync(0xFFFFFFFFu, __uint_as_float(odd ? xe[i] : xo[i]), 16);
                        const float gb = __shfl_xor_sync(0xFFFFFFFFu, __uint_as_float(odd ? xe[i + 1] : xo[i + 1]), 16);
                        const float2 da = odd ? make_float2(ga, __uint_as_float(xo[i])) : make_float2(__uint_as_float(xe[i]), ga);
                        const float2 db = odd ? make_float2(gb, __uint_as_float(xo[i + 1])) : make_float2(__uint_as_float(xe[i + 1]), gb);
                        const float4 tw = *reinterpret_cast<const float4 *>(trow + 8 * m1);
                        v[m1] = cmul(da, make_float2(tw.x, tw.y));
                        v[m1 + 1] = cmul(db, make_float2(tw.z, tw.w));
                    }
                }
                idft32(v);  // v[n1] = u[64 n1 + n2]
                if (t + tlm < t1) {
                    float *const dst = it.plane + (size_t)(t + tlm) * it.ld + col0 + n2;
#pragma unroll
                    for (int n1 = 0; n1 < 32; ++n1) {
                        const float pw = HALF ? fmaf(v[n1].x, v[n1].x, v[n1].y * v[n1].y) * pscale
                                              : fmaf(v[n1].x, v[n1].x, v[n1].y * v[n1].y);
                        if ((omask >> n1) & 1u) dst[64 * n1] = pw;
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------------------------ MMA issue for group g
        const int g = w - kMmaWarp0;
        if (lane == 0) {
            constexpr uint32_t id1 = tc::idesc_f16(128, 64, !HALF);
            const uint32_t bs = smem_u32(smem + g * kGroupBytes);
            const uint32_t d1 = tm + kColD1 + 64 * g;
            int p = 0;
            for (int item = blockIdx.x * kGroups + g; item < n_items; item += n_virt) {
                const Item it = jobs.get(item);
                for (int t = it.t0; t < it.t1; t += 2, ++p) {
                    tc_wait(&bars[bar_b1full(g)], p & 1, aborted);
                    if (*aborted) continue;
                    tc::fence_after_sync();
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint64_t bh = tc::desc_kmajor(bs + 256 * kk, 128, 2048);
                        const uint64_t bl = tc::desc_kmajor(bs + kB1Term + 256 * kk, 128, 2048);
                        tc::mma_ts(d1, tm + kColAlo + 8 * kk, bh, id1, kk > 0);
                        tc::mma_ts(d1, tm + kColAhi + 8 * kk, bl, id1, 1u);
                        tc::mma_ts(d1, tm + kColAhi + 8 * kk, bh, id1, 1u);
                    }
                    tc::commit(reinterpret_cast<uint64_t *>(&bars[bar_d1full(g)]));
                }
            }
        }
        __syncwarp();
    }

    // Teardown: nothing of this CTA may be in flight when its TMEM is freed. Without an abort
    // every MMA was waited for; after one, wait (bounded) for the MMAs each issuer issued.
    tc::fence_before_sync();
    __syncthreads();
    if (*aborted) {
        for (int g = 0; g < kGroups; ++g) {
            if (tid == (kMmaWarp0 + g) * 32) tc::commit(reinterpret_cast<uint64_t *>(&bars[kBarFin]));
            mbar_wait(&bars[kBarFin], (unsigned)(g & 1));
            __syncthreads();
        }
    }
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

cudaError_t device_status_tc_async(unsigned *h_flags, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(h_flags, g_device_status, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
}

}  // namespace fdas
