// Harmonic summing with threshold detection (Sec. 2.2, Algorithm 1).
//
// Stretch read by fundamental (the default): HP_k(i, j) = sum_{l=1..k} P[c + l*i][l*j] on
// D_k = {|k*i| <= c, k*j <= n-1}, summed in float32 in the order l = 1, 2, ..., k. As in the
// paper's MultipleHP kernels, all planes are computed at once and no HP plane is stored: one
// thread owns one fundamental (i, j) and keeps the running sum in a register.
//
// GB300 mapping:
//   fdas_hs_reset    zeroes the per-plane crossing counters and peak keys in the workspace.
//   fdas_hs_k1       the single-plane rows (|i| > c/2): 16-byte streaming loads, 4096 columns per
//                    CTA. fdas_search with FP32 skips it: the convolution takes those rows' HP_1.
//   fdas_hs_kl<KL>   the rows with at least two planes (|i| <= c/2) in three launches, by their
//                    plane count K(i) = min(n_harm, floor(c/|i|)): 5-16, 3-4 and 2 (kGroups), each
//                    compiled for KL terms with a per-row cap at K(i). A CTA takes 16 chunks (8 in
//                    the batched form) of 256 J columns (J = 8, 6 or 2 fundamentals per thread for
//                    up to 4, 8 or 16 planes); in each chunk a thread issues every strided gather P[c + l i][l j] of
//                    its J fundamentals before summing, through the read-only path, and warps whose
//                    columns all have the same number of terms skip the per-element domain test.
//                    Crossings are rare and take a separate path: a ballot, one atomicAdd per warp,
//                    and a prefix popcount for each lane's slot. Each candidate
//                    is one 64-bit key whose ascending order is the canonical order (power desc,
//                    i asc, j asc). The loudest point of every plane comes from warp reductions
//                    (redux max of the power bits, then redux min of the column), a block merge in
//                    shared memory, and at most one 64-bit atomicMax per block and plane.
//   fdas_hs_hh8/16   the highest-harmonic indexing (FDAS_INDEX_HIGHEST), one launch over all rows.
//   The row-group launches (and fdas_hs_k1) are independent, so they run side by side on the
//   caller's stream and two auxiliary streams of the library, forked and joined with events.
//   fdas_hs_finalize one CTA per plane. A bitonic sort of the raw keys (2, 4 or 16 keys per thread in
//                    registers, shuffles for the middle strides, shared memory for the largest), then
//                    the top cand_cap keys decoded into fdas_cand records, the counts and the peaks.
#include <type_traits>

#include "hs_keys.cuh"

namespace fdas {
namespace {

constexpr int kHsThreads = 256;
constexpr int kFinThreads = 1024;

__global__ void fdas_hs_reset(unsigned long long *counters, unsigned long long *peaks, int n_harm) {
    const int t = threadIdx.x;
    if (t < n_harm) {
        counters[t] = 0ull;
        peaks[t] = 0ull;
    }
}

constexpr int kHsWarps = kHsThreads / 32;

// Block-level merge of the warps' peak keys and one atomicMax per block and plane, skipped when the
// block's key cannot win (peak keys only grow).
template <int KL>
__device__ __forceinline__ void block_peaks(const unsigned long long (&key)[KL], unsigned long long *peaks) {
    __shared__ unsigned long long warp_key[kHsWarps][KL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < KL; ++k) warp_key[warp][k] = key[k];
    }
    __syncthreads();
    if (threadIdx.x < KL) {
        unsigned long long m = 0ull;
#pragma unroll
        for (int w = 0; w < kHsWarps; ++w) m = warp_key[w][threadIdx.x] > m ? warp_key[w][threadIdx.x] : m;
        if (m > *(volatile unsigned long long *)&peaks[threadIdx.x]) atomicMax(&peaks[threadIdx.x], m);
    }
}

// Rows with a single plane (|2 i| > c): HP_1 = P. Each thread streams kK1Vec groups of 4
// consecutive columns, one 16-byte load each when the row stride allows it.
constexpr int kK1Vec = 4;
constexpr int kK1Cols = kHsThreads * 4 * kK1Vec;  // 4096 columns per CTA

__device__ __forceinline__ void hs_row_k1(const float *__restrict__ prow, int n, float ta, int row, int j0,
                                          unsigned long long *raw, unsigned long long *counters,
                                          unsigned long long *peaks, bool vec) {
    const int lane = threadIdx.x & 31;
    float v[kK1Vec][4];
#pragma unroll
    for (int g = 0; g < kK1Vec; ++g) {
        const int jt = j0 + 4 * (threadIdx.x + kHsThreads * g);
        if (vec && jt + 3 < n) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(prow + jt));
            v[g][0] = q.x, v[g][1] = q.y, v[g][2] = q.z, v[g][3] = q.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[g][u] = (jt + u < n) ? __ldg(prow + jt + u) : -1.0f;
        }
    }
    float best = -1.0f;
    int bestj = 0;
#pragma unroll
    for (int g = 0; g < kK1Vec; ++g)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool gt = v[g][u] > best;  // invalid columns hold -1 and never win
            best = gt ? v[g][u] : best;
            bestj = gt ? j0 + 4 * (threadIdx.x + kHsThreads * g) + u : bestj;
        }
    if (__any_sync(0xFFFFFFFFu, best > ta)) {
#pragma unroll
        for (int g = 0; g < kK1Vec; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                emit(v[g][u] > ta, v[g][u], row, (unsigned)(j0 + 4 * (threadIdx.x + kHsThreads * g) + u), 1, lane,
                     counters, raw);
    }
    unsigned long long key[1] = {warp_peak_key(best, bestj, row)};
    block_peaks<1>(key, peaks);
}

// Number of terms of fundamental column j: the planes l <= KL with l j <= n-1 (0 for j >= n).
template <int KL>
__device__ __forceinline__ int term_count(int j, int n) {
    if (j >= n) return 0;
    if (j == 0) return KL;
    const int t = (n - 1) / j;
    return t < KL ? t : KL;
}

// Rows with KL >= 2 planes. A CTA covers CH chunks of 256 J fundamental columns (J = jpt<KL>()); in a
// chunk, lane L of warp w handles j = jc + 32 J w + L + 32 u, u < J, so every gather of a warp is one coalesced stride-l
// access along a plane row. The per-plane best points accumulate over the chunks, and the peak
// reductions, the block merge and the atomics run once per CTA. UNIFORM: every fundamental of the
// warp's chunk has the same number T of terms, which holds for all warps but those straddling a
// boundary j = (n-1)/l.
constexpr int kChunks = 8;      // batched launches (their CTA tables assume this width)
constexpr int kChunksOne = 16;  // one spectrum: fewer, wider CTAs took the FP32 harmonic stage from 0.296
                                // to 0.284 ms at N = 2^21 (12 chunks: 0.288, 24: 0.285, 32: 0.287)
// Fundamentals per thread and chunk: more for few planes (more gathers in flight per thread: the
// 2- and 4-plane launches went from 0.166 to 0.126 ms at N = 2^21 with 8 instead of 4, the 5- to
// 8-plane launch gained 4% with 6 instead of 4), fewer for many planes, to keep the gathers in
// registers (8 for up to 8 planes spilled and lost 10%).
template <int KL>
__host__ __device__ constexpr int jpt() { return KL <= 4 ? 8 : KL <= 9 ? 6 : 2; }

template <int KL, bool UNIFORM>
__device__ __forceinline__ void hs_chunk(const float *const (&rp)[KL], const float (&ta)[KL], int n, int row,
                                         int klast, int jbase, int T, int lane, unsigned long long *raw,
                                         unsigned long long *counters, float (&best)[KL], int (&bestj)[KL]) {
    float v[jpt<KL>()][KL];
    int terms[jpt<KL>()];
#pragma unroll
    for (int u = 0; u < jpt<KL>(); ++u) terms[u] = UNIFORM ? T : min(term_count<KL>(jbase + 32 * u, n), klast);
    // Term l of fundamental jbase + 32 u sits at p[l] + 32 l u: one 64-bit address per term, then
    // constant offsets.
    const float *p[KL];
#pragma unroll
    for (int l = 1; l <= KL; ++l) p[l - 1] = rp[l - 1] + (size_t)l * (unsigned)jbase;
#pragma unroll
    for (int l = 1; l <= KL; ++l) {
        if (UNIFORM && l > T) break;  // warp-uniform
#pragma unroll
        for (int u = 0; u < jpt<KL>(); ++u) v[u][l - 1] = (UNIFORM || l <= terms[u]) ? __ldg(p[l - 1] + 32 * l * u) : 0.0f;
    }
    bool any_hit = false;
#pragma unroll
    for (int u = 0; u < jpt<KL>(); ++u) {
        const int j = jbase + 32 * u;
        float hp = 0.0f;
#pragma unroll
        for (int l = 1; l <= KL; ++l) {
            if (UNIFORM && l > T) break;
            hp = (l == 1) ? v[u][0] : __fadd_rn(hp, v[u][l - 1]);
            const bool ok = UNIFORM || l <= terms[u];
            const bool gt = ok && hp > best[l - 1];
            best[l - 1] = gt ? hp : best[l - 1];
            bestj[l - 1] = gt ? j : bestj[l - 1];
            any_hit |= ok && hp > ta[l - 1];
        }
    }
    if (__any_sync(0xFFFFFFFFu, any_hit)) {  // rare: recompute the same sums and compact the crossings
#pragma unroll
        for (int u = 0; u < jpt<KL>(); ++u) {
            const unsigned j = (unsigned)(jbase + 32 * u);
            float hp = 0.0f;
#pragma unroll
            for (int l = 1; l <= KL; ++l) {
                if (UNIFORM && l > T) break;  // warp-uniform; terms past T were not loaded
                hp = (l == 1) ? v[u][0] : __fadd_rn(hp, v[u][l - 1]);
                emit(l <= terms[u] && hp > ta[l - 1], hp, row, j, l, lane, counters, raw);
            }
        }
    }
}

// Row i takes part in klast <= KL planes: rows with fewer planes than the kernel was compiled for cap
// their term counts at klast (and never touch rows c + l i for l > klast).
template <int KL, int CH>
__device__ __forceinline__ void hs_row(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh,
                                       int n_temp, unsigned mask, int c, int i, int klast, int j0,
                                       unsigned long long *raw, unsigned long long *counters,
                                       unsigned long long *peaks) {
    const int row = c + i;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *rp[KL];
    float ta[KL];
#pragma unroll
    for (int l = 1; l <= KL; ++l) {
        rp[l - 1] = plane + (size_t)(l <= klast ? c + l * i : row) * ld;
        ta[l - 1] = (l <= klast && ((mask >> (l - 1)) & 1u)) ? __ldg(&thresh[(l - 1) * n_temp + row])
                                                           : __int_as_float(0x7f800000);
    }
    float best[KL];
    int bestj[KL];
#pragma unroll
    for (int l = 0; l < KL; ++l) {
        best[l] = -1.0f;
        bestj[l] = 0;
    }
    for (int ch = 0; ch < CH; ++ch) {
        const int jw = j0 + ch * (kHsThreads * jpt<KL>()) + warp * (32 * jpt<KL>());
        if (jw >= n) break;  // warp-uniform
        const int t_first = min(term_count<KL>(jw, n), klast);
        const int t_last = min(term_count<KL>(jw + 32 * jpt<KL>() - 1, n), klast);
        if (t_first == t_last)  // warp-uniform
            hs_chunk<KL, true>(rp, ta, n, row, klast, jw + lane, t_last, lane, raw, counters, best, bestj);
        else
            hs_chunk<KL, false>(rp, ta, n, row, klast, jw + lane, 0, lane, raw, counters, best, bestj);
    }
    unsigned long long key[KL];
#pragma unroll
    for (int l = 0; l < KL; ++l) key[l] = (l < klast) ? warp_peak_key(best[l], bestj[l], row) : 0ull;
    block_peaks<KL>(key, peaks);
}

// Row i of a group with klast planes: |i| runs over [lo, hi], both signs, and i = 0 when lo == 0.
__device__ __forceinline__ int group_row_offset(int y, int lo) {
    if (lo == 0) {
        if (y == 0) return 0;
        const int a = (y + 1) >> 1;  // 1, 1, 2, 2, ...
        return (y & 1) ? -a : a;
    }
    const int a = lo + (y >> 1);
    return (y & 1) ? a : -a;
}

// Row i of the group |i| <= hi (the rows with the most planes) in family order: first i = 0, then
// the positive rows and then the negative ones, each sign by families b, 2b, 4b, ... for odd b
// (1, 2, 4, 8, 3, 6, 5, 7 for hi = 8). Term l of row i reads plane row c + l i, so rows of one family
// read many of the same plane rows (rows 1, 2, 4 read 16 distinct rows, not 24); launched next to
// one another, they find more of those rows in L2.
__device__ __forceinline__ int family_row_offset(int y, int hi) {
    if (y == 0) return 0;
    const int sgn = y <= hi ? 1 : -1;
    int k = (y - 1) % hi;
    for (int b = 1; b <= hi; b += 2)
        for (int m = b; m <= hi; m *= 2) {
            if (k == 0) return sgn * m;
            --k;
        }
    return sgn * hi;
}

// One launch per group of rows sharing klast = min(n_harm, floor(c/|i|)) planes, so each kernel is
// compiled for exactly its number of terms. Grid: (column blocks of 1024 fundamentals, rows of the group).
__global__ void __launch_bounds__(kHsThreads, 4)
    fdas_hs_k1(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh, int n_temp,
               unsigned mask, int lo, unsigned long long *__restrict__ raw, unsigned long long *counters,
               unsigned long long *peaks) {
    const int c = (n_temp - 1) / 2;
    const int row = c + group_row_offset(blockIdx.y, lo);
    const float ta = (mask & 1u) ? __ldg(&thresh[row]) : __int_as_float(0x7f800000);
    const bool vec = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(plane) & 15) == 0;
    hs_row_k1(plane + (size_t)row * ld, n, ta, row, blockIdx.x * kK1Cols, raw, counters, peaks, vec);
}

// A group of rows with at least two planes, |i| in [lo, hi], in one launch compiled for KL terms;
// row i caps its terms at its own klast = min(n_harm, floor(c/|i|)) <= KL.
// Grid: (column blocks, rows of the group).
template <int KL>
__global__ void __launch_bounds__(kHsThreads, KL <= 3 ? 4 : 2)
    fdas_hs_kl(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh, int n_temp,
               unsigned mask, int n_harm, int lo, unsigned long long *__restrict__ raw, unsigned long long *counters,
               unsigned long long *peaks) {
    const int c = (n_temp - 1) / 2;
    const int i = lo == 0 ? family_row_offset(blockIdx.y, (int)(gridDim.y - 1) / 2) : group_row_offset(blockIdx.y, lo);
    const int ai = i < 0 ? -i : i;
    const int klast = ai == 0 ? n_harm : min(n_harm, c / ai);
    hs_row<KL, kChunksOne>(plane, n, ld, thresh, n_temp, mask, c, i, klast,
                           blockIdx.x * (kChunksOne * kHsThreads * jpt<KL>()), raw, counters, peaks);
}

// ---- highest-harmonic indexing (FDAS_INDEX_HIGHEST) ------------------------------------------------
// HP_k(i, j) = sum_{l=1..k} of P[c + rd(l i, k)][rd(l j, k)], float32 running sums in the order
// l = 1..k, rd = round half away from zero. A term depends on l/k only as a rational number, so the
// terms of all planes k <= K come from the reduced fractions q = a/b, b <= K (22 for K = 8, 80 for
// K = 16): term (l, k) of fundamental (i, j) is P[c + rd(a i, b)][rd(a j, b)] with a/b = l/k in
// lowest terms.
//
// A CTA takes one row i and W fundamental columns [j0, j0 + W). For each fraction it first copies
// the source columns [rd(a j0, b), rd(a (j0 + W - 1), b)] of row c + rd(a i, b) into its own
// shared-memory segment with coalesced 16-byte loads; then every plane is summed from the segments.
// Consecutive threads take consecutive columns, so they read the same or consecutive words of a
// segment (rd(a j, b) moves by a/b <= 1 per column) and the reads are free of bank conflicts.
//
//   fdas_hs_hh8   up to 8 planes. W = 1680 = 4 x 420, thread t < 420 takes j = j0 + t + 420 v, v < 4.
//                 Because 420 = lcm(1..7) and 1680 divides j0, rd(a j, b) = a j0 / b + rd(a t, b)
//                 + 420 a v / b exactly for b <= 7: one division per fraction and thread, then every
//                 term is a shared-memory load at a constant offset. For b = 8 the division is a shift.
//   fdas_hs_hh16  9 to 16 planes (80 fractions): W = 512, two columns per thread, one division per
//                 term.

// Greatest common divisor, and the reduced fractions a/b (1 <= a <= b) ordered by b, then a.
__host__ __device__ constexpr int gcd_c(int x, int y) {
    while (y != 0) {
        const int t = x % y;
        x = y;
        y = t;
    }
    return x;
}
__host__ __device__ constexpr int frac_count(int bmax) {
    int n = 0;
    for (int b = 1; b <= bmax; ++b)
        for (int a = 1; a <= b; ++a) n += gcd_c(a, b) == 1 ? 1 : 0;
    return n;
}
// Position of l/k (1 <= l <= k) in that order.
__host__ __device__ constexpr int frac_index(int l, int k) {
    const int g = gcd_c(l, k), a = l / g, b = k / g;
    int n = frac_count(b - 1);
    for (int x = 1; x < a; ++x) n += gcd_c(x, b) == 1 ? 1 : 0;
    return n;
}
// Fraction number q of that order: denominator and numerator.
__host__ __device__ constexpr int frac_b(int q) {
    int b = 1;
    while (frac_count(b) <= q) ++b;
    return b;
}
__host__ __device__ constexpr int frac_a(int q) {
    const int b = frac_b(q);
    int left = q - frac_count(b - 1), a = 0;
    while (left >= 0) {
        ++a;
        if (gcd_c(a, b) == 1) --left;
    }
    return a;
}
constexpr int kHhMaxFrac = 80;  // frac_count(16)
static_assert(frac_count(8) == 22 && frac_count(16) == kHhMaxFrac, "Farey counts");
static_assert(frac_a(0) == 1 && frac_b(0) == 1 && frac_a(3) == 2 && frac_b(3) == 3 && frac_a(21) == 7 &&
                  frac_b(21) == 8 && frac_index(6, 8) == 5 && frac_a(8) == 3 && frac_b(8) == 5 &&
                  frac_a(79) == 15 && frac_b(79) == 16,
              "fraction order");

// round(x / b) for x >= 0, b > 0, halves up (away from zero).
__host__ __device__ __forceinline__ int rd_pos(int x, int b) { return (2 * x + b) / (2 * b); }
// round(a / b) for b > 0, halves away from zero, exactly in integers.
__host__ __device__ __forceinline__ int round_div(int a, int b) {
    const int m = rd_pos(a < 0 ? -a : a, b);
    return a < 0 ? -m : m;
}

template <int L, int K>
struct HhTerm {
    static constexpr int q = frac_index(L, K), a = frac_a(q), b = frac_b(q);
};
// f(std::integral_constant<int, k>) for k = K..KMAX: loop bodies whose index must be a
// compile-time constant (term offsets, fraction numbers) whatever the size of the body.
template <int K, int KMAX, class F>
__device__ __forceinline__ void for_each_k(F &&f) {
    if constexpr (K <= KMAX) {
        f(std::integral_constant<int, K>{});
        for_each_k<K + 1, KMAX>(f);
    }
}
// The running sum of terms 1..L of plane K in the order l = 1..L; term(integral_constant<L>, K).
template <int K, int L, int V, class Term>
__device__ __forceinline__ float hh_sum(const Term &term) {
    const float x = term(std::integral_constant<int, L>{}, std::integral_constant<int, K>{},
                         std::integral_constant<int, V>{});
    if constexpr (L == 1)
        return x;
    else
        return __fadd_rn(hh_sum<K, L - 1, V>(term), x);
}

// Copies source columns [x0, x1] of one fraction (x0 on a 16-byte boundary when vec) into dst, the
// threads of the CTA each taking whole 16-byte groups (vec) or single floats.
__device__ __forceinline__ void hh_stage(float *dst, const float *src, int x0, int x1, bool vec, int tid,
                                         int nthreads) {
    if (vec) {
        const int nv = ((x1 - x0) >> 2) + 1;  // ends at or before the row's 16-byte boundary past x1
#pragma unroll 4
        for (int e = tid; e < nv; e += nthreads)
            reinterpret_cast<float4 *>(dst)[e] = __ldg(reinterpret_cast<const float4 *>(src) + e);
    } else {
        for (int e = tid; e <= x1 - x0; e += nthreads) dst[e] = __ldg(src + e);
    }
}

// The per-thread detection and peak bookkeeping shared by both kernels: hits bit (k - 1) + KMAX u.
template <int KMAX>
struct HhTrack {
    float best[KMAX];
    int bestj[KMAX];
    float ta[KMAX];
    unsigned hits = 0u;
};

template <int KMAX, int NW, int NV, class Term>
__device__ __forceinline__ void hh_finish(HhTrack<KMAX> &tr, const Term &term, int n_harm, int row, int lane,
                                          int jcol0, int jstep, unsigned long long *raw,
                                          unsigned long long *counters, unsigned long long *peaks) {
    // Crossings are rare: recompute the same sums for the planes where a lane of the warp crossed.
    for_each_k<1, KMAX>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if (k > n_harm) return;
        unsigned pm = 0u;
#pragma unroll
        for (int v = 0; v < NV; ++v) pm |= 1u << (k - 1 + KMAX * v);
        if (!__any_sync(0xFFFFFFFFu, (tr.hits & pm) != 0u)) return;
        for_each_k<0, NV - 1>([&](auto vc) {
            constexpr int v = decltype(vc)::value;
            const float hp = hh_sum<k, k, v>(term);
            emit(((tr.hits >> (k - 1 + KMAX * v)) & 1u) != 0u, hp, row, (unsigned)(jcol0 + jstep * v), k, lane,
                 counters, raw);
        });
    });
    __shared__ unsigned long long warp_key[NW][KMAX];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const unsigned long long key = (k < n_harm) ? warp_peak_key(tr.best[k], tr.bestj[k], row) : 0ull;
        if (lane == 0) warp_key[warp][k] = key;
    }
    __syncthreads();
    if (threadIdx.x < KMAX) {
        unsigned long long m = 0ull;
#pragma unroll
        for (int w = 0; w < NW; ++w) m = warp_key[w][threadIdx.x] > m ? warp_key[w][threadIdx.x] : m;
        if (m > *(volatile unsigned long long *)&peaks[threadIdx.x]) atomicMax(&peaks[threadIdx.x], m);
    }
}

// Plane sums of one column, then the thread's best point and crossings per plane.
template <int KMAX, int V, class Term>
__device__ __forceinline__ void hh_column(HhTrack<KMAX> &tr, const Term &term, int n_harm, bool ok, int j) {
    constexpr int v = V;
    for_each_k<1, KMAX>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if (k > n_harm) return;  // uniform
        const float hp = hh_sum<k, k, V>(term);
        const bool gt = ok && hp > tr.best[k - 1];
        tr.best[k - 1] = gt ? hp : tr.best[k - 1];
        tr.bestj[k - 1] = gt ? j : tr.bestj[k - 1];
        tr.hits |= (ok && hp > tr.ta[k - 1]) ? 1u << (k - 1 + KMAX * v) : 0u;
    });
}

template <int KMAX>
__device__ __forceinline__ void hh_track_init(HhTrack<KMAX> &tr, const float *__restrict__ thresh, int n_temp,
                                              unsigned mask, int n_harm, int row) {
#pragma unroll
    for (int k = 1; k <= KMAX; ++k) {
        tr.best[k - 1] = -1.0f;
        tr.bestj[k - 1] = 0;
        tr.ta[k - 1] = (k <= n_harm && ((mask >> (k - 1)) & 1u)) ? __ldg(&thresh[(k - 1) * n_temp + row])
                                                                 : __int_as_float(0x7f800000);
    }
}

// ---- up to 8 planes
constexpr int kHh8Step = 420;                  // lcm(1, ..., 7)
constexpr int kHh8V = 4;                       // columns per thread
constexpr int kHh8W = kHh8Step * kHh8V;        // 1680 columns per CTA
constexpr int kHh8Threads = 448;               // 14 warps; threads 420..447 only stage
constexpr int kHh8NQ = 22;
__host__ __device__ constexpr int hh8_seg(int q) {
    return ((frac_a(q) * kHh8W + frac_b(q) - 1) / frac_b(q) + 8 + 3) & ~3;
}
__host__ __device__ constexpr int hh8_off(int q) {
    int o = 0;
    for (int x = 0; x < q; ++x) o += hh8_seg(x);
    return o;
}
constexpr int kHh8SmemBytes = hh8_off(kHh8NQ) * 4;
static_assert(kHh8SmemBytes <= 100 * 1024, "two CTAs per SM");

// Fraction q's segment: source columns [x0, x1] of row c + rd(a i, b), x0 on a 16-byte boundary.
struct HhSpan {
    const float *src;
    int x0, x1;
};
__device__ __forceinline__ HhSpan hh_span(const float *plane, size_t ld, int c, int i, int j0, int jl, int a, int b) {
    const int x0 = rd_pos(a * j0, b) & ~3;
    return {plane + (size_t)(c + round_div(a * i, b)) * ld + x0, x0, rd_pos(a * jl, b)};
}

// Compile-time table of the 22 fractions' numerators, denominators and segment offsets.
struct Hh8Frac {
    unsigned char a[kHh8NQ], b[kHh8NQ];
    int off[kHh8NQ];
    __host__ __device__ constexpr Hh8Frac() : a{}, b{}, off{} {
        for (int q = 0; q < kHh8NQ; ++q) {
            a[q] = (unsigned char)frac_a(q);
            b[q] = (unsigned char)frac_b(q);
            off[q] = hh8_off(q);
        }
    }
};
__constant__ Hh8Frac c_hh8;

template <int Q>
__device__ __forceinline__ void hh8_divide(int (&r)[kHh8NQ], int t, int j0, int n_harm) {
    if constexpr (Q < kHh8NQ) {
        constexpr int a = frac_a(Q), b = frac_b(Q);
        if (b <= n_harm) {
            if constexpr (b <= 7)
                r[Q] = (int)((unsigned)(2 * a * t + b) / (unsigned)(2 * b));  // rd(a t, b)
            else
                r[Q] = hh8_off(Q) - (rd_pos(a * j0, b) & ~3);  // segment offset minus its first column
        }
        hh8_divide<Q + 1>(r, t, j0, n_harm);
    }
}

__global__ void __launch_bounds__(kHh8Threads, 2)
    fdas_hs_hh8(const float *__restrict__ plane, int n, size_t ld, bool vec, const float *__restrict__ thresh,
                int n_temp, unsigned mask, int n_harm, unsigned long long *__restrict__ raw,
                unsigned long long *counters, unsigned long long *peaks) {
    extern __shared__ float4 hh_seg4[];
    const float *const S = reinterpret_cast<const float *>(hh_seg4);
    const int c = (n_temp - 1) / 2;
    const int row = blockIdx.y, i = row - c;
    const int lane = threadIdx.x & 31;
    const int j0 = blockIdx.x * kHh8W;
    const int jl = min(j0 + kHh8W - 1, n - 1);
    // Staging: warp w copies fractions w and w + 14 (b <= n_harm), its lanes taking 16-byte groups.
    for (int q = threadIdx.x >> 5; q < kHh8NQ; q += kHh8Threads / 32) {
        const int b = c_hh8.b[q];
        if (b > n_harm) continue;  // warp-uniform
        const HhSpan sp = hh_span(plane, ld, c, i, j0, jl, c_hh8.a[q], b);
        hh_stage(reinterpret_cast<float *>(hh_seg4) + c_hh8.off[q], sp.src, sp.x0, sp.x1, vec, lane, 32);
    }
    HhTrack<8> tr;
    hh_track_init<8>(tr, thresh, n_temp, mask, n_harm, row);
    const bool act = threadIdx.x < kHh8Step;
    const int t = act ? threadIdx.x : 0;  // idle threads read inside the segments
    int r[kHh8NQ];
    hh8_divide<0>(r, t, j0, n_harm);
    __syncthreads();

    // Term (l, k) of column v: for b <= 7 one load at a constant offset from r[q]; for b = 8 a shift.
    auto term = [&](auto lc, auto kc, auto vc) -> float {
        using T = HhTerm<decltype(lc)::value, decltype(kc)::value>;
        constexpr int v = decltype(vc)::value;
        if constexpr (T::b <= 7)
            return S[r[T::q] + (hh8_off(T::q) + kHh8Step * T::a * v / T::b)];
        else
            return S[r[T::q] + ((2 * T::a * (j0 + t + kHh8Step * v) + 8) >> 4)];
    };
    auto columns = [&](auto full) {
        for_each_k<0, kHh8V - 1>([&](auto vc) {
            constexpr int v = decltype(vc)::value;
            const int j = j0 + t + kHh8Step * v;
            hh_column<8, v>(tr, term, n_harm, act && (decltype(full)::value || j < n), j);
        });
    };
    if (j0 + kHh8W <= n)
        columns(std::true_type{});
    else
        columns(std::false_type{});
    hh_finish<8, kHh8Threads / 32, kHh8V>(tr, term, n_harm, row, lane, j0 + t, kHh8Step, raw, counters, peaks);
}

// ---- 9 to 16 planes
constexpr int kHh16J = 2;
constexpr int kHh16W = kHsThreads * kHh16J;  // 512 columns per CTA
__host__ __device__ constexpr int hh16_seg(int q) {
    return ((frac_a(q) * kHh16W + frac_b(q) - 1) / frac_b(q) + 8 + 3) & ~3;
}
__host__ __device__ constexpr int hh16_off(int q) {
    int o = 0;
    for (int x = 0; x < q; ++x) o += hh16_seg(x);
    return o;
}

// Segment offsets and first columns per launch, for the fractions with b <= n_harm.
struct HhTable {
    int nq;
    int smem_floats;
    unsigned char a[kHhMaxFrac], b[kHhMaxFrac];
    int off[kHhMaxFrac];
};

HhTable hh16_table(int n_harm) {
    HhTable t{};
    for (int q = 0; q < kHhMaxFrac && frac_b(q) <= n_harm; ++q) {
        t.a[q] = (unsigned char)frac_a(q);
        t.b[q] = (unsigned char)frac_b(q);
        t.off[q] = hh16_off(q);
        t.nq = q + 1;
    }
    t.smem_floats = hh16_off(t.nq);
    return t;
}

__global__ void __launch_bounds__(kHsThreads)
    fdas_hs_hh16(const float *__restrict__ plane, int n, size_t ld, bool vec, const float *__restrict__ thresh,
                 int n_temp, unsigned mask, int n_harm, const __grid_constant__ HhTable tab,
                 unsigned long long *__restrict__ raw, unsigned long long *counters, unsigned long long *peaks) {
    extern __shared__ float4 hh_seg4[];
    const float *const S = reinterpret_cast<const float *>(hh_seg4);
    __shared__ int s_adj[kHhMaxFrac];  // segment offset minus the segment's first column
    const int c = (n_temp - 1) / 2;
    const int row = blockIdx.y, i = row - c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kHh16W;
    const int jl = min(j0 + kHh16W - 1, n - 1);
    // One warp per fraction, fractions dealt out round robin.
    for (int q = warp; q < tab.nq; q += kHsWarps) {
        const HhSpan sp = hh_span(plane, ld, c, i, j0, jl, tab.a[q], tab.b[q]);
        if (lane == 0) s_adj[q] = tab.off[q] - sp.x0;
        hh_stage(reinterpret_cast<float *>(hh_seg4) + tab.off[q], sp.src, sp.x0, sp.x1, vec, lane, 32);
    }
    HhTrack<16> tr;
    hh_track_init<16>(tr, thresh, n_temp, mask, n_harm, row);
    __syncthreads();
    const int jb = j0 + 32 * (kHh16J * warp) + lane;
    auto term = [&](auto lc, auto kc, auto vc) -> float {
        using T = HhTerm<decltype(lc)::value, decltype(kc)::value>;
        const int j = min(jb + 32 * decltype(vc)::value, jl);  // keeps the reads inside the staged columns
        return S[s_adj[T::q] + (int)((unsigned)(2 * T::a * j + T::b) / (unsigned)(2 * T::b))];
    };
    auto columns = [&](auto full) {
        for_each_k<0, kHh16J - 1>([&](auto vc) {
            constexpr int v = decltype(vc)::value;
            const int j = jb + 32 * v;
            hh_column<16, v>(tr, term, n_harm, decltype(full)::value || j < n, j);
        });
    };
    if (j0 + kHh16W <= n)
        columns(std::true_type{});
    else
        columns(std::false_type{});
    hh_finish<16, kHsWarps, kHh16J>(tr, term, n_harm, row, lane, jb, 32, raw, counters, peaks);
}

using HsKernel = void (*)(const float *, int, size_t, const float *, int, unsigned, int, int, unsigned long long *,
                          unsigned long long *, unsigned long long *);

// Compiled term counts, and the kernel for a group whose rows have at most kmax planes.
constexpr int kl_size(int kmax) { return kmax <= 2 ? 2 : kmax <= 4 ? 4 : kmax <= 8 ? 8 : 16; }
HsKernel hs_kernel(int kmax) {
    switch (kl_size(kmax)) {
        case 2: return fdas_hs_kl<2>;
        case 4: return fdas_hs_kl<4>;
        case 8: return fdas_hs_kl<8>;
        default: return fdas_hs_kl<16>;
    }
}
constexpr int kl_width(int kmax) {
    return kl_size(kmax) == 2 ? jpt<2>() : kl_size(kmax) == 4 ? jpt<4>() : kl_size(kmax) == 8 ? jpt<8>() : jpt<16>();
}

// Row groups of the harmonic sum for rows with at least two planes: [kmin, kmax] ranges of
// klast = min(n_harm, floor(c/|i|)), each launched once. Rows with few planes keep their own,
// smaller kernel (more resident warps); rows with many planes share one launch. Measured on the
// 2^21 workload against one merged launch, one launch per plane count, and {4..16, 2..3}, this
// partition was the fastest (0.428 ms against 0.462-0.464 ms).
struct Group {
    int kmin, kmax;
};
constexpr Group kGroups[] = {{5, 16}, {3, 4}, {2, 2}};

// |i| range of the rows whose klast lies in [kmin, kmax]; false if there is none.
bool group_rows(int c, int n_harm, int kmin, int kmax, int *lo, int *hi) {
    if (kmin > n_harm) return false;
    *lo = (kmax >= n_harm) ? 0 : c / (kmax + 1) + 1;
    *hi = c / kmin;
    return *hi >= *lo;
}

__device__ __forceinline__ fdas_cand decode_cand(unsigned long long key, int c, int k) {
    fdas_cand r;
    r.power = __uint_as_float(0xFFFFFFFFu - (unsigned)(key >> 32));
    r.i = (int16_t)((int)((key >> 24) & 0xFFu) - c);
    r.j = (unsigned)(key & 0xFFFFFFu);
    r.k = (uint8_t)k;
    r.pad = 0;
    return r;
}

// One bitonic step of stride S < E between a thread's own keys (index base + e).
template <int E, int S>
__device__ __forceinline__ void fin_reg_step(unsigned long long (&r)[E], int base, int size) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if ((e & S) != 0) continue;
        const bool up = ((base + e) & size) == 0;
        const unsigned long long a = r[e], b = r[e + S];
        const bool sw = (a > b) == up;
        r[e] = sw ? b : a;
        r[e + S] = sw ? a : b;
    }
}

// Ascending bitonic sort of the nr keys at src, padded with ~0 to np2 = 32 E 2^m >= nr, with E keys
// per thread: thread t holds keys [E t, E t + E) in registers. Strides below E are exchanges inside
// a thread, strides E..16 E warp shuffles, and only strides >= 32 E go through shared memory.
// The first nout keys are decoded to candidates of plane k.
template <int E>
__device__ __forceinline__ void fin_sort(const unsigned long long *__restrict__ src, int nr, int np2, int nout, int c,
                                         int k, int cand_cap, fdas_cand *cands, unsigned long long *keys) {
    const int nthr = np2 / E;  // active threads, whole warps
    const bool active = (int)threadIdx.x < nthr;
    const int base = (int)threadIdx.x * E;
    const int lane = threadIdx.x & 31;
    unsigned long long r[E];
    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e) r[e] = base + e < nr ? src[base + e] : ~0ull;
    }
    for (int size = 2; size <= np2; size <<= 1) {
        if ((size >> 1) >= 32 * E) {
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) keys[base + e] = r[e];
            }
            __syncthreads();
            for (int stride = size >> 1; stride >= 32 * E; stride >>= 1) {
                for (int x = threadIdx.x; x < (np2 >> 1); x += blockDim.x) {
                    const int lo = 2 * x - (x & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long a = keys[lo], b = keys[hi];
                    if ((a > b) == up) {
                        keys[lo] = b;
                        keys[hi] = a;
                    }
                }
                __syncthreads();
            }
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) r[e] = keys[base + e];
            }
            __syncthreads();  // every read done before the next writes
        }
        if (active) {
            for (int stride = min(size >> 1, 16 * E); stride >= E; stride >>= 1) {
                const int lx = stride / E;            // partner lane distance
                const bool lower = (lane & lx) == 0;  // this thread holds the lower index of each pair
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, r[e], lx);
                    const bool up = ((base + e) & size) == 0;
                    r[e] = (lower == up) ? (r[e] < o ? r[e] : o) : (r[e] > o ? r[e] : o);
                }
            }
            if (E > 8 && size >= 16) fin_reg_step<E, (E > 8 ? 8 : 0)>(r, base, size);
            if (E > 4 && size >= 8) fin_reg_step<E, (E > 4 ? 4 : 0)>(r, base, size);
            if (E > 2 && size >= 4) fin_reg_step<E, (E > 2 ? 2 : 0)>(r, base, size);
            fin_reg_step<E, 1>(r, base, size);
        }
    }
    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (base + e < nout) cands[(size_t)(k - 1) * cand_cap + base + e] = decode_cand(r[e], c, k);
    }
}

// Counts, peak and the top cand_cap candidates of plane k, from its workspace.
__device__ __forceinline__ void finalize_plane(int k, const unsigned long long *__restrict__ raw,
                                               const unsigned long long *counters, const unsigned long long *peaks,
                                               int n_temp, int cand_cap, fdas_cand *cands, uint32_t *counts,
                                               fdas_cand *peak_out, unsigned long long *keys) {
    const int c = (n_temp - 1) / 2;
    const unsigned long long total = counters[k - 1];
    const int nr = (int)(total < FDAS_RAW_CAP ? total : FDAS_RAW_CAP);
    if (threadIdx.x == 0) {
        counts[k - 1] = (uint32_t)(total < 0xFFFFFFFFull ? total : 0xFFFFFFFFull);
        if (peak_out) {
            const unsigned long long pk = peaks[k - 1];
            fdas_cand r;
            r.power = __uint_as_float((unsigned)(pk >> 32));
            const unsigned loc = 0xFFFFFFFFu - (unsigned)(pk & 0xFFFFFFFFull);
            r.i = (int16_t)((int)(loc >> 24) - c);
            r.j = loc & 0xFFFFFFu;
            r.k = (uint8_t)k;
            r.pad = 0;
            peak_out[k - 1] = r;
        }
    }
    if (nr == 0) return;
    const int nout = nr < cand_cap ? nr : cand_cap;
    const unsigned long long *src = raw + (size_t)(k - 1) * FDAS_RAW_CAP;
    // Keys per thread: 2 up to 2048 keys, 4 up to 4096, 16 up to FDAS_RAW_CAP (1024 threads).
    int np2 = 64;
    while (np2 < nr) np2 <<= 1;
    if (np2 <= 2048)
        fin_sort<2>(src, nr, np2, nout, c, k, cand_cap, cands, keys);
    else if (np2 <= 4096)
        fin_sort<4>(src, nr, np2, nout, c, k, cand_cap, cands, keys);
    else
        fin_sort<16>(src, nr, np2, nout, c, k, cand_cap, cands, keys);
}

__global__ void __launch_bounds__(kFinThreads)
    fdas_hs_finalize(const unsigned long long *__restrict__ raw, const unsigned long long *counters,
                     const unsigned long long *peaks, int n_temp, int cand_cap, fdas_cand *cands, uint32_t *counts,
                     fdas_cand *peak_out) {
    extern __shared__ unsigned long long keys[];
    finalize_plane(blockIdx.x + 1, raw, counters, peaks, n_temp, cand_cap, cands, counts, peak_out, keys);
}

// ---- batched forms: one launch per stage for every spectrum of a batch ----------------------------

// Spectrum of CTA x in a launch of W columns per CTA: the last job whose first CTA in such launches
// (blk2 for 16384 columns, blk0 for 12288, blk1 for 4096) is <= x.
template <int W>
__device__ __forceinline__ int first_block(const HsJob &J) {
    return W == 16384 ? J.blk2 : W == 12288 ? J.blk0 : J.blk1;
}
template <int W>
__device__ __forceinline__ int job_of_block(const HsBatch &B, int x) {
    int lo = 0, hi = B.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int first = first_block<W>(B.job[mid]);
        if (first <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void fdas_hs_reset_batch(const HsBatch B, int n_harm) {
    const HsJob &J = B.job[blockIdx.x];
    const int t = threadIdx.x;
    if (t < n_harm) {
        J.counters[t] = 0ull;
        J.peaks[t] = 0ull;
    }
}

__global__ void __launch_bounds__(kHsThreads, 4)
    fdas_hs_k1_batch(const HsBatch B, const float *__restrict__ thresh, int n_temp, unsigned mask, int lo) {
    const HsJob &J = B.job[job_of_block<kK1Cols>(B, blockIdx.x)];
    const int c = (n_temp - 1) / 2;
    const int row = c + group_row_offset(blockIdx.y, lo);
    const float ta = (mask & 1u) ? __ldg(&thresh[row]) : __int_as_float(0x7f800000);
    const bool vec = (J.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(J.plane) & 15) == 0;
    hs_row_k1(J.plane + (size_t)row * J.ld, J.n, ta, row, (blockIdx.x - J.blk1) * kK1Cols, J.raw, J.counters, J.peaks,
              vec);
}

// CTA widths: 16384 columns (kernels for up to 4 terms), 12288 (up to 8) or 4096 (16 terms, and the
// single-plane rows). HsJob.blk2 / blk0 / blk1 are the spectrum's first CTA in launches of each width.
template <int KL>
__global__ void __launch_bounds__(kHsThreads, KL <= 3 ? 4 : 2)
    fdas_hs_kl_batch(const HsBatch B, const float *__restrict__ thresh, int n_temp, unsigned mask, int n_harm, int lo) {
    constexpr int W = kChunks * kHsThreads * jpt<KL>();
    const HsJob &J = B.job[job_of_block<W>(B, blockIdx.x)];
    const int c = (n_temp - 1) / 2;
    const int i = group_row_offset(blockIdx.y, lo);
    const int ai = i < 0 ? -i : i;
    const int klast = ai == 0 ? n_harm : min(n_harm, c / ai);
    hs_row<KL, kChunks>(J.plane, J.n, (size_t)J.ld, thresh, n_temp, mask, c, i, klast,
               (blockIdx.x - first_block<W>(J)) * W, J.raw, J.counters,
               J.peaks);
}

__global__ void __launch_bounds__(kFinThreads) fdas_hs_finalize_batch(const HsBatch B, int n_temp, int cand_cap) {
    extern __shared__ unsigned long long keys[];
    const HsJob &J = B.job[blockIdx.y];
    finalize_plane(blockIdx.x + 1, J.raw, J.counters, J.peaks, n_temp, cand_cap, J.cands, J.counts, J.peak_out, keys);
}

using HsBatchKernel = void (*)(const HsBatch, const float *, int, unsigned, int, int);

HsBatchKernel hs_batch_kernel(int kmax) {
    switch (kl_size(kmax)) {
        case 2: return fdas_hs_kl_batch<2>;
        case 4: return fdas_hs_kl_batch<4>;
        case 8: return fdas_hs_kl_batch<8>;
        default: return fdas_hs_kl_batch<16>;
    }
}

}  // namespace

cudaError_t launch_hs_reset(const fdas_params &p, const HsWorkspace &ws, cudaStream_t s) {
    fdas_hs_reset<<<1, 32, 0, s>>>(ws.counters, ws.peaks, p.n_harm);
    return cudaGetLastError();
}

// Auxiliary streams for the concurrent row-group launches, with the fork and join events of a call,
// kept per host thread and CUDA context:
//   - calls from different threads never share a stream or an event, so a graph capture in one
//     thread cannot pick up another thread's kernels;
//   - the calls of one thread share one set whatever their caller streams, so the row-group launches
//     of successive spectra queue behind one another. Measured with two streams of spectra of 2^21
//     bins, that was faster than one set per caller stream (1378 against 1269 spectra/s), and the
//     request loop's p99 latency at 1000 arrivals/s was lower (15.3 against 16.9 ms);
//   - a set whose streams are part of a capture in progress serves only calls on a stream of that same
//     capture; any other call takes another set (made for it if needed), so eager work never lands in
//     a graph being captured;
//   - a set made for a context that was destroyed (cudaDeviceReset) is never used again: each set
//     holds the driver's context id, which is unique for the life of the process.
// Sets are never created while the caller's stream is being captured: such a call runs its launches on
// the caller's stream alone (same results, no overlap) if no set of that capture exists. A thread keeps
// at most kAuxSets sets; streams and events are kept until the process exits.
constexpr int kAuxSets = 8;
struct AuxSet {
    unsigned long long ctx;   // driver context id
    unsigned long long used;  // last use, in this thread's call count
    cudaStream_t st[2];
    cudaEvent_t ev[3];
};

// Capture state of s: 0 not capturing, 1 capturing (with *id), -1 unknown (the query failed: for
// instance on the legacy stream while a blocking stream is captured; the error is cleared).
int capture_state(cudaStream_t s, unsigned long long *id) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    *id = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, id) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return cs == cudaStreamCaptureStatusNone ? 0 : 1;
}

cudaError_t make_aux(AuxSet &a) {
    a.st[0] = a.st[1] = nullptr;
    a.ev[0] = a.ev[1] = a.ev[2] = nullptr;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&a.st[k], cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&a.ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (int k = 0; k < 2; ++k)
            if (a.st[k]) cudaStreamDestroy(a.st[k]);
        for (int k = 0; k < 3; ++k)
            if (a.ev[k]) cudaEventDestroy(a.ev[k]);
        a.st[0] = nullptr;
    }
    return e;
}

// The calling thread's set for a call on stream s in the current context, or *out = nullptr when the
// launches must stay on s.
cudaError_t aux_set(cudaStream_t s, AuxSet **out) {
    thread_local AuxSet sets[kAuxSets];
    thread_local unsigned long long calls = 0;
    *out = nullptr;
    unsigned long long ctx = 0;
    cudaError_t e = FDAS_NOTE(current_context_id(&ctx));
    if (e != cudaSuccess) return e;
    unsigned long long sid = 0;
    const int scap = capture_state(s, &sid);
    if (scap < 0) return cudaSuccess;  // unknown: stay on s
    ++calls;
    AuxSet *pick = nullptr, *empty = nullptr, *other = nullptr;
    for (AuxSet &a : sets) {
        if (a.st[0] == nullptr) {
            if (!empty) empty = &a;
            continue;
        }
        if (a.ctx != ctx) {
            if (!other) other = &a;
            continue;
        }
        unsigned long long aid = 0;
        const int acap = capture_state(a.st[0], &aid);
        const bool usable = acap == 0 || (acap == 1 && scap == 1 && aid == sid);
        if (usable && (!pick || a.used > pick->used)) pick = &a;  // the most recently used one
    }
    if (!pick) {
        if (scap != 0) return cudaSuccess;  // create nothing inside a capture
        pick = empty ? empty : other;       // a set of another context is forgotten, not touched
        if (!pick) return cudaSuccess;      // every set is held by captures: stay on s
        e = FDAS_NOTE(make_aux(*pick));
        if (e != cudaSuccess) return e;
        pick->ctx = ctx;
    }
    pick->used = calls;
    *out = pick;
    return cudaSuccess;
}

// Enqueues launch(k, stream) for k < count. The launches must be independent of one another. With
// concurrent (and two or more launches) they run side by side: k = 0 on s, k = 1 and 3 on the first
// auxiliary stream, k = 2 on the second, forked from s and joined back into it by events, so that
// one launch's tail overlaps the others' work. Work enqueued on s afterwards waits for all of them.
// Each call records and waits on its set's events before it returns, so no other call sees them
// half-way.
template <class F>
cudaError_t side_by_side(cudaStream_t s, int count, bool concurrent, F &&launch) {
    AuxSet *aux = nullptr;
    cudaError_t e = cudaSuccess;
    if (concurrent && count >= 2) e = aux_set(s, &aux);
    if (e != cudaSuccess) return e;
    const bool fork = aux != nullptr;
    cudaStream_t st[3] = {s, s, s};
    if (fork) {
        st[1] = aux->st[0];
        st[2] = aux->st[1];
        e = FDAS_NOTE(cudaEventRecord(aux->ev[0], s));
        if (e == cudaSuccess) e = FDAS_NOTE(cudaStreamWaitEvent(st[1], aux->ev[0], 0));
        if (e == cudaSuccess) e = FDAS_NOTE(cudaStreamWaitEvent(st[2], aux->ev[0], 0));
    }
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        launch(k, fork ? st[k == 0 ? 0 : (k & 1) ? 1 : 2] : s);
        e = FDAS_NOTE(cudaGetLastError());
    }
    if (fork) {
        if (e == cudaSuccess) e = FDAS_NOTE(cudaEventRecord(aux->ev[1], st[1]));
        if (e == cudaSuccess) e = FDAS_NOTE(cudaEventRecord(aux->ev[2], st[2]));
        if (e == cudaSuccess) e = FDAS_NOTE(cudaStreamWaitEvent(s, aux->ev[1], 0));
        if (e == cudaSuccess) e = FDAS_NOTE(cudaStreamWaitEvent(s, aux->ev[2], 0));
    }
    return e;
}

cudaError_t launch_harmonic(const fdas_params &p, const float *plane, size_t n, size_t ld, const float *thresh,
                            fdas_cand *cands, uint32_t *counts, fdas_cand *peaks, const HsWorkspace &ws,
                            cudaStream_t s, bool hp1_done, bool concurrent) {
    // hp1_done: the workspace was reset before the convolution, which also took the HP_1 candidates
    // and peak of the single-plane rows; no single-plane launch runs then.
    cudaError_t e = cudaSuccess;
    if (!hp1_done) {
        e = launch_hs_reset(p, ws, s);
        if (e != cudaSuccess) return e;
    }
    const unsigned mask = p.harm_mask;
    if (p.harm_index == FDAS_INDEX_HIGHEST) {
        const bool vec = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(plane) & 15) == 0;
        if (p.n_harm <= 8) {
            const dim3 grid((unsigned)((n + kHh8W - 1) / kHh8W), (unsigned)p.n_temp);
            e = cudaFuncSetAttribute(fdas_hs_hh8, cudaFuncAttributeMaxDynamicSharedMemorySize, kHh8SmemBytes);
            if (e != cudaSuccess) return e;
            fdas_hs_hh8<<<grid, kHh8Threads, kHh8SmemBytes, s>>>(plane, (int)n, ld, vec, thresh, p.n_temp, mask,
                                                                 p.n_harm, ws.raw, ws.counters, ws.peaks);
        } else {
            const HhTable tab = hh16_table(p.n_harm);
            const int smem_hh = tab.smem_floats * (int)sizeof(float);
            const dim3 grid((unsigned)((n + kHh16W - 1) / kHh16W), (unsigned)p.n_temp);
            e = cudaFuncSetAttribute(fdas_hs_hh16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_hh);
            if (e != cudaSuccess) return e;
            fdas_hs_hh16<<<grid, kHsThreads, smem_hh, s>>>(plane, (int)n, ld, vec, thresh, p.n_temp, mask, p.n_harm,
                                                           tab, ws.raw, ws.counters, ws.peaks);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int smem = FDAS_RAW_CAP * (int)sizeof(unsigned long long);
        e = cudaFuncSetAttribute(fdas_hs_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        fdas_hs_finalize<<<p.n_harm, kFinThreads, smem, s>>>(ws.raw, ws.counters, ws.peaks, p.n_temp, p.cand_cap,
                                                              cands, counts, peaks);
        return cudaGetLastError();
    }
    // Rows with at least two planes in a few launches (kGroups), then the single-plane rows
    // (|i| > c/2; every row when n_harm = 1) streamed by fdas_hs_k1.
    const int c = (p.n_temp - 1) / 2;
    const int lo1 = p.n_harm >= 2 ? c / 2 + 1 : 0;
    struct Launch {
        HsKernel kernel;  // nullptr: fdas_hs_k1
        dim3 grid;
        int lo;
    };
    Launch L[4];
    int nl = 0;
    for (const Group &gr : kGroups) {
        int lo, hi;
        if (!group_rows(c, p.n_harm, gr.kmin, gr.kmax, &lo, &hi)) continue;
        const int kmax = gr.kmax < p.n_harm ? gr.kmax : p.n_harm;
        const int per = kChunksOne * kHsThreads * kl_width(kmax);
        const int rows = (lo == 0) ? 2 * hi + 1 : 2 * (hi - lo + 1);
        L[nl++] = {hs_kernel(kmax), dim3((unsigned)((n + per - 1) / per), (unsigned)rows), lo};
    }
    const int rows1 = lo1 == 0 ? 2 * c + 1 : 2 * (c - lo1 + 1);
    if (rows1 > 0 && !hp1_done)
        L[nl++] = {nullptr, dim3((unsigned)((n + kK1Cols - 1) / kK1Cols), (unsigned)rows1), lo1};
    // The launches are independent: they only add to the workspace's counters, keys and peak keys
    // atomically. The largest (the first group) stays on the caller's stream.
    e = side_by_side(s, nl, concurrent, [&](int k, cudaStream_t sk) {
        if (L[k].kernel)
            L[k].kernel<<<L[k].grid, kHsThreads, 0, sk>>>(plane, (int)n, ld, thresh, p.n_temp, mask, p.n_harm, L[k].lo,
                                                          ws.raw, ws.counters, ws.peaks);
        else
            fdas_hs_k1<<<L[k].grid, kHsThreads, 0, sk>>>(plane, (int)n, ld, thresh, p.n_temp, p.harm_mask, L[k].lo,
                                                         ws.raw, ws.counters, ws.peaks);
    });
    if (e != cudaSuccess) return e;
    const int smem = FDAS_RAW_CAP * (int)sizeof(unsigned long long);
    e = cudaFuncSetAttribute(fdas_hs_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fdas_hs_finalize<<<p.n_harm, kFinThreads, smem, s>>>(ws.raw, ws.counters, ws.peaks, p.n_temp, p.cand_cap, cands,
                                                          counts, peaks);
    return cudaGetLastError();
}

// CTAs of one spectrum of n bins in launches of 16384, 12288 and 4096 columns per CTA (rows with up
// to 4, up to 8 and 16 planes; the single-plane rows use 4096 too).
void harmonic_blocks(const fdas_params &p, size_t n, int *blocks_16k, int *blocks_12k, int *blocks_4k) {
    (void)p;
    static_assert(kChunks * kHsThreads * jpt<2>() == 16384 && kChunks * kHsThreads * jpt<4>() == 16384,
                  "rows with up to 4 planes: 16384 columns per CTA");
    static_assert(kChunks * kHsThreads * jpt<8>() == 12288, "rows with up to 8 planes: 12288 columns per CTA");
    static_assert(kChunks * kHsThreads * jpt<16>() == kK1Cols, "16 planes and single-plane rows: 4096 columns");
    *blocks_16k = (int)((n + 16383) / 16384);
    *blocks_12k = (int)((n + 12287) / 12288);
    *blocks_4k = (int)((n + kK1Cols - 1) / kK1Cols);
}

cudaError_t prepare_streams(cudaStream_t s) {
    AuxSet *aux = nullptr;
    return aux_set(s, &aux);
}

cudaError_t prepare_harmonic_batch() {
    return cudaFuncSetAttribute(fdas_hs_finalize_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                FDAS_RAW_CAP * (int)sizeof(unsigned long long));
}

cudaError_t launch_hs_reset_batch(const fdas_params &p, const HsBatch &B, cudaStream_t s) {
    fdas_hs_reset_batch<<<B.count, 32, 0, s>>>(B, p.n_harm);
    return cudaGetLastError();
}

cudaError_t launch_harmonic_batch(const fdas_params &p, const HsBatch &B, int total_16k, int total_12k, int total_4k,
                                  const float *thresh, cudaStream_t s, bool hp1_done) {
    cudaError_t e = cudaSuccess;
    if (!hp1_done) {
        e = launch_hs_reset_batch(p, B, s);
        if (e != cudaSuccess) return e;
    }
    const int c = (p.n_temp - 1) / 2;
    const int lo1 = p.n_harm >= 2 ? c / 2 + 1 : 0;
    struct Launch {
        HsBatchKernel kernel;  // nullptr: fdas_hs_k1_batch
        dim3 grid;
        int lo;
    };
    Launch L[4];
    int nl = 0;
    for (const Group &gr : kGroups) {
        int lo, hi;
        if (!group_rows(c, p.n_harm, gr.kmin, gr.kmax, &lo, &hi)) continue;
        const int kmax = gr.kmax < p.n_harm ? gr.kmax : p.n_harm;
        const int rows = (lo == 0) ? 2 * hi + 1 : 2 * (hi - lo + 1);
        const int w = kChunks * kHsThreads * kl_width(kmax);
        const unsigned gx = (unsigned)(w == 16384 ? total_16k : w == 12288 ? total_12k : total_4k);
        L[nl++] = {hs_batch_kernel(kmax), dim3(gx, (unsigned)rows), lo};
    }
    const int rows1 = lo1 == 0 ? 2 * c + 1 : 2 * (c - lo1 + 1);
    if (rows1 > 0 && !hp1_done) L[nl++] = {nullptr, dim3((unsigned)total_4k, (unsigned)rows1), lo1};
    // Independent launches, side by side (inside a graph capture the stream's auxiliary streams join
    // it, if they were made before the capture began).
    e = side_by_side(s, nl, true, [&](int k, cudaStream_t sk) {
        if (L[k].kernel)
            L[k].kernel<<<L[k].grid, kHsThreads, 0, sk>>>(B, thresh, p.n_temp, p.harm_mask, p.n_harm, L[k].lo);
        else
            fdas_hs_k1_batch<<<L[k].grid, kHsThreads, 0, sk>>>(B, thresh, p.n_temp, p.harm_mask, L[k].lo);
    });
    if (e != cudaSuccess) return e;
    fdas_hs_finalize_batch<<<dim3((unsigned)p.n_harm, (unsigned)B.count), kFinThreads,
                             FDAS_RAW_CAP * sizeof(unsigned long long), s>>>(B, p.n_temp, p.cand_cap);
    return cudaGetLastError();
}

}  // namespace fdas
