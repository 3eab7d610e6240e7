// Harmonic summing with threshold detection (Sec. 2.2, Algorithm 1).
//
// Stretch read by fundamental: HP_k(i, j) = sum_{l=1..k} P[c + l*i][l*j] on
// D_k = {|k*i| <= c, k*j <= n-1}, summed in float32 in the order l = 1, 2, ..., k. As in the
// paper's MultipleHP kernels, all planes are computed at once and no HP plane is stored: one
// thread owns one fundamental (i, j) and keeps the running sum in a register.
//
// GB300 mapping:
//   fdas_hs_reset    zeroes the per-plane crossing counters and peak keys in the workspace.
//   fdas_hs_k1/kl<K> one launch per group of rows that take part in the same number K of planes
//                    (K = min(n_harm, floor(c/|i|))), each compiled for exactly K terms; grid
//                    (column blocks, rows of the group). Rows with one plane stream 16-byte loads,
//                    4096 columns per CTA. The others take 8 chunks of 1024 columns per CTA; in each
//                    chunk a thread issues every strided gather P[c + l i][l j] of its 4
//                    fundamentals before summing, through the read-only path, and warps whose
//                    columns all have the same number of terms skip the per-element domain test. Crossings are rare and take a separate path: a ballot, one
//                    atomicAdd per warp, and a prefix popcount for each lane's slot. Each candidate
//                    is one 64-bit key whose ascending order is the canonical order (power desc,
//                    i asc, j asc). The loudest point of every plane comes from warp reductions
//                    (redux max of the power bits, then redux min of the column), a block merge in
//                    shared memory, and at most one 64-bit atomicMax per block and plane.
//   fdas_hs_finalize one CTA per plane. It bitonic-sorts the raw keys in shared memory, then decodes
//                    the top cand_cap keys into fdas_cand records and writes the counts and peaks.
#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kHsThreads = 256;
constexpr int kFinThreads = 1024;

// Candidate key, ascending = canonical order (power desc, then row i asc, then column j asc).
__device__ __forceinline__ unsigned long long cand_key(float power, int row, unsigned j) {
    const unsigned pb = __float_as_uint(power);  // power >= 0, so the bits order like the values
    return ((unsigned long long)(0xFFFFFFFFu - pb) << 32) | ((unsigned long long)row << 24) | j;
}
// Peak key, descending = canonical order.
__device__ __forceinline__ unsigned long long peak_key(float power, int row, unsigned j) {
    const unsigned pb = __float_as_uint(power);
    return ((unsigned long long)pb << 32) | (0xFFFFFFFFu - (((unsigned)row << 24) | j));
}

__global__ void fdas_hs_reset(unsigned long long *counters, unsigned long long *peaks, int n_harm) {
    const int t = threadIdx.x;
    if (t < n_harm) {
        counters[t] = 0ull;
        peaks[t] = 0ull;
    }
}

constexpr int kHsWarps = kHsThreads / 32;

// Warp-wide candidate compaction: one ballot, one atomicAdd per warp, a prefix popcount per lane.
__device__ __forceinline__ void emit(bool hit, float hp, int row, unsigned j, int plane_k, int lane,
                                     unsigned long long *counters, unsigned long long *raw) {
    const unsigned ballot = __ballot_sync(0xFFFFFFFFu, hit);
    if (!ballot) return;
    const int leader = __ffs(ballot) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&counters[plane_k - 1], (unsigned long long)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (hit) {
        const unsigned long long slot = base + __popc(ballot & ((1u << lane) - 1u));
        if (slot < FDAS_RAW_CAP) raw[(size_t)(plane_k - 1) * FDAS_RAW_CAP + slot] = cand_key(hp, row, j);
    }
}

// The loudest point of plane k over a warp: redux max of the power bits (non-negative floats order
// like their bits), then redux min of the column among the lanes that hold that power.
__device__ __forceinline__ unsigned long long warp_peak_key(float best, int bestj, int row) {
    const unsigned pb = best >= 0.0f ? __float_as_uint(best) : 0u;
    const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, pb);
    const unsigned jmin = __reduce_min_sync(0xFFFFFFFFu, (best >= 0.0f && pb == mx) ? (unsigned)bestj : 0xFFFFFFFFu);
    if (jmin == 0xFFFFFFFFu) return 0ull;
    return peak_key(__uint_as_float(mx), row, jmin);
}

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

// Rows with KL >= 2 planes. A CTA covers kChunks chunks of 256 J fundamental columns (J = jpt<KL>()); in a
// chunk, lane L of warp w handles j = jc + 32 J w + L + 32 u, u < J, so every gather of a warp is one coalesced stride-l
// access along a plane row. The per-plane best points accumulate over the chunks, and the peak
// reductions, the block merge and the atomics run once per CTA. UNIFORM: every fundamental of the
// warp's chunk has the same number T of terms, which holds for all warps but those straddling a
// boundary j = (n-1)/l.
constexpr int kChunks = 8;
// Fundamentals per thread and chunk: fewer for many planes, to keep the gathers in registers.
template <int KL>
__host__ __device__ constexpr int jpt() { return KL <= 9 ? 4 : 2; }

template <int KL, bool UNIFORM>
__device__ __forceinline__ void hs_chunk(const float *const (&rp)[KL], const float (&ta)[KL], int n, int row,
                                         int jbase, int T, int lane, unsigned long long *raw,
                                         unsigned long long *counters, float (&best)[KL], int (&bestj)[KL]) {
    float v[jpt<KL>()][KL];
    int terms[jpt<KL>()];
#pragma unroll
    for (int u = 0; u < jpt<KL>(); ++u) terms[u] = UNIFORM ? T : term_count<KL>(jbase + 32 * u, n);
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

template <int KL>
__device__ __forceinline__ void hs_row(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh,
                                       int n_temp, unsigned mask, int c, int i, int j0, unsigned long long *raw,
                                       unsigned long long *counters, unsigned long long *peaks) {
    const int row = c + i;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *rp[KL];
    float ta[KL];
#pragma unroll
    for (int l = 1; l <= KL; ++l) {
        rp[l - 1] = plane + (size_t)(c + l * i) * ld;
        ta[l - 1] = ((mask >> (l - 1)) & 1u) ? __ldg(&thresh[(l - 1) * n_temp + row]) : __int_as_float(0x7f800000);
    }
    float best[KL];
    int bestj[KL];
#pragma unroll
    for (int l = 0; l < KL; ++l) {
        best[l] = -1.0f;
        bestj[l] = 0;
    }
    for (int ch = 0; ch < kChunks; ++ch) {
        const int jw = j0 + ch * (kHsThreads * jpt<KL>()) + warp * (32 * jpt<KL>());
        if (jw >= n) break;  // warp-uniform
        const int t_first = term_count<KL>(jw, n), t_last = term_count<KL>(jw + 32 * jpt<KL>() - 1, n);
        if (t_first == t_last)  // warp-uniform
            hs_chunk<KL, true>(rp, ta, n, row, jw + lane, t_last, lane, raw, counters, best, bestj);
        else
            hs_chunk<KL, false>(rp, ta, n, row, jw + lane, 0, lane, raw, counters, best, bestj);
    }
    unsigned long long key[KL];
#pragma unroll
    for (int l = 0; l < KL; ++l) key[l] = warp_peak_key(best[l], bestj[l], row);
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

template <int KL>
__global__ void __launch_bounds__(kHsThreads, KL <= 3 ? 4 : 2)
    fdas_hs_kl(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh, int n_temp,
               unsigned mask, int lo, unsigned long long *__restrict__ raw, unsigned long long *counters,
               unsigned long long *peaks) {
    const int c = (n_temp - 1) / 2;
    hs_row<KL>(plane, n, ld, thresh, n_temp, mask, c, group_row_offset(blockIdx.y, lo),
               blockIdx.x * (kChunks * kHsThreads * jpt<KL>()), raw, counters, peaks);
}

using HsKernel = void (*)(const float *, int, size_t, const float *, int, unsigned, int, unsigned long long *,
                          unsigned long long *, unsigned long long *);

HsKernel hs_kernel(int klast) {
    switch (klast) {
        case 1: return fdas_hs_k1;
        case 2: return fdas_hs_kl<2>;
        case 3: return fdas_hs_kl<3>;
        case 4: return fdas_hs_kl<4>;
        case 5: return fdas_hs_kl<5>;
        case 6: return fdas_hs_kl<6>;
        case 7: return fdas_hs_kl<7>;
        case 8: return fdas_hs_kl<8>;
        case 9: return fdas_hs_kl<9>;
        case 10: return fdas_hs_kl<10>;
        case 11: return fdas_hs_kl<11>;
        case 12: return fdas_hs_kl<12>;
        case 13: return fdas_hs_kl<13>;
        case 14: return fdas_hs_kl<14>;
        case 15: return fdas_hs_kl<15>;
        default: return fdas_hs_kl<16>;
    }
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
    int np2 = 1;
    while (np2 < nr) np2 <<= 1;
    const unsigned long long *src = raw + (size_t)(k - 1) * FDAS_RAW_CAP;
    for (int x = threadIdx.x; x < np2; x += blockDim.x) keys[x] = x < nr ? src[x] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
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
    }
    const int nout = nr < cand_cap ? nr : cand_cap;
    for (int x = threadIdx.x; x < nout; x += blockDim.x) cands[(size_t)(k - 1) * cand_cap + x] = decode_cand(keys[x], c, k);
}

__global__ void __launch_bounds__(kFinThreads)
    fdas_hs_finalize(const unsigned long long *__restrict__ raw, const unsigned long long *counters,
                     const unsigned long long *peaks, int n_temp, int cand_cap, fdas_cand *cands, uint32_t *counts,
                     fdas_cand *peak_out) {
    extern __shared__ unsigned long long keys[];
    finalize_plane(blockIdx.x + 1, raw, counters, peaks, n_temp, cand_cap, cands, counts, peak_out, keys);
}

// ---- batched forms: one launch per stage for every spectrum of a batch ----------------------------

// Spectrum of CTA x: the last job whose first CTA (field blk0 or blk1) is <= x.
template <bool K1>
__device__ __forceinline__ int job_of_block(const HsBatch &B, int x) {
    int lo = 0, hi = B.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int first = K1 ? B.job[mid].blk1 : B.job[mid].blk0;
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
    const HsJob &J = B.job[job_of_block<true>(B, blockIdx.x)];
    const int c = (n_temp - 1) / 2;
    const int row = c + group_row_offset(blockIdx.y, lo);
    const float ta = (mask & 1u) ? __ldg(&thresh[row]) : __int_as_float(0x7f800000);
    const bool vec = (J.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(J.plane) & 15) == 0;
    hs_row_k1(J.plane + (size_t)row * J.ld, J.n, ta, row, (blockIdx.x - J.blk1) * kK1Cols, J.raw, J.counters, J.peaks,
              vec);
}

template <int KL>
__global__ void __launch_bounds__(kHsThreads, KL <= 3 ? 4 : 2)
    fdas_hs_kl_batch(const HsBatch B, const float *__restrict__ thresh, int n_temp, unsigned mask, int lo) {
    const HsJob &J = B.job[job_of_block<false>(B, blockIdx.x)];
    const int c = (n_temp - 1) / 2;
    hs_row<KL>(J.plane, J.n, (size_t)J.ld, thresh, n_temp, mask, c, group_row_offset(blockIdx.y, lo),
               (blockIdx.x - J.blk0) * (kChunks * kHsThreads * jpt<KL>()), J.raw, J.counters, J.peaks);
}

__global__ void __launch_bounds__(kFinThreads) fdas_hs_finalize_batch(const HsBatch B, int n_temp, int cand_cap) {
    extern __shared__ unsigned long long keys[];
    const HsJob &J = B.job[blockIdx.y];
    finalize_plane(blockIdx.x + 1, J.raw, J.counters, J.peaks, n_temp, cand_cap, J.cands, J.counts, J.peak_out, keys);
}

using HsBatchKernel = void (*)(const HsBatch, const float *, int, unsigned, int);

HsBatchKernel hs_batch_kernel(int klast) {
    switch (klast) {
        case 1: return fdas_hs_k1_batch;
        case 2: return fdas_hs_kl_batch<2>;
        case 3: return fdas_hs_kl_batch<3>;
        case 4: return fdas_hs_kl_batch<4>;
        case 5: return fdas_hs_kl_batch<5>;
        case 6: return fdas_hs_kl_batch<6>;
        case 7: return fdas_hs_kl_batch<7>;
        case 8: return fdas_hs_kl_batch<8>;
        case 9: return fdas_hs_kl_batch<9>;
        case 10: return fdas_hs_kl_batch<10>;
        case 11: return fdas_hs_kl_batch<11>;
        case 12: return fdas_hs_kl_batch<12>;
        case 13: return fdas_hs_kl_batch<13>;
        case 14: return fdas_hs_kl_batch<14>;
        case 15: return fdas_hs_kl_batch<15>;
        default: return fdas_hs_kl_batch<16>;
    }
}

}  // namespace

cudaError_t launch_harmonic(const fdas_params &p, const float *plane, size_t n, size_t ld, const float *thresh,
                            fdas_cand *cands, uint32_t *counts, fdas_cand *peaks, const HsWorkspace &ws,
                            cudaStream_t s) {
    fdas_hs_reset<<<1, 32, 0, s>>>(ws.counters, ws.peaks, p.n_harm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Rows grouped by their number of planes klast: klast = n_harm for |i| <= c / n_harm, and
    // klast = K < n_harm for c/(K+1) < |i| <= c/K.
    const int c = (p.n_temp - 1) / 2;
    for (int K = p.n_harm; K >= 1; --K) {
        const int per = kChunks * kHsThreads * (K <= 9 ? jpt<9>() : jpt<10>());  // columns per CTA
        const unsigned gx = (unsigned)((n + per - 1) / per);
        const int lo = (K == p.n_harm) ? 0 : c / (K + 1) + 1;
        const int hi = c / K;
        if (hi < lo) continue;
        const int rows = (lo == 0) ? 2 * hi + 1 : 2 * (hi - lo + 1);
        const unsigned gxk = (K == 1) ? (unsigned)((n + kK1Cols - 1) / kK1Cols) : gx;
        hs_kernel(K)<<<dim3(gxk, (unsigned)rows), kHsThreads, 0, s>>>(plane, (int)n, ld, thresh, p.n_temp, p.harm_mask,
                                                                    lo, ws.raw, ws.counters, ws.peaks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int smem = FDAS_RAW_CAP * (int)sizeof(unsigned long long);
    e = cudaFuncSetAttribute(fdas_hs_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fdas_hs_finalize<<<p.n_harm, kFinThreads, smem, s>>>(ws.raw, ws.counters, ws.peaks, p.n_temp, p.cand_cap, cands,
                                                          counts, peaks);
    return cudaGetLastError();
}

// CTAs of one spectrum of n bins in the launches of rows with K >= 2 planes (all groups use the same
// column width for n_harm <= 9) and in the launch of single-plane rows.
void harmonic_blocks(const fdas_params &p, size_t n, int *blocks_kl, int *blocks_k1) {
    const int per = kChunks * kHsThreads * (p.n_harm <= 9 ? jpt<9>() : jpt<10>());
    *blocks_kl = (int)((n + per - 1) / per);
    *blocks_k1 = (int)((n + kK1Cols - 1) / kK1Cols);
}

cudaError_t prepare_harmonic_batch() {
    return cudaFuncSetAttribute(fdas_hs_finalize_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                FDAS_RAW_CAP * (int)sizeof(unsigned long long));
}

cudaError_t launch_harmonic_batch(const fdas_params &p, const HsBatch &B, int total_kl, int total_k1,
                                  const float *thresh, cudaStream_t s) {
    fdas_hs_reset_batch<<<B.count, 32, 0, s>>>(B, p.n_harm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int c = (p.n_temp - 1) / 2;
    for (int K = p.n_harm; K >= 1; --K) {
        const int lo = (K == p.n_harm) ? 0 : c / (K + 1) + 1;
        const int hi = c / K;
        if (hi < lo) continue;
        const int rows = (lo == 0) ? 2 * hi + 1 : 2 * (hi - lo + 1);
        const unsigned gx = (unsigned)(K == 1 ? total_k1 : total_kl);
        hs_batch_kernel(K)<<<dim3(gx, (unsigned)rows), kHsThreads, 0, s>>>(B, thresh, p.n_temp, p.harm_mask, lo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    fdas_hs_finalize_batch<<<dim3((unsigned)p.n_harm, (unsigned)B.count), kFinThreads,
                             FDAS_RAW_CAP * sizeof(unsigned long long), s>>>(B, p.n_temp, p.cand_cap);
    return cudaGetLastError();
}

}  // namespace fdas
