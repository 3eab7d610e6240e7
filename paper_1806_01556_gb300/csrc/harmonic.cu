// Harmonic summing with threshold detection (Sec. 2.2, Algorithm 1).
//
// Stretch read by fundamental: HP_k(i, j) = sum_{l=1..k} P[c + l*i][l*j] on
// D_k = {|k*i| <= c, k*j <= n-1}, summed in float32 in the order l = 1, 2, ..., k. As in the
// paper's MultipleHP kernels, all planes are computed at once and no HP plane is stored: one
// thread owns one fundamental (i, j) and keeps the running sum in a register.
//
// GB300 mapping:
//   fdas_hs_reset    zeroes the per-plane crossing counters and peak keys in the workspace.
//   fdas_hs          grid (column blocks, plane rows). Each thread handles 4 fundamentals of one
//                    row (2 when more than 8 planes are summed), j = j0 + tid + 256 u. It issues
//                    every strided gather P[c + l i][l j] before summing, so many loads are in
//                    flight, and reads through the read-only path. Crossings are compacted warp by warp: a ballot, one atomicAdd per warp,
//                    and a prefix popcount for each lane's slot. Each candidate is stored as one
//                    64-bit key whose ascending order is the canonical order
//                    (power desc, i asc, j asc). The loudest point of every plane is kept per
//                    thread, reduced across the warp with shuffles, and merged with one 64-bit
//                    atomicMax per warp.
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

// Fundamentals per thread: fewer when more planes are summed, to keep the gathers in registers.
template <int KMAX>
__host__ __device__ constexpr int hs_jpt() { return KMAX <= 8 ? 4 : 2; }

template <int KMAX>
__global__ void __launch_bounds__(kHsThreads)
    fdas_hs(const float *__restrict__ plane, int n, size_t ld, const float *__restrict__ thresh, int n_temp,
            int n_harm, unsigned mask, unsigned long long *__restrict__ raw, unsigned long long *counters,
            unsigned long long *peaks) {
    const int c = (n_temp - 1) / 2;
    const int row = blockIdx.y;  // c + i
    const int i = row - c;
    const int ai = i < 0 ? -i : i;
    // Planes k with |k i| <= c exist in this row. All of them are summed (the peak of every plane
    // is reported), and candidates are emitted for the planes selected by mask.
    const int klast = (ai == 0) ? n_harm : min(n_harm, c / ai);
    const int jend = n;
    constexpr int kJpt = hs_jpt<KMAX>();
    const int j0 = blockIdx.x * (kHsThreads * kJpt);

    const int lane = threadIdx.x & 31;
    float best[KMAX];
    unsigned bestj[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        best[k] = -1.0f;
        bestj[k] = 0u;
    }

    // Gather every term of every fundamental of this thread first.
    float v[kJpt][KMAX];
    int km[kJpt];
#pragma unroll
    for (int u = 0; u < kJpt; ++u) {
        const int j = j0 + threadIdx.x + kHsThreads * u;
        int terms = 0;
        if (j < jend) terms = (j == 0) ? klast : min(klast, (n - 1) / j);
        km[u] = terms;
#pragma unroll
        for (int l = 1; l <= KMAX; ++l) {
            if (l <= terms) v[u][l - 1] = __ldg(plane + (size_t)(c + l * i) * ld + (size_t)l * j);
        }
    }

#pragma unroll
    for (int u = 0; u < kJpt; ++u) {
        const unsigned j = (unsigned)(j0 + threadIdx.x + kHsThreads * u);
        float hp = 0.0f;
#pragma unroll
        for (int k = 1; k <= KMAX; ++k) {
            if (k > klast) break;  // block-uniform
            const bool valid = k <= km[u];
            if (valid) hp = (k == 1) ? v[u][0] : __fadd_rn(hp, v[u][k - 1]);
            if (valid && hp > best[k - 1]) {
                best[k - 1] = hp;
                bestj[k - 1] = j;
            }
            const bool hit = valid && ((mask >> (k - 1)) & 1u) && hp > __ldg(&thresh[(k - 1) * n_temp + row]);
            const unsigned ballot = __ballot_sync(0xFFFFFFFFu, hit);
            if (ballot) {
                const int leader = __ffs(ballot) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&counters[k - 1], (unsigned long long)__popc(ballot));
                base = __shfl_sync(0xFFFFFFFFu, base, leader);
                if (hit) {
                    const unsigned long long slot = base + __popc(ballot & ((1u << lane) - 1u));
                    if (slot < FDAS_RAW_CAP) raw[(size_t)(k - 1) * FDAS_RAW_CAP + slot] = cand_key(hp, row, j);
                }
            }
        }
    }

    // Loudest point per plane: warp-shuffle max of the 64-bit peak key, one atomicMax per warp.
#pragma unroll
    for (int k = 1; k <= KMAX; ++k) {
        if (k > klast) break;
        unsigned long long key = best[k - 1] >= 0.0f ? peak_key(best[k - 1], row, bestj[k - 1]) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, key, off);
            key = o > key ? o : key;
        }
        if (lane == 0 && key) atomicMax(&peaks[k - 1], key);
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

__global__ void __launch_bounds__(kFinThreads)
    fdas_hs_finalize(const unsigned long long *__restrict__ raw, const unsigned long long *counters,
                     const unsigned long long *peaks, int n_temp, int cand_cap, fdas_cand *cands, uint32_t *counts,
                     fdas_cand *peak_out) {
    extern __shared__ unsigned long long keys[];
    const int k = blockIdx.x + 1;
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

}  // namespace

cudaError_t launch_harmonic(const fdas_params &p, const float *plane, size_t n, size_t ld, const float *thresh,
                            fdas_cand *cands, uint32_t *counts, fdas_cand *peaks, const HsWorkspace &ws,
                            cudaStream_t s) {
    fdas_hs_reset<<<1, 32, 0, s>>>(ws.counters, ws.peaks, p.n_harm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p.n_harm <= 8) {
        constexpr int per = kHsThreads * hs_jpt<8>();
        dim3 grid((unsigned)((n + per - 1) / per), (unsigned)p.n_temp);
        fdas_hs<8><<<grid, kHsThreads, 0, s>>>(plane, (int)n, ld, thresh, p.n_temp, p.n_harm, p.harm_mask, ws.raw,
                                               ws.counters, ws.peaks);
    } else {
        constexpr int per = kHsThreads * hs_jpt<FDAS_MAX_HARM>();
        dim3 grid((unsigned)((n + per - 1) / per), (unsigned)p.n_temp);
        fdas_hs<FDAS_MAX_HARM><<<grid, kHsThreads, 0, s>>>(plane, (int)n, ld, thresh, p.n_temp, p.n_harm, p.harm_mask,
                                                           ws.raw, ws.counters, ws.peaks);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int smem = FDAS_RAW_CAP * (int)sizeof(unsigned long long);
    e = cudaFuncSetAttribute(fdas_hs_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fdas_hs_finalize<<<p.n_harm, kFinThreads, smem, s>>>(ws.raw, ws.counters, ws.peaks, p.n_temp, p.cand_cap, cands,
                                                          counts, peaks);
    return cudaGetLastError();
}

}  // namespace fdas
