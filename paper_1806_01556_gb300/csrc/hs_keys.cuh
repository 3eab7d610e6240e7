// Candidate and peak keys of the harmonic planes, and the warp-level helpers that emit candidates
// and find peaks, shared by the harmonic-sum kernels and by the convolution when it detects HP_1
// itself. Internal linkage: each translation unit that includes this has its own copy.
#pragma once
#include "fdas_internal.cuh"

namespace fdas {
namespace {

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
// like their bits), then redux min of the location (row << 24 | column) among the lanes that hold
// that power. A lane with best < 0 has no point.
__device__ __forceinline__ unsigned long long warp_peak_key_loc(float best, unsigned loc) {
    const unsigned pb = best >= 0.0f ? __float_as_uint(best) : 0u;
    const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, pb);
    const unsigned lmin = __reduce_min_sync(0xFFFFFFFFu, (best >= 0.0f && pb == mx) ? loc : 0xFFFFFFFFu);
    if (lmin == 0xFFFFFFFFu) return 0ull;
    return ((unsigned long long)mx << 32) | (0xFFFFFFFFu - lmin);
}
// The same when every lane of the warp works on one row.
__device__ __forceinline__ unsigned long long warp_peak_key(float best, int bestj, int row) {
    return warp_peak_key_loc(best, ((unsigned)row << 24) | (unsigned)bestj);
}

}  // namespace
}  // namespace fdas
