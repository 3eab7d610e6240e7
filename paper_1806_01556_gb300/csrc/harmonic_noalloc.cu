// fdas_harmonic_sum_noalloc: the harmonic-sum entry point for callers that cannot allocate
// device memory. Its scratch (crossing counters, per-plane peak keys and raw candidate keys)
// lives in one file-scope device array instead of a caller-provided workspace. The array is
// sized for up to 8 harmonic planes (the paper's N_hp). The CUDA driver loads it into a device's
// memory when the library's code is first loaded there (with lazy module loading, the default, that
// is the first call of this entry point on that device, inside its address lookup), and it stays
// until the process exits or the context is reset.
#include <mutex>

#include "fdas_internal.cuh"

namespace {

constexpr size_t kNoallocWords = FDAS_NOALLOC_SCRATCH_BYTES / sizeof(unsigned long long);
static_assert(FDAS_NOALLOC_SCRATCH_BYTES % sizeof(unsigned long long) == 0, "scratch size in whole words");

// Shared by every call on a device; kernels reach it through the address fetched below.
static __device__ __align__(256) unsigned long long g_fdas_noalloc_scratch[kNoallocWords];

constexpr int kMaxDevices = 128;
struct ScratchAddr {
    unsigned long long ctx;  // driver context id the address belongs to (0: none yet)
    void *addr;              // device address of the array in that context
};
ScratchAddr g_scratch_addr[kMaxDevices];  // per device ordinal
std::mutex g_scratch_mutex;

// In host code g_fdas_noalloc_scratch is only a host-side stand-in for the device array, so its
// device address is looked up once per device, with that device current. The address belongs to the
// device's context: after cudaDeviceReset the device gets a new context (with a new id), in which the
// array is loaded again, so the address is looked up again then.
cudaError_t scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long ctx = 0;
    e = fdas::current_context_id(&ctx);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_addr[dev].addr == nullptr || g_scratch_addr[dev].ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fdas_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = ScratchAddr{ctx, p};
    }
    *out = g_scratch_addr[dev].addr;
    return cudaSuccess;
}

}  // namespace

extern "C" fdas_status fdas_harmonic_sum_noalloc(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                                 const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts,
                                                 fdas_cand *d_peaks, fdas_stream_t stream) {
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    // Same argument checks as fdas_harmonic_sum, before the device address is looked up.
    if (n < 1 || n > FDAS_MAX_N || ld < n || !d_plane || !d_thresh || !d_cands || !d_counts) return FDAS_ERR_INVALID_ARG;
    if (fdas_workspace_bytes(p, n) > FDAS_NOALLOC_SCRATCH_BYTES) return FDAS_ERR_WORKSPACE;
    void *ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) return FDAS_ERR_CUDA;
    // The harmonic-sum launch sequence zeroes the counters and peak keys before its main kernel,
    // so whatever an earlier call left in the array does not leak into this one.
    // One stream only: the concurrent form would create the library's auxiliary streams.
    return fdas::harmonic_sum_checked(p, d_plane, n, ld, d_thresh, d_cands, d_counts, d_peaks, ws,
                                      FDAS_NOALLOC_SCRATCH_BYTES, stream, false);
}
