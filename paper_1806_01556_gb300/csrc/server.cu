// Serving form: a request loop that admits spectra by HBM footprint into a fixed device arena, keeps
// several requests in flight on separate streams (so the convolution of one overlaps the harmonic
// sum of another), and returns each result with its submit, admit and completion times.
// Declarations and the full contract are in include/fdas.h.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "fdas_internal.cuh"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) of the device arena, in kAlign units; host-side bookkeeping only.
class Arena {
   public:
    explicit Arena(size_t size) { free_[0] = size; }
    // Offset of a block of `bytes`, or SIZE_MAX if no free block is large enough.
    size_t alloc(size_t bytes) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {  // merge with the following block
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {  // merge with the preceding block
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

   private:
    std::map<size_t, size_t> free_;  // offset -> length of each free block
};

struct Request {
    const void *h_spec;
    uint64_t n;
    uint64_t id;
    fdas_cand *h_cands;
    double submit_s;
};

// Device layout of one admitted request inside its arena block.
struct Footprint {
    size_t spec, plane, ws, cands, counts, peaks, total;
    size_t ld;
};

Footprint footprint(const fdas_params &p, uint64_t n) {
    Footprint f;
    f.ld = (size_t)((n + 63) / 64 * 64);
    size_t off = 0;
    f.spec = off;
    off += align_up((size_t)n * 8);
    f.plane = off;
    off += align_up((size_t)p.n_temp * f.ld * 4);
    f.ws = off;
    off += align_up(fdas_workspace_bytes(&p, n));
    f.cands = off;
    off += align_up((size_t)p.n_harm * p.cand_cap * sizeof(fdas_cand));
    f.counts = off;
    off += align_up((size_t)p.n_harm * 4);
    f.peaks = off;
    off += align_up((size_t)p.n_harm * sizeof(fdas_cand));
    f.total = off;
    return f;
}

struct Slot {
    bool busy = false;
    Request req{};
    size_t off = 0, bytes = 0;
    double admit_s = 0;
    fdas_status status = FDAS_OK;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    char *h_stage = nullptr;  // pinned: candidates, counts, peaks of this slot
};

}  // namespace

struct fdas_server {
    fdas_params p;
    int device = 0;
    size_t arena_bytes = 0;
    char *d_arena = nullptr;
    void *d_tmpl = nullptr;
    float *d_thresh = nullptr;
    Arena *arena = nullptr;
    std::vector<Slot> slots;
    size_t cand_bytes = 0;
    size_t status_off = 0;  // offset of the two device status words in a slot's staging buffer
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::deque<fdas_result> completed;
    int inflight = 0;
    bool stop = false;
    fdas_status fatal = FDAS_OK;
    std::thread worker;

    void run();
    bool admit_locked();
    bool complete_one(Slot &s);
};

// Launch one request on its slot: copy in, search, copy the small results back, record completion.
static fdas_status launch_request(fdas_server *sv, Slot &s, const Footprint &f) {
    char *base = sv->d_arena + s.off;
    cudaStream_t st = s.stream;
    const Request &r = s.req;
    if (cudaMemcpyAsync(base + f.spec, r.h_spec, (size_t)r.n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FDAS_ERR_CUDA;
    fdas_status rc = fdas_search(&sv->p, base + f.spec, r.n, sv->d_tmpl, reinterpret_cast<float *>(base + f.plane),
                                 f.ld, sv->d_thresh, reinterpret_cast<fdas_cand *>(base + f.cands),
                                 reinterpret_cast<uint32_t *>(base + f.counts),
                                 reinterpret_cast<fdas_cand *>(base + f.peaks), base + f.ws,
                                 fdas_workspace_bytes(&sv->p, r.n), st);
    if (rc != FDAS_OK) return rc;
    const size_t nh = (size_t)sv->p.n_harm;
    if (cudaMemcpyAsync(s.h_stage, base + f.cands, sv->cand_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(s.h_stage + sv->cand_bytes, base + f.counts, nh * 4, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(s.h_stage + sv->cand_bytes + nh * 4, base + f.peaks, nh * sizeof(fdas_cand),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        fdas::device_status_async(reinterpret_cast<unsigned *>(s.h_stage + sv->status_off), st) != cudaSuccess ||
        cudaEventRecord(s.done, st) != cudaSuccess)
        return FDAS_ERR_CUDA;
    return FDAS_OK;
}

// Admit pending requests, oldest first, while a slot is free and the oldest one's footprint fits.
bool fdas_server::admit_locked() {
    bool any = false;
    while (!pending.empty()) {
        Slot *free_slot = nullptr;
        for (auto &s : slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        if (!free_slot) break;
        const Request r = pending.front();
        const Footprint f = footprint(p, r.n);
        const size_t off = arena->alloc(f.total);
        if (off == SIZE_MAX) break;  // wait for memory to free up (requests keep their order)
        pending.pop_front();
        Slot &s = *free_slot;
        s.busy = true;
        s.req = r;
        s.off = off;
        s.bytes = f.total;
        s.admit_s = now_s();
        s.status = launch_request(this, s, f);
        ++inflight;
        any = true;
    }
    return any;
}

bool fdas_server::complete_one(Slot &s) {
    if (s.status == FDAS_OK) {
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) return false;
        if (q != cudaSuccess) s.status = FDAS_ERR_CUDA;
    } else {
        cudaStreamSynchronize(s.stream);  // nothing of the failed request may still run on the slot
    }
    fdas_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = s.req.id;
    res.n = s.req.n;
    res.status = s.status;
    res.submit_s = s.req.submit_s;
    res.admit_s = s.admit_s;
    res.done_s = now_s();
    if (s.status == FDAS_OK) {
        // The device status words, copied behind this request's search: a kernel that gave up on a
        // bounded wait since the last clear makes the result invalid.
        unsigned flags[2];
        std::memcpy(flags, s.h_stage + status_off, sizeof(flags));
        if ((flags[0] | flags[1]) & FDAS_DEV_WAIT_TIMEOUT) res.status = FDAS_ERR_TIMEOUT;
    }
    if (res.status == FDAS_OK) {
        const size_t nh = (size_t)p.n_harm;
        std::memcpy(res.counts, s.h_stage + cand_bytes, nh * 4);
        std::memcpy(res.peaks, s.h_stage + cand_bytes + nh * 4, nh * sizeof(fdas_cand));
        if (s.req.h_cands) std::memcpy(s.req.h_cands, s.h_stage, cand_bytes);
    }
    arena->release(s.off, s.bytes);
    s.busy = false;
    --inflight;
    completed.push_back(res);
    return true;
}

void fdas_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
        bool progress = false;
        for (auto &s : slots)
            if (s.busy && complete_one(s)) progress = true;
        if (admit_locked()) progress = true;
        if (progress) cv.notify_all();
        if (stop && inflight == 0 && (pending.empty() || fatal != FDAS_OK)) break;
        if (!progress) {
            // Idle or waiting on the GPU: poll the in-flight events every 50 microseconds.
            cv.wait_for(lock, std::chrono::microseconds(inflight ? 50 : 2000));
        }
    }
}

extern "C" {

fdas_status fdas_server_create(const fdas_params *p, size_t device_bytes, int max_inflight, fdas_server **out) {
    if (!out) return FDAS_ERR_INVALID_ARG;
    *out = nullptr;
    fdas_status st = fdas_check_params(p);
    if (st != FDAS_OK) return st;
    if (max_inflight < 1 || max_inflight > 16 || device_bytes < ((size_t)1 << 20)) return FDAS_ERR_INVALID_ARG;
    fdas_server *sv = new (std::nothrow) fdas_server;
    if (!sv) return FDAS_ERR_INVALID_ARG;
    sv->p = *p;
    sv->arena_bytes = align_up(device_bytes);
    sv->cand_bytes = (size_t)p->n_harm * p->cand_cap * sizeof(fdas_cand);
    cudaError_t e = cudaGetDevice(&sv->device);
    // Device memory is taken once, here: the template bank, the thresholds and the request arena.
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_tmpl, fdas_templates_bytes(p));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sv->d_thresh), (size_t)p->n_harm * p->n_temp * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sv->d_arena), sv->arena_bytes);
    std::vector<float> ta((size_t)p->n_harm * p->n_temp);
    if (e == cudaSuccess && fdas_default_thresholds(p, 6.0, 0, ta.data()) != FDAS_OK) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMemcpy(sv->d_thresh, ta.data(), ta.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fdas_make_templates(p, sv->d_tmpl, nullptr) != FDAS_OK) e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    sv->slots.resize((size_t)max_inflight);
    sv->status_off = (sv->cand_bytes + (size_t)p->n_harm * (4 + sizeof(fdas_cand)) + 7) / 8 * 8;
    const size_t stage = sv->status_off + 2 * sizeof(unsigned);
    for (auto &s : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&s.h_stage), stage);
    }
    if (e != cudaSuccess) {
        fdas_server_destroy(sv);
        return FDAS_ERR_CUDA;
    }
    sv->arena = new Arena(sv->arena_bytes);
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return FDAS_OK;
}

size_t fdas_server_request_bytes(const fdas_params *p, uint64_t n) {
    if (fdas_check_params(p) != FDAS_OK || n < 1 || n > FDAS_MAX_N) return 0;
    return footprint(*p, n).total;
}

fdas_status fdas_server_submit(fdas_server *sv, const void *h_spec, uint64_t n, uint64_t id, fdas_cand *h_cands) {
    if (!sv || !h_spec || n < 1 || n > FDAS_MAX_N) return FDAS_ERR_INVALID_ARG;
    if (footprint(sv->p, n).total > sv->arena_bytes) return FDAS_ERR_WORKSPACE;  // could never be admitted
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->stop) return FDAS_ERR_INVALID_ARG;
        sv->pending.push_back(Request{h_spec, n, id, h_cands, now_s()});
    }
    sv->cv.notify_all();
    return FDAS_OK;
}

fdas_status fdas_server_poll(fdas_server *sv, fdas_result *out, int max_results, int *n_out, int wait_ms) {
    if (!sv || !out || !n_out || max_results < 1) return FDAS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    if (sv->completed.empty() && wait_ms > 0)
        sv->cv.wait_for(lock, std::chrono::milliseconds(wait_ms), [sv] { return !sv->completed.empty(); });
    int k = 0;
    while (k < max_results && !sv->completed.empty()) {
        out[k++] = sv->completed.front();
        sv->completed.pop_front();
    }
    *n_out = k;
    return FDAS_OK;
}

void fdas_server_stats(fdas_server *sv, int *pending, int *inflight) {
    if (!sv) return;
    std::lock_guard<std::mutex> lock(sv->mu);
    if (pending) *pending = (int)sv->pending.size();
    if (inflight) *inflight = sv->inflight;
}

void fdas_server_destroy(fdas_server *sv) {
    if (!sv) return;
    if (sv->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            sv->stop = true;
        }
        sv->cv.notify_all();
        sv->worker.join();
    }
    for (auto &s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.h_stage) cudaFreeHost(s.h_stage);
    }
    cudaFree(sv->d_arena);
    cudaFree(sv->d_tmpl);
    cudaFree(sv->d_thresh);
    delete sv->arena;
    delete sv;
}

}  // extern "C"
