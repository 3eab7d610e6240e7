/*
 * fdas.h - C ABI of the FDAS hot path on one GB300 (sm_103a).
 *
 * The Fourier-domain acceleration search (FDAS) module of Wang, Thiagaraj and Sinnen,
 * "Combining Multiple Optimized FPGA-based Pulsar Search Modules Using OpenCL", has two stages
 * (Sec. 2 and Sec. 3.1, Eq. t_FDAS):
 *   1. FT convolution. One complex input spectrum is correlated with N_temp acceleration
 *      templates of N_tap taps by overlap-save (Sec. 2.1). The power |y|^2 of each output forms
 *      the filter-output plane (FOP), here called the F-A plane.
 *   2. Harmonic summing with threshold detection over that plane (Sec. 2.2, Algorithm 1),
 *      which yields a candidate list per harmonic plane.
 *
 * Conventions for every call below:
 *   - Pointers named d_* are device pointers and h_* are host pointers. The caller owns every
 *     buffer, and no call allocates device memory.
 *   - Device buffers must be 16-byte aligned. cudaMalloc gives 256 bytes.
 *   - Calls that take a stream enqueue work on it and return without waiting, except
 *     fdas_search_host. A CUDA error seen at launch is returned as FDAS_ERR_CUDA. An error that
 *     happens later on the device shows up at the caller's next synchronisation.
 *   - Arguments are checked before any work is enqueued. A bad argument returns a negative
 *     status and enqueues nothing.
 *   - Complex values are interleaved float pairs (re, im), "complex64".
 *   - stream is a cudaStream_t. NULL means the legacy default stream.
 */
#ifndef FDAS_H
#define FDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fdas_stream_t; /* same type as cudaStream_t */

typedef int fdas_status;
#define FDAS_OK 0
#define FDAS_ERR_INVALID_ARG (-1) /* null/misaligned pointer, size out of range, bad params     */
#define FDAS_ERR_UNSUPPORTED (-2) /* valid parameters this build has no kernel for             */
#define FDAS_ERR_WORKSPACE (-3)   /* workspace smaller than fdas_workspace_bytes()             */
#define FDAS_ERR_CUDA (-4)        /* a CUDA runtime call or kernel launch failed               */
#define FDAS_ERR_TIMEOUT (-5)     /* a kernel gave up on a bounded device wait: outputs invalid */

/* Arithmetic of the FT convolution: plain FP32 FFTs, or part of each inverse DFT as a GEMM on the
 * tensor cores with 16-bit operands split in two (BF16 halves, or FP16 halves with scaling). */
#define FDAS_FP32 0
#define FDAS_BF16X3 1
#define FDAS_FP16S 2

/* Largest supported spectrum length. Candidate keys pack the column j into 24 bits. */
#define FDAS_MAX_N (1u << 24)
/* Per harmonic plane, up to this many threshold crossings are kept for the top-cand_cap
 * selection. Beyond it, counts[] still counts every crossing, but the kept set is whichever
 * crossings arrived first on the device, so the top-cand_cap choice is no longer exact. */
#define FDAS_RAW_CAP 16384
#define FDAS_MAX_CAND_CAP 4096
#define FDAS_MAX_HARM 16
#define FDAS_MAX_BATCH 256

/*
 * Search parameters (the paper's parameter table in Sec. 2, "FDAS Module Parameters").
 *   n_temp    N_temp, number of templates = plane rows. Odd, 3..255. Default 85.
 *   z_min     drift of template 0 in Fourier bins. The grid must be symmetric:
 *             z_min = -(n_temp-1)/2 * z_step. Default -42.
 *   z_step    drift step between templates, >= 1. Default 1. Template t has z_t = z_min + t*z_step.
 *   n_tap     N_tap, taps per template. Odd, 3..fft_len/2. Default 421.
 *   fft_len   overlap-save segment length F (AOLS-2048 in Sec. 2.1). Only 2048 in this build.
 *   n_harm    N_hp, harmonic planes summed, 1..16. Default 8.
 *   harm_mask bit k-1 set: report candidates of HP_k. Nonzero, no bit at or above n_harm.
 *   cand_cap  N_cand, candidates kept per reported plane, 1..4096. Default 200.
 *   precision  arithmetic of the FT convolution: FDAS_FP32 (default), FDAS_BF16X3 or FDAS_FP16S
 *              (the inverse DFTs partly on the tensor cores with split 16-bit operands).
 *   harm_index how a harmonic plane is indexed (the paper's "stretch" is not defined):
 *              FDAS_INDEX_FUNDAMENTAL (default): SP_k(i, j) = FOP(k i, k j), HP_k = HP_{k-1} + SP_k,
 *                on |k i| <= c, k j <= N-1 (c = (n_temp-1)/2);
 *              FDAS_INDEX_HIGHEST: (i, j) is the k-th (highest) harmonic, the lower harmonics sit at
 *                rounded fractions, HP_k(i, j) = sum_{l=1..k} FOP(rd(l i, k), rd(l j, k)) with
 *                rd(a, b) = round(a / b), halves away from zero, on the whole plane. Not incremental
 *                in k, so it reads the plane about (n_harm+1)/2 times as often. Not in the batched form.
 */
#define FDAS_INDEX_FUNDAMENTAL 0
#define FDAS_INDEX_HIGHEST 1
typedef struct {
    int32_t n_temp;
    int32_t z_min;
    int32_t z_step;
    int32_t n_tap;
    int32_t fft_len;
    int32_t n_harm;
    uint32_t harm_mask;
    int32_t cand_cap;
    int32_t precision;
    int32_t harm_index;
} fdas_params;

/* One candidate: HP_k(i, j) = power > TA(k, i). With FDAS_INDEX_FUNDAMENTAL, i is the fundamental's
 * template offset from the zero-drift row (drift z = i*z_step) and j its column (Fourier bin); with
 * FDAS_INDEX_HIGHEST they are those of the k-th harmonic. k is the harmonic plane (1-based). */
typedef struct {
    float power;
    uint32_t j;
    int16_t i;
    uint8_t k;
    uint8_t pad;
} fdas_cand;

/* Fill *p with the defaults above (85 templates, z = -42..42, 421 taps, F = 2048, 8 planes,
 * all reported, 200 candidates, FP32, fundamental indexing). */
void fdas_default_params(fdas_params *p);

/* FDAS_OK if *p is valid and this build has kernels for it. Otherwise FDAS_ERR_INVALID_ARG or
 * FDAS_ERR_UNSUPPORTED. */
fdas_status fdas_check_params(const fdas_params *p);

/* Human-readable name of a status code. The string is static. */
const char *fdas_status_string(fdas_status s);

/* The last CUDA error that this thread's calls met (behind an FDAS_ERR_CUDA, or inside a call that
 * recovered from it): the CUDA error's name and message, and the library function and source line
 * that saw it. Empty if there was none. The string is thread-local and stays valid until this
 * thread's next library call. No counterpart in the paper. */
const char *fdas_last_error(void);

/* Device-side status of the current device: bit FDAS_DEV_WAIT_TIMEOUT is set when a kernel gave up
 * on a bounded wait (the convolution waits on an mbarrier for each template's bulk copy, for about
 * one second at most). Such a kernel still ends, but its outputs are not valid. The paper has no
 * counterpart: its kernels run on an FPGA without such waits.
 *   *flags receives the bits (OR over every launch since the last clear); clear != 0 zeroes them.
 *   The read is synchronous with respect to the device (it waits for earlier work on the legacy
 *   default stream). Returns FDAS_ERR_INVALID_ARG for a null flags, FDAS_ERR_CUDA if the read fails.
 * How a timeout reaches the caller: an asynchronous call returns before its kernels run, so it
 * cannot return what they find later; the caller reads this word after synchronising. The calls
 * that wait on the device themselves read it before they return, and report FDAS_ERR_TIMEOUT when
 * FDAS_DEV_WAIT_TIMEOUT is set: fdas_search_host, fdas_batch_plan_tune, and the request loop's
 * per-request fdas_result.status. They leave the word as it is (clear it with this call). */
#define FDAS_DEV_WAIT_TIMEOUT 1u
fdas_status fdas_device_status(uint32_t *flags, int clear);

/* Sets the device status word of the current device to flags (synchronously, like
 * fdas_device_status). A diagnostic with no counterpart in the paper: it lets a program test its
 * handling of FDAS_ERR_TIMEOUT without making any kernel wait run out. Returns FDAS_ERR_CUDA if the
 * write fails. */
fdas_status fdas_set_device_status(uint32_t flags);

/* Measures the FP32 CUDA-core peak of the current device: a kernel of independent FFMA chains on
 * every SM (each FFMA counts 2 flop) runs for about `ms` milliseconds (10..2000), timed with CUDA
 * events. *tflops receives the rate in TFLOP/s and *elapsed_ms the timed duration. A diagnostic with
 * no counterpart in the paper: it is the denominator of the FP32 convolution's roofline.
 * Synchronous. Returns FDAS_ERR_INVALID_ARG for null outputs or ms out of range, FDAS_ERR_CUDA if a
 * CUDA call fails. */
fdas_status fdas_measure_fp32_peak(float ms, double *tflops, float *elapsed_ms);

/* Diagnostic of the bounded-wait path; no counterpart in the paper. Runs, on the current device,
 * one thread that waits on an mbarrier nothing completes, through the same bounded wait the
 * convolution kernels use. The wait gives up after about one second and the kernel returns.
 * *flags receives the device status bits that this left (FDAS_DEV_WAIT_TIMEOUT expected). The
 * status word is cleared before and after. Synchronous: it waits for the device to go idle.
 * Returns FDAS_ERR_INVALID_ARG for a null flags, FDAS_ERR_CUDA if a CUDA call fails. */
fdas_status fdas_check_wait_timeout(uint32_t *flags);

/* Size of the template bank written by fdas_make_templates: (n_temp + 1) * fft_len * 8 bytes.
 * Returns 0 for invalid parameters. */
size_t fdas_templates_bytes(const fdas_params *p);

/* Size of a plane of n columns with row stride ld (floats): n_temp * ld * 4 bytes. */
size_t fdas_plane_bytes(const fdas_params *p, size_t n, size_t ld);

/* Device workspace needed by fdas_harmonic_sum and fdas_search for a spectrum of n bins.
 * It holds candidate counters, per-plane peaks and up to FDAS_RAW_CAP raw candidate keys per
 * plane: 8 * n_harm * (FDAS_RAW_CAP + 4) bytes. Returns 0 for invalid parameters. */
size_t fdas_workspace_bytes(const fdas_params *p, size_t n);

/*
 * Threshold array TA(k, i) of Algorithm 1 (Sec. 2.2), computed on the host.
 * Row k-1 (k = 1..n_harm) holds the threshold of HP_k for every row offset i:
 * h_thresh[(k-1)*n_temp + (i + (n_temp-1)/2)].
 *   kind 0: the x with P(Gamma(k,1) > x) = Q(sigma), the one-sided Gaussian tail at sigma. For
 *           integer k, P(Gamma(k,1) > x) = exp(-x) sum_{m<k} x^m/m!. This is the false-alarm
 *           rate of a sum of k unit-mean exponential powers.
 *   kind 1: mean + sigma*sd = k + sigma*sqrt(k).
 * The value is computed in double precision and rounded to float. h_thresh holds
 * n_harm*n_temp floats.
 */
fdas_status fdas_default_thresholds(const fdas_params *p, double sigma, int kind, float *h_thresh);

/*
 * Template bank (FIR coefficients of the FT convolution; Sec. 2.1, 85 filters of 421 taps).
 * The paper does not define the kernel. This library uses the Fourier response of a linearly
 * drifting tone, indexed by mean frequency:
 *     A_z(q) = integral_0^1 exp(2 pi i (-(q + z/2) tau + z tau^2/2)) d tau,
 * evaluated in double precision on the device (composite 16-point Gauss-Legendre quadrature).
 * Template t uses z_t = z_min + t*z_step and taps a_t[q] = A_{z_t}(q), q = -h..h, with
 * h = (n_tap-1)/2.
 * d_tmpl (fdas_templates_bytes bytes, complex64) receives:
 *   rows t = 0..n_temp-1: T_t[m] = conj( sum_q a_t[q] exp(-2 pi i m q / F) ), m = 0..F-1.
 *                         This is the DFT (Eq. 2) of the taps placed wrapped in a length-F array.
 *   row n_temp:           the twiddle table w[k] = exp(-2 pi i k / F), k = 0..F-1.
 * The DFT and the twiddles are computed in double precision and rounded once to float.
 * The bank is read-only input to fdas_convolve and fdas_search.
 */
fdas_status fdas_make_templates(const fdas_params *p, void *d_tmpl, fdas_stream_t stream);

/*
 * FT convolution by overlap-save (Sec. 2.1: OLS-FDFIR, AOLS-2048-P with power), producing the
 * F-A plane:
 *     P[t][j] = | sum_{q=-h}^{h} X[j+q] conj(a_t[q]) |^2,  X = 0 outside [0, n),
 * for t = 0..n_temp-1 and j = 0..n-1.
 * Each segment of F input points (overlap n_tap-1) is transformed once, multiplied by every
 * template and transformed back. Only the L = F - n_tap + 1 valid outputs per segment are
 * stored, so the paper's "discard" step of the FOP preparation (Sec. 3.2) is fused into the store.
 *   d_spec  complex64[n], the input spectrum. 1 <= n <= FDAS_MAX_N.
 *   d_tmpl  bank from fdas_make_templates with the same parameters.
 *   d_plane float32[n_temp][ld], ld >= n. Columns n..ld-1 are not written.
 * Arithmetic is float32 with float32 FFTs.
 */
fdas_status fdas_convolve(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl,
                          float *d_plane, size_t ld, fdas_stream_t stream);

/*
 * Harmonic summing with threshold detection (Sec. 2.2, Algorithm 1), with the stretch read by
 * fundamental:
 *     HP_k(i, j) = sum_{l=1}^{k} P[c + l*i][l*j],  c = (n_temp-1)/2,
 * on the domain |k*i| <= c, k*j <= n-1. The sum is float32, running in the order l = 1, 2, ..., k.
 * A point is a candidate of plane k when bit k-1 of harm_mask is set and
 * HP_k(i, j) > d_thresh[(k-1)*n_temp + c + i] (strict, float32).
 *   d_plane  float32[n_temp][ld], e.g. from fdas_convolve.
 *   d_thresh float32[n_harm][n_temp] (see fdas_default_thresholds).
 *   d_cands  fdas_cand[n_harm][cand_cap]. Slot k-1 receives the top min(counts[k-1], cand_cap)
 *            crossings of HP_k in canonical order: power descending, then i, then j ascending.
 *            Slots past that are not written.
 *   d_counts uint32[n_harm]: total crossings per plane (0 for planes not reported).
 *   d_peaks  fdas_cand[n_harm] or NULL: the first point of each HP_k in canonical order,
 *            whether or not it crosses the threshold.
 *   d_ws     workspace of at least fdas_workspace_bytes(p, n) bytes, used for counters and raw
 *            candidate keys. Its contents need no initialisation.
 * Calls that share d_ws must not overlap on the device.
 * The kernels of one call may run side by side on two auxiliary streams of the library, forked from
 * and joined back into `stream` with events, so work enqueued on `stream` afterwards, and a graph
 * captured from `stream`, see the whole harmonic sum. The pair belongs to the calling host thread and
 * CUDA context and serves all of that thread's caller streams, so successive harmonic sums of one
 * thread queue behind one another on it; it is made at the first call that needs it (or in
 * fdas_make_templates) and kept until the process exits. Calls from other threads never share it, so a
 * capture in one thread records none of another thread's work. While a pair takes part in a capture,
 * it serves only calls on that capture's streams; another call of the same thread gets a second pair
 * (up to 8 per thread). No pair is made while `stream` is being captured: a captured call that finds
 * none runs its kernels on `stream` alone, with the same results. A pair made before cudaDeviceReset
 * is never used afterwards.
 */
fdas_status fdas_harmonic_sum(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                              const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts,
                              fdas_cand *d_peaks, void *d_ws, size_t ws_bytes, fdas_stream_t stream);

/*
 * Launch shape of the convolution kernel (not part of the method; the paper's counterpart is the
 * compile-time parallelisation factor of its OpenCL kernels, Sec. 3.3 "Parallelisation Factor").
 *   ctas_per_sm           0: one CTA per work item, as many resident as fit (3 per SM). k > 0: a
 *                         persistent grid of k CTAs per SM that loop over the work items, which leaves
 *                         room on every SM for kernels of other streams (e.g. the harmonic sum of the
 *                         previous spectrum).
 *   templates_per_item    0: a work item is one segment with all n_temp templates (the segment is
 *                         transformed once). k > 0: items of k templates; each item transforms its
 *                         segment again, which gives more, smaller items.
 * Results do not depend on the launch shape.
 */
typedef struct {
    int32_t ctas_per_sm;
    int32_t templates_per_item;
} fdas_launch_config;

/* fdas_convolve with an explicit launch shape (NULL = the defaults, as fdas_convolve). */
fdas_status fdas_convolve_cfg(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl, float *d_plane,
                              size_t ld, const fdas_launch_config *cfg, fdas_stream_t stream);

/* The whole FDAS path for one spectrum (Sec. 3.1, Eq. t_FDAS, with no separate FOP preparation):
 * fdas_search_convolve then fdas_search_harmonic on the same stream. The plane and the candidate
 * lists equal those of fdas_convolve followed by fdas_harmonic_sum, bit for bit, except that when
 * a plane has more than FDAS_RAW_CAP crossings the kept set (whichever arrived first) may differ. */
fdas_status fdas_search(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl,
                        float *d_plane, size_t ld, const float *d_thresh, fdas_cand *d_cands,
                        uint32_t *d_counts, fdas_cand *d_peaks, void *d_ws, size_t ws_bytes,
                        fdas_stream_t stream);

/*
 * fdas_search with the spectrum and the results in host memory: the end-to-end call.
 * It copies h_spec (complex64[n], pinned memory recommended) into d_spec, runs fdas_search,
 * copies the candidates, counts and (if h_peaks is not NULL) peaks back to the host, and waits
 * for the stream. d_cands, d_counts and d_peaks are device staging buffers of the same shapes as
 * in fdas_harmonic_sum (d_peaks may be NULL only if h_peaks is NULL). Returns FDAS_ERR_TIMEOUT if,
 * once the stream is done, the device status word shows that a kernel gave up on a bounded wait
 * (fdas_device_status); the results are not valid then.
 */
/*
 * The two stages of fdas_search, for callers that time or schedule them apart. Arguments as in
 * fdas_search; both must run, in this order, on the same plane and workspace.
 *   fdas_search_convolve: resets the workspace, then runs the convolution. With FDAS_FP32 it also
 *     takes the HP_1 candidates and the HP_1 peak while each plane value is in registers: HP_1 is the
 *     F-A plane itself (Algorithm 1 with k = 1), so the harmonic sum needs no single-plane pass.
 *   fdas_search_harmonic: the remaining harmonic planes, detection and the candidate lists.
 */
fdas_status fdas_search_convolve(const fdas_params *p, const void *d_spec, size_t n, const void *d_tmpl,
                                 float *d_plane, size_t ld, const float *d_thresh, void *d_ws, size_t ws_bytes,
                                 fdas_stream_t stream);
fdas_status fdas_search_harmonic(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                 const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                                 void *d_ws, size_t ws_bytes, fdas_stream_t stream);

fdas_status fdas_search_host(const fdas_params *p, const void *h_spec, size_t n, void *d_spec,
                             const void *d_tmpl, float *d_plane, size_t ld, const float *d_thresh,
                             fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                             fdas_cand *h_cands, uint32_t *h_counts, fdas_cand *h_peaks, void *d_ws,
                             size_t ws_bytes, fdas_stream_t stream);

/*
 * fdas_search_host without the final wait: the copy in, the search and the copies out are enqueued
 * on `stream` and the call returns. h_cands, h_counts and h_peaks hold the results once the stream
 * has reached that point (cudaStreamSynchronize, or an event recorded after the call); h_spec must
 * not change before then. Everything is ordered on `stream` alone, so the copy in waits for the
 * stream's previous work. With pinned host buffers and three sets of device buffers used on three
 * streams in turn, each copy in waits only for a search two spectra back and overlaps the other
 * streams' searches (at N = 2^21 on a GB300 the end-to-end rate then matches the device-resident
 * one; with two streams about half of each copy stays exposed). Arguments and checks as in
 * fdas_search_host.
 */
fdas_status fdas_search_host_async(const fdas_params *p, const void *h_spec, size_t n, void *d_spec,
                                   const void *d_tmpl, float *d_plane, size_t ld, const float *d_thresh,
                                   fdas_cand *d_cands, uint32_t *d_counts, fdas_cand *d_peaks,
                                   fdas_cand *h_cands, uint32_t *h_counts, fdas_cand *h_peaks, void *d_ws,
                                   size_t ws_bytes, fdas_stream_t stream);

/*
 * Scratch size of fdas_harmonic_sum_noalloc: the workspace of 8 harmonic planes,
 * 8 * 8 * (FDAS_RAW_CAP + 4) bytes (about 1 MiB).
 */
#define FDAS_NOALLOC_SCRATCH_BYTES ((size_t)8 * 8 * (FDAS_RAW_CAP + 4))

/*
 * fdas_harmonic_sum without a caller-provided workspace. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at all. Examples are a stage that is
 * handed only its input and output buffers by the framework that owns the GPU, or a real-time
 * loop that must never call cudaMalloc (which can synchronise the whole device).
 *
 * The scratch is a static device array of FDAS_NOALLOC_SCRATCH_BYTES inside libfdas. Every GPU
 * that loads the library's device code holds it until the process exits. The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine. Arguments and results are as
 * for fdas_harmonic_sum, which it calls with that array as d_ws, on `stream` alone (no auxiliary
 * streams).
 *   - Parameter sets whose workspace exceeds the array (n_harm > 8) are rejected with
 *     FDAS_ERR_WORKSPACE, before anything is enqueued.
 *   - The first call on a device looks up the array's device address, with that device current.
 *     With CUDA's lazy module loading (the default), that lookup is also what loads the array into
 *     the device's memory: the driver reserves its FDAS_NOALLOC_SCRATCH_BYTES then. Later calls
 *     reserve nothing. Make that first call before any stream capture, and before measuring free
 *     memory if the figure matters.
 *   - cudaDeviceReset destroys the array with the context. The next call on that device (in the new
 *     context) loads it again and looks up its new address; the address cached for the old context is
 *     never used again.
 *   - All calls on a device share the one array, which keeps the last call's contents. Each call
 *     clears the counters it needs before use. Calls that overlap on the GPU (on different
 *     streams, or from different host threads) race on the array and must be serialised by the
 *     caller.
 */
fdas_status fdas_harmonic_sum_noalloc(const fdas_params *p, const float *d_plane, size_t n, size_t ld,
                                      const float *d_thresh, fdas_cand *d_cands, uint32_t *d_counts,
                                      fdas_cand *d_peaks, fdas_stream_t stream);

/* ---- Batched form: many spectra (DM trials) of uneven length in one launch per stage ---------- */

/* One spectrum of a batch, with its own outputs (shapes as in fdas_search). */
typedef struct {
    const void *d_spec; /* complex64[n] */
    uint64_t n;         /* 1..FDAS_MAX_N */
    float *d_plane;     /* float32[n_temp][ld] */
    uint64_t ld;        /* >= n */
    fdas_cand *d_cands; /* [n_harm][cand_cap] */
    uint32_t *d_counts; /* [n_harm] */
    fdas_cand *d_peaks; /* [n_harm] or NULL */
} fdas_batch_item;

/* Workspace of fdas_search_batch for count spectra: one harmonic-sum workspace per spectrum
 * (fdas_workspace_bytes rounded up to 256 bytes each). Returns 0 for invalid arguments. */
size_t fdas_batch_workspace_bytes(const fdas_params *p, int count);

/*
 * fdas_search on count (1..FDAS_MAX_BATCH) spectra of any lengths, with one launch per stage for the
 * whole batch rather than per spectrum. The paper pipelines a stream of input arrays through one
 * device (Sec. 3.3) or spreads them over devices (Sec. 3.5, "single bitstream, multiple inputs").
 * Here one GPU takes them all at once:
 *   - a persistent convolution kernel whose CTAs loop over every (spectrum, segment) work item;
 *   - the harmonic sum of every spectrum: one launch per group of rows, then one finalize launch.
 * Results are those of fdas_search on each spectrum alone, bit for bit. The per-spectrum tables are
 * kernel parameters, so the call enqueues kernels only: no allocation, copy or synchronisation. It
 * can therefore be captured in a CUDA graph. cfg (NULL = defaults) shapes the convolution launch; a
 * persistent grid always has ctas_per_sm (0 means 3) CTAs per SM.
 */
fdas_status fdas_search_batch(const fdas_params *p, const fdas_batch_item *items, int count, const void *d_tmpl,
                              const float *d_thresh, void *d_ws, size_t ws_bytes, const fdas_launch_config *cfg,
                              fdas_stream_t stream);

/*
 * fdas_harmonic_sum on count (1..FDAS_MAX_BATCH) planes of any lengths, with the batched kernels of
 * fdas_search_batch: one launch per group of rows over every plane, then one finalize launch
 * (Sec. 2.2, Algorithm 1, as in fdas_harmonic_sum). Each item's d_plane (n_temp x ld floats) is
 * read; its d_spec is not used and may be NULL. Results are those of fdas_harmonic_sum on each plane
 * alone, bit for bit. d_ws holds fdas_batch_workspace_bytes(p, count) bytes. Enqueues kernels only.
 */
fdas_status fdas_harmonic_sum_batch(const fdas_params *p, const fdas_batch_item *items, int count,
                                    const float *d_thresh, void *d_ws, size_t ws_bytes, fdas_stream_t stream);

/*
 * A batch plan: fdas_search_batch with fixed buffers, replayed as a CUDA graph.
 *   create  checks and copies the item list (the buffers themselves are not copied and must stay valid).
 *   tune    times the candidate convolution launch shapes (ctas_per_sm in {0, 2}, templates_per_item in
 *           {0, 43, 29, 17}) on the plan's own spectra with CUDA events, keeps the fastest, and returns
 *           it with its convolution time per batch. It waits on stream, and returns FDAS_ERR_TIMEOUT
 *           (keeping the previous shape) if a timed kernel gave up on a bounded wait.
 *   launch  enqueues the batch on stream. The first launch (and the first after tune) captures the
 *           launches into a CUDA graph on the plan's private stream (a thread-local capture: other
 *           threads may run searches meanwhile); later launches replay that graph.
 *   destroy frees the plan and its graph.
 * A plan holds host memory and a CUDA graph; it allocates no device memory.
 */
typedef struct fdas_batch_plan fdas_batch_plan;
fdas_status fdas_batch_plan_create(const fdas_params *p, const fdas_batch_item *items, int count, const void *d_tmpl,
                                   const float *d_thresh, void *d_ws, size_t ws_bytes, fdas_batch_plan **plan);
fdas_status fdas_batch_plan_tune(fdas_batch_plan *plan, fdas_stream_t stream, fdas_launch_config *chosen,
                                 float *ms_per_batch);
fdas_status fdas_batch_plan_launch(fdas_batch_plan *plan, fdas_stream_t stream);
void fdas_batch_plan_destroy(fdas_batch_plan *plan);

/* ---- Serving form: a request loop with admission by device-memory footprint --------------------- */

/* One finished request (times are seconds on the host's steady clock). */
typedef struct {
    uint64_t id;                       /* the caller's request id */
    uint64_t n;                        /* spectrum length */
    fdas_status status;                /* FDAS_OK, or the error of this request (FDAS_ERR_TIMEOUT: the
                                          device status showed a bounded wait that gave up) */
    int32_t pad;
    double submit_s;                   /* fdas_server_submit returned */
    double admit_s;                    /* the request got a slot and its device memory, and was launched */
    double done_s;                     /* the worker saw its results on the host */
    uint32_t counts[FDAS_MAX_HARM];    /* as d_counts of fdas_search (first n_harm entries) */
    fdas_cand peaks[FDAS_MAX_HARM];    /* as d_peaks of fdas_search (first n_harm entries) */
} fdas_result;

/*
 * A request loop for a continuous stream of spectra. The paper processes a stream of input arrays
 * through the FDAS module with double or triple buffering between its stages (Sec. 3.3, pipeline
 * period max(t_FT, t_FOP, t_HM)). Here the buffers are device-resident and the stages of different
 * requests overlap on the GPU.
 *   create  takes all device memory once: the template bank, the 6-sigma thresholds and an arena of
 *           device_bytes for requests. It starts a worker thread on the current device. Up to
 *           max_inflight (1..16, 3 = triple buffering) requests run at once, each on its own stream.
 *   request_bytes  the arena footprint of one request of n bins (spectrum, plane, workspace, results).
 *   submit  queues a spectrum (host complex64[n]; pinned memory recommended; it must stay valid until
 *           the request's result has been polled). h_cands (host fdas_cand[n_harm][cand_cap], or NULL)
 *           receives the candidates. Requests are admitted in order as a slot and arena memory become
 *           free; requests that arrive while others run join them on the GPU. Returns FDAS_ERR_WORKSPACE
 *           if the request could never fit the arena.
 *   poll    moves up to max_results finished requests into out (waiting up to wait_ms for the first).
 *   stats   current queue length and requests in flight.
 *   destroy waits until every submitted request has finished, then frees everything.
 * Results are those of fdas_search on the same spectrum alone, bit for bit.
 */
typedef struct fdas_server fdas_server;
fdas_status fdas_server_create(const fdas_params *p, size_t device_bytes, int max_inflight, fdas_server **server);
size_t fdas_server_request_bytes(const fdas_params *p, uint64_t n);
fdas_status fdas_server_submit(fdas_server *server, const void *h_spec, uint64_t n, uint64_t id, fdas_cand *h_cands);
fdas_status fdas_server_poll(fdas_server *server, fdas_result *out, int max_results, int *n_out, int wait_ms);
void fdas_server_stats(fdas_server *server, int *pending, int *inflight);
void fdas_server_destroy(fdas_server *server);

#ifdef __cplusplus
}
#endif

#endif /* FDAS_H */
