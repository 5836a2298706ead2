/*
 * cyc.h -- C ABI of libcyc, a streaming estimator of second-order cyclic statistics on
 * one NVIDIA GB300 (sm_103a).
 *
 * What a stream estimates (arXiv 2405.16911, Sec. 2 discrete estimators and Sec. 4
 * Eq. (impl-corr); here for one input, x = y, and lags m >= 0), over every sample pushed
 * so far:
 *
 *   R_CONV[a][m] = (1/N_eff) sum_{n=0}^{N_eff-1} x[n+m] conj(x[n]) exp(-j 2 pi a (n0+n))
 *   R_CONJ[a][m] = (1/N_eff) sum_{n=0}^{N_eff-1} x[n+m]      x[n]  exp(-j 2 pi a (n0+n))
 *
 *   N_eff = max(0, T - M), T = samples pushed, M = max(lags), n0 = start index.
 *
 * Signed lags shift the window by M^- = -min(lags) (see cyc_params), and streams made by
 * cyc_create_xy take a second input y in place of the conjugated factor (cross forms).
 *
 * CONV is the cyclic autocorrelation (Eq. (ACF-def)), CONJ the conjugate cyclic
 * correlation (Eq. (CCF-def)); the paper's block attribute `conj` selects between
 * them (Sec. 4), here a bitmask selects one or both.  a is a normalised cycle frequency
 * in cycles/sample (Sec. 2: alpha~ = alpha / f_s); any finite value is accepted and a
 * and a + 1 give the same result.  All lags share one n-range, so the result does not
 * depend on how the samples are cut into pushes: the last M samples of every push wait
 * for the next one (the paper's input buffer, Sec. 4, holds samples for the same reason).
 *
 * Conventions for every entry point:
 *  - Return 0 on success, a negative CYC_E* code on failure; cyc_last_error() then
 *    gives a thread-local message.  Nothing is half-applied on CYC_EINVAL.
 *  - A handle is not thread-safe.  Distinct handles may be used from distinct threads.
 *  - Samples are interleaved complex64: float re, float im (8 bytes per sample).
 *  - Results are interleaved complex FP64, layout [form][alpha index][lag index][re, im],
 *    forms in the order CONV then CONJ (only those selected), alphas and lags in the
 *    order given at creation (duplicates allowed).
 */
#ifndef CYC_H
#define CYC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CYC_API __attribute__((visibility("default")))
#else
#define CYC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CYC_OK         0
#define CYC_EINVAL    (-1)   /* bad argument: empty list, negative lag, non-finite a, n < 0 ... */
#define CYC_ENOMEM    (-2)   /* device or host allocation failed */
#define CYC_ECUDA     (-3)   /* a CUDA runtime call failed (message names it) */
#define CYC_EAGAIN    (-4)   /* server: stream not admitted (memory budget / slots), retry later */
#define CYC_ETIMEDOUT (-5)   /* a bounded device wait gave up */
#define CYC_ENODATA   (-6)   /* N_eff == 0: nothing to read; the output is left untouched */
#define CYC_ENOTSUP   (-7)   /* valid request that the library does not implement */

/* ---- forms (bitmask) ---- */
#define CYC_CONV 1           /* x[n+m] conj(x[n]) */
#define CYC_CONJ 2           /* x[n+m] x[n]       */
#define CYC_BOTH 3

/* ---- projection precision (the a-projection, Sec. 4 Set mode; sums are always FP64) ---- */
#define CYC_P_FP32   0       /* FP32 CUDA-core complex GEMM, FP32 accumulate */
#define CYC_P_FP16   1       /* tensor cores, FP16 operands, one pass, FP32 accumulate */
#define CYC_P_BF16X3 2       /* tensor cores, BF16 hi/lo split, hi*hi + hi*lo + lo*hi, FP32 accumulate */
/* The tensor-core precisions run on pairs of SMs (two-CTA clusters issuing cta_group::2
 * MMAs); a device that cannot hold such clusters reports CYC_ENOTSUP for them.  A cycle
 * frequency a and its negative -a (mod 1), when both are in a stream's list, share one pair
 * of real weight rows and cost the tensor work of one; 0 and 1/2 share one more. */

typedef struct cyc_stream cyc_stream;   /* opaque, owned by the library */

/*
 * Creation parameters.  Arrays are copied; the caller keeps ownership.
 *   lags[nlags]       signed lags m (Sec. 4 Set mode spans -max_lag .. max_lag), |m| <= 2^20 and
 *                     max - min <= 2^20 (CYC_EINVAL otherwise).  With M^- = max(0, -min m) and
 *                     M^+ = max(0, max m), term n pairs x[n + m] with the reference sample
 *                     at n, n = M^- .. T - M^+ - 1 (Eq. (impl-corr): the window starts M^-
 *                     samples in), N_eff = T - M^- - M^+, and the phase is that of n.
 *   alphas[nalphas]   normalised cycle frequencies (finite doubles)
 *   conj_flag         CYC_CONV, CYC_CONJ or CYC_BOTH
 *   precision         CYC_P_*
 *   n0                absolute index of the first sample (phase origin, any int64)
 *   max_chunk         samples of one device pass: pushes are staged behind each other and
 *                     projected together once a pass is full (and before any call that reads
 *                     the stream), longer pushes are cut.  0 selects 1 << 20.  Device staging
 *                     memory is 2 * (M + max_chunk) * 8 B.
 *   cuda_stream       cudaStream_t the stream's work is ordered on; NULL = the legacy
 *                     default stream of `device`
 *   device            CUDA device ordinal
 */
typedef struct cyc_params {
    const int32_t* lags;
    int32_t        nlags;
    const double*  alphas;
    int32_t        nalphas;
    int32_t        conj_flag;
    int32_t        precision;
    int64_t        n0;
    int64_t        max_chunk;
    void*          cuda_stream;
    int32_t        device;
} cyc_params;

/* cyc_create: FP32 projection, n0 = 0, default stream of device 0.  *out receives the handle. */
CYC_API int cyc_create(const int32_t* lags, int nlags, const double* alphas, int nalphas,
               int conj_flag, cyc_stream** out);

/* cyc_create_ex: every parameter explicit (see cyc_params). */
CYC_API int cyc_create_ex(const cyc_params* p, cyc_stream** out);

/*
 * cyc_create_xy: a stream with two inputs x and y, the cross forms of Eq. (impl-corr):
 *   CONV  R[a][m] = (1/N_eff) sum_n x[n+m] conj(y[n]) exp(-j 2 pi a n)   (cyclic cross-correlation)
 *   CONJ  R[a][m] = (1/N_eff) sum_n x[n+m] y[n]       exp(-j 2 pi a n)   (conjugate form)
 * with n over the same range as cyc_params describes.  Samples arrive through
 * cyc_push_xy only; cyc_read, cyc_reset, cyc_save and cyc_load work as for one input (the
 * blob then carries both tails).  Server streams have one input.
 */
CYC_API int cyc_create_xy(const cyc_params* p, cyc_stream** out);

/*
 * cyc_create_window: the block's windowed output (Sec. 4, Eq. (impl-corr) evaluated at
 * window starts n0 = k * hop, k = 0, 1, ...).  Window k is the estimate over the win_len
 * reference samples n = k * hop + M^- .. k * hop + M^- + win_len - 1 (sample indices from
 * the first pushed sample), normalised by win_len, with the window-local phase of the
 * equation: exp(-j 2 pi a n') with n' = 0 at the window's first reference sample.  The
 * running sums of cyc_read keep their meaning.  A window is complete once its last x
 * sample has been pushed; completed windows wait in a device ring of `capacity` windows
 * for cyc_read_windows.  A push that would complete more windows than the ring has room
 * for fails with CYC_EAGAIN before doing anything (read windows, then push again).  Window
 * sums are formed from hop sums rounded once to FP32 and wait in FP32 until read (about
 * 1e-7 of each entry beyond the projection's own error); the update that adds a hop and
 * drops the oldest cancels exactly, so long streams carry no drift.
 *   win_len   positive multiple of hop, win_len / hop <= 65536
 *   hop       >= 1 samples between window starts (hop = 1: a window per sample, the block's
 *             own output rate); below 16 only with CYC_P_FP32, whose passes then hold as
 *             many hops as 64 MB of FP32 partials allow
 *   capacity  1 .. 2^20 windows of F * (distinct a) * nlags * 8 bytes each (held in FP32
 *             until read; plus device state of (win_len / hop) * (distinct a) * F * nlags
 *             * 8 bytes for the hop sums and 2 * (distinct a) * F * nlags * 16 bytes)
 *   cross     0: one input (cyc_push); 1: two inputs (cyc_push_xy), as cyc_create_xy
 * cyc_save / cyc_load return CYC_ENOTSUP for windowed streams.
 */
CYC_API int cyc_create_window(const cyc_params* p, int64_t win_len, int64_t hop, int64_t capacity, int cross,
                              cyc_stream** out);

/*
 * cyc_create_full: the paper's Full mode -- every cycle frequency of [-1/2, 1/2) on the
 * uniform grid a_k = -1/2 + k/A, k = 0 .. A-1 (p->alphas and p->nalphas are ignored; the
 * output's cycle-frequency index is k).  The result is the same estimator as a stream with
 * those alphas (same layout for cyc_read, same range of n, absolute phase); on this grid the
 * phase depends on n only through n mod A, so a push folds its lag products modulo A
 * (float-float sums of FP32 runs, about 48 significant bits) and cyc_read takes one A-point
 * DFT per column: O(samples x columns) work per push instead of O(samples x columns x A).
 * Pushes are folded in batches: 8-byte aligned device chunks are read where they are and
 * folded, up to 16 chunks and max_chunk samples at a time, in one launch (when the next push
 * would not fit, and before any call that reads or replaces the stream's state: cyc_read,
 * cyc_sync, cyc_save, cyc_load, cyc_reset, cyc_info, ...).  As for every stream, a device
 * chunk must stay unchanged until the next cyc_read / cyc_sync.
 *   A          power of two in [2, 4096]
 *   precision  must be CYC_P_FP32 (FP32 lag products, float-float folding, FP64 DFT); else CYC_EINVAL
 *   cross      0: one input (cyc_push); 1: two inputs (cyc_push_xy)
 * cyc_save / cyc_load, cyc_reset work as for any stream; cyc_sums returns CYC_ENOTSUP (the
 * folds are float-float, not FP64 sums); windows are not available.
 */
CYC_API int cyc_create_full(const cyc_params* p, int32_t A, int cross, cyc_stream** out);

/*
 * cyc_create_full_window: the paper's Full mode per window (Sec. 4: with win_len = A, one
 * A-point FFT per lag over each window; each window's output holds nlags * A values per form).
 * Window k covers the A reference samples n = k * hop + M^- .. k * hop + M^- + A - 1 (sample
 * indices from the first pushed sample) and, for every lag m and form f, gives
 *   W_k[f][kk][l] = (1/A) sum_{n'=0}^{A-1} x[n0 + n' + m_l] c_f(y[n0 + n']) exp(-j 2 pi a_kk n'),
 *   a_kk = -1/2 + kk/A,  n0 = k * hop + M^-,
 * i.e. Eq. (impl-corr) at that window with the window-local phase, on the whole grid.  A
 * window is complete once its last x sample has been pushed; completed windows wait in a
 * device ring of `capacity` windows (FP32, F * A * nlags * 8 bytes each) for
 * cyc_read_windows ([nwin][F][A][nlags] complex FP64).  A push that would complete more
 * windows than the ring has room for fails with CYC_EAGAIN before doing anything.  Pushes
 * are folded in batches as for cyc_create_full, and the stream keeps its running estimate
 * (cyc_read) as well.
 *   A          power of two in [2, 4096] (the window length and the FFT size)
 *   hop        1 .. 2^30 samples between window starts (hop = 1: a window per sample, the
 *              block's own output rate)
 *   capacity   1 .. 2^20 windows (the ring at most 64 GB)
 *   precision  must be CYC_P_FP32 (FP32 lag products and FFT); else CYC_EINVAL
 * cyc_save / cyc_load / cyc_sums return CYC_ENOTSUP.
 */
CYC_API int cyc_create_full_window(const cyc_params* p, int32_t A, int64_t hop, int64_t capacity, int cross,
                                   cyc_stream** out);

/*
 * cyc_read_windows: move up to max_win completed windows, oldest first, out of the ring into
 * out ([nwin][F][nalphas][nlags] complex FP64, host or device memory of the stream's device,
 * synchronous).  *nwin receives how many were written (0 when none are complete), *first_k
 * the index k of the first of them.  CYC_EINVAL on a stream not made by cyc_create_window or
 * cyc_create_full_window.
 */
CYC_API int cyc_read_windows(cyc_stream* s, double* out, int64_t max_win, int64_t* nwin, int64_t* first_k);

/*
 * cyc_read_spectrum: cyclic spectra of the current estimate (the cyclic correlogram; the
 * paper names cyclic spectra as its next step, Sec. 6): for every form and cycle frequency,
 *   S[f][a][q] = sum_l w(m_l) R[f][a][l] exp(-j 2 pi f_q m_l),   f_q = -1/2 + q/Q, q < Q,
 * over the stream's (signed) lags m_l, with R as cyc_read returns it.  taper 0: w = 1;
 * taper 1: the Hann lag window w(m) = 0.5 + 0.5 cos(pi m / (Mmax + 1)), Mmax = max |m_l|.
 * out: [F][nalphas][Q] complex FP64, host or device memory of the stream's device;
 * synchronous.  Q in [1, 65536]; CYC_ENODATA when N_eff is 0.  Device scratch of
 * nlags * Q + F * nalphas * Q complex doubles is kept with the stream after the first call.
 */
CYC_API int cyc_read_spectrum(cyc_stream* s, int32_t Q, int32_t taper, double* out);

/*
 * cyc_detect: cycle-frequency estimation (the paper's next step, Sec. 6) on the stream's
 * current estimate R (as cyc_read would return it), per form, reading the stream's cycle-
 * frequency list as a circular grid in the order given (the uniform grid -1/2 + k/A is the
 * intended use).  A constant-false-alarm rule:
 *   s(a)   = max over lags m of |R^a(m)|^2; 0 for the conventional form at a = 0 (mod 1, in
 *            the fixed point of cyc_phase_increment) of a one-input stream, whose entry is
 *            the signal's power
 *   nu(a)  = median of s over the list positions a +- 2 .. a +- win (indices modulo nalphas;
 *            the mean of the two middle values of the 2 (win - 1))
 *   flags[f][a] bit 1 (value 2): s(a) >= s(a - 1) and s(a) >= s(a + 1)  (a local maximum)
 *   flags[f][a] bit 0 (value 1): a local maximum with s(a) > kappa * nu(a)  (detected)
 *   ratio[f][a] = s(a) / nu(a) (nu floored at 1e-300), FP32
 * kappa > 0 (8.4 gives about 1e-3 false alarms per signal on 512 a x 64 lags x 2 forms of
 * the serving mix of modulated signals); win in [2, 32] (16 is the usual choice).  flags
 * ([F][nalphas] bytes) and ratio ([F][nalphas] floats, may be NULL) are host or device
 * memory of the stream's device; *ndetected (optional) receives the number of detections.
 * Synchronous.  CYC_ENODATA when N_eff is 0.  Device scratch of F * nalphas * 13 bytes is
 * kept with the stream after the first call.
 */
CYC_API int cyc_detect(cyc_stream* s, double kappa, int32_t win, uint8_t* flags, float* ratio, int32_t* ndetected);

/*
 * cyc_push: append nsamples samples (interleaved complex64) to the stream and add their
 * contribution to the FP64 running sums (Sec. 4 Eq. (impl-corr), accumulated over the
 * whole stream).  The samples are staged at once; their projection runs when max_chunk
 * samples are staged (several short pushes share one launch) or when a call reads the
 * stream (cyc_read, cyc_sync, ...).  on_device != 0: `chunk` is device memory of the
 * stream's device, read in stream order -- keep it unchanged until the next cyc_read /
 * cyc_sync.
 * on_device == 0: host memory; pageable memory is consumed before return, page-locked
 * memory is read in stream order like device memory -- on a copy stream of the handle's own,
 * so that the copy of one push overlaps the projection of the previous one (the projection
 * waits for its copy).  nsamples == 0 is a no-op.
 */
CYC_API int cyc_push(cyc_stream* s, const void* chunk, int64_t nsamples, int on_device);

/* cyc_push_xy: as cyc_push for a stream made by cyc_create_xy: nsamples samples of x and
 * the same nsamples of y (both interleaved complex64, both on the device or both on the
 * host).  cyc_push on such a stream, or cyc_push_xy on a one-input stream: CYC_EINVAL. */
CYC_API int cyc_push_xy(cyc_stream* s, const void* x_chunk, const void* y_chunk, int64_t nsamples, int on_device);

/*
 * cyc_read: wait for the stream's work, then write R = sums / N_eff (layout above) to
 * `out`, which may be host or device memory of at least F * nalphas * nlags * 16 bytes
 * (device memory 16-byte aligned: CYC_EINVAL otherwise).  A host `out` is filled from a
 * page-locked buffer of F * nalphas * nlags * 16 bytes (up to 64 MB) that the handle keeps
 * after its first host read; for Set-mode streams the read kernel writes the result there
 * through the buffer's device address (no separate copy).
 * *n_eff (optional) receives N_eff.  CYC_ENODATA when N_eff == 0 (out untouched).
 */
CYC_API int cyc_read(cyc_stream* s, double* out, int64_t* n_eff);

/* cyc_sync: wait until all work queued by this stream has finished. */
CYC_API int cyc_sync(cyc_stream* s);

/* cyc_reset: drop all samples and sums (parameters kept).  The zeroing of the sums is
 * queued on the stream's CUDA stream; the call does not wait for it.  FP32 streams with at
 * most 32 distinct cycle frequencies (and no windows, no Full mode) queue nothing here: their
 * next projection writes its totals instead of adding them, or the first call that reads the
 * sums (cyc_read, cyc_sums, cyc_save, ...) zeroes them first. */
CYC_API int cyc_reset(cyc_stream* s);

/* cyc_destroy: free the handle and its device memory (NULL is a no-op). */
CYC_API int cyc_destroy(cyc_stream* s);

/*
 * cyc_save / cyc_load: the whole stream state (sample count, N_eff, the carried tail of
 * up to M samples, the FP64 sums) as an opaque host blob.  cyc_save with buf == NULL
 * stores the needed size in *len.  cyc_load restores into a handle created with the
 * same lags, alphas, forms and n0 (CYC_EINVAL otherwise); pushing after a load gives
 * the same result as never having stopped.
 */
CYC_API int cyc_save(cyc_stream* s, void* buf, size_t* len);
CYC_API int cyc_load(cyc_stream* s, const void* buf, size_t len);

/*
 * cyc_info: sizes of a handle.  Any pointer may be NULL.
 *   forms: number of forms F; nunique: distinct a mod 1 actually computed;
 *   total: samples pushed; n_eff: committed terms.
 */
CYC_API int cyc_info(cyc_stream* s, int* forms, int* nunique, int64_t* total, int64_t* n_eff);

/*
 * cyc_profile: enable (1) or disable (0) timing of this stream's projection kernel with
 * CUDA events recorded on its CUDA stream around every launch.
 * cyc_profile_read: totals since the previous cyc_profile_read (waits for the stream):
 *   proj_ms        summed device time of the projection launches (0 when disabled)
 *   proj_launches  projection launches
 *   kernels        all kernel launches made by this stream (projection, sum update, read)
 * Any output pointer may be NULL.
 */
CYC_API int cyc_profile(cyc_stream* s, int enable);
CYC_API int cyc_profile_read(cyc_stream* s, double* proj_ms, int64_t* proj_launches, int64_t* kernels);

/*
 * cyc_sums / cyc_set_n_eff: the stream's raw running sums for merging time shards of one
 * stream across GPUs (one process per GPU).  Because the phase uses the absolute sample
 * index, shard r of a stream -- a handle with the same lags, alphas, forms and precision,
 * start index n0 + a_r, fed samples [a_r, b_r + M) of the stream -- holds exactly the sums
 * of the committed terms [a_r, b_r); the whole stream's sums are their SUM and its N_eff
 * the SUM of the counts.
 *   cyc_sums      waits for the stream's work and returns the device address of its FP64
 *                 running sums (*nvalues complex values, interleaved re, im; an internal
 *                 layout that is the same for handles created with the same parameters) and
 *                 its N_eff.  The array stays the handle's; a caller may add into it in place
 *                 (e.g. a SUM all-reduce across the ranks' handles) while no push is queued.
 *   cyc_set_n_eff sets the count cyc_read (and cyc_read_spectrum, cyc_detect) divides by:
 *                 after merging, the total of the ranks' counts.  The handle then describes
 *                 the merged stream for reading; pushing more samples into it afterwards does
 *                 not continue that stream (cyc_reset first).
 * CYC_ENOTSUP for windowed streams and for Full-mode streams (cyc_create_full).
 */
CYC_API int cyc_sums(cyc_stream* s, double** sums, int64_t* nvalues, int64_t* n_eff);
CYC_API int cyc_set_n_eff(cyc_stream* s, int64_t n_eff);

/*
 * cyc_set_wait_budget: how long (SM clock cycles) each bounded wait inside the stream's
 * tensor-core projection kernel waits for a producer, a copy or the tensor core before it
 * gives up; 0 restores the default of 2e9 (about a second at 2 GHz).  A wait that gives up
 * makes every other wait of the kernel give up at once, the kernel winds down (in-flight
 * copies and tensor-core work are waited for), and the next cyc_sync / cyc_read reports
 * CYC_ETIMEDOUT; the sums are then unreliable (cyc_reset).  Applies to launches queued
 * after the call; the FP32 paths have no waits.  cycles in [0, 2^40].
 * Test hook: the environment variable CYC_TEST_WITHHOLD_ARRIVAL=1 at stream creation makes
 * the tensor-core kernel of that stream leave one producer arrival out, so that a wait
 * runs out -- the only way to exercise this path without a fault; never set it otherwise.
 */
CYC_API int cyc_set_wait_budget(cyc_stream* s, int64_t cycles);

/*
 * cyc_phase_increment: the fixed-point form in which a stream holds cycle frequency a:
 * *phi = round(a * 2^64) mod 2^64, so the phase of sample n is phi * n mod 2^64 in units
 * of 2^-64 cycles (exact for any n; Sec. 2's exp(-j 2 pi a~ n)).  Host-only, no GPU
 * needed.  CYC_EINVAL if a is not finite or phi is NULL.
 */
CYC_API int cyc_phase_increment(double a, uint64_t* phi);

/* ======================================================================================
 * Serving: many concurrent streams, continuously batched.
 *
 * A server owns a device, a memory budget and an engine thread.  Streams are opened
 * (admitted only if their device memory fits the budget and a slot is free), chunks are
 * submitted from any thread, and the engine repeatedly forms a batch from every open
 * stream that has new samples: the new committed n-range of each stream becomes work
 * items (up to 512 cycle frequencies -- 256 pairs a, -a -- x 128 columns x at most
 * item_samples terms) for one
 * persistent tensor-core kernel, followed by an FP64 fold into each stream's sums, both
 * replayed from a captured CUDA graph.  Chunks that arrive while a batch runs join the
 * next one, so streams of very different rates share the GPU.  Each stream computes the
 * same estimate as a cyc_stream with the same parameters (Sec. 4, Eq. (impl-corr)).
 * ====================================================================================== */
typedef struct cyc_server cyc_server;

typedef struct cyc_server_params {
    int32_t  max_streams;   /* open streams at most (slots); 0 selects 256 */
    int32_t  precision;     /* CYC_P_BF16X3 or CYC_P_FP16 */
    uint64_t mem_budget;    /* device bytes for stream state; 0 selects half the free memory */
    int64_t  ring_samples;  /* per-stream sample ring (rounded up to a power of two); 0: 1 << 22 */
    int32_t  max_items;     /* work items per batch; 0 selects 1024 (512 KiB of partials each) */
    int64_t  item_samples;  /* committed terms per work item at most; 0 selects 65536 */
    int32_t  device;        /* CUDA device ordinal */
} cyc_server_params;

/* One finished chunk: its contribution is in the stream's sums (everything that the
 * samples up to the chunk's end allow; the last M samples still wait for the next chunk).
 * Times are host monotonic seconds: when cyc_server_submit returned, and when the engine
 * saw the batch that completed the chunk finish. */
typedef struct cyc_done {
    int32_t  sid;
    int32_t  status;        /* 0 or a CYC_E* code */
    uint64_t tag;
    int64_t  nsamples;
    double   submit_s;
    double   done_s;
} cyc_done;

/* Create a server (engine thread started) / stop it and free everything. */
CYC_API int cyc_server_create(const cyc_server_params* p, cyc_server** out);
CYC_API int cyc_server_destroy(cyc_server* srv);

/* Open a stream (lags >= 0, max lag <= 2560; arrays copied).  CYC_EAGAIN when no slot is
 * free or its device memory would exceed the budget: retry after a close. */
CYC_API int cyc_server_open(cyc_server* srv, const int32_t* lags, int nlags, const double* alphas,
                            int nalphas, int conj_flag, int64_t n0, int* sid);

/* Queue nsamples host samples (interleaved complex64) of stream sid; they are on the
 * device when the call returns, so the buffer may be reused.  CYC_EAGAIN when the
 * stream's ring has no room yet (earlier chunks still being processed): retry. */
CYC_API int cyc_server_submit(cyc_server* srv, int sid, const void* chunk, int64_t nsamples, uint64_t tag);

/* Up to `max` finished chunks, oldest first, without waiting; *ndone receives the count. */
CYC_API int cyc_server_poll(cyc_server* srv, cyc_done* done, int max, int* ndone);

/* Wait until every submitted chunk is finished (CYC_ETIMEDOUT after timeout_s seconds). */
CYC_API int cyc_server_drain(cyc_server* srv, double timeout_s);

/* R of stream sid (layout and meaning as cyc_read; host or device `out`), after all of its
 * submitted samples are in the sums.  CYC_ENODATA when N_eff == 0. */
CYC_API int cyc_server_read(cyc_server* srv, int sid, double* out, int64_t* n_eff);

/* Close stream sid once its work is done; its memory returns to the budget. */
CYC_API int cyc_server_close(cyc_server* srv, int sid);

/* Counters since creation: batches run, work items run, device busy milliseconds
 * (sum of batch durations), bytes held by open streams.  Any pointer may be NULL. */
CYC_API int cyc_server_stats(cyc_server* srv, int64_t* batches, int64_t* items, double* busy_ms,
                             uint64_t* bytes_held);

/* ======================================================================================
 * Learned cycle-frequency proposer.
 *
 * The paper's future work is the estimation of cycle frequencies themselves (Sec. 6);
 * here a small net proposes, from cheap spectra, which cycle frequencies of the 512-bin
 * grid a = -1/2 + k/512 carry lines, so that the estimator (Sec. 4) runs at those few
 * instead of the full grid -- and falls back to the full grid when it is unsure.
 *
 * Features (cyc_features): for each signal, Welch-averaged periodograms (16 segments of
 * 4096 samples, Hann window) of x, x^2 and the lag products x[n+d] conj(x[n]) for
 * d = 0, 1, 2, 3, 4, 6, 8, 12, 16 -- spectra whose lines are the conjugate and the
 * conventional cycle frequencies (Sec. 2) -- as log10, bin j at frequency -1/2 + j/4096,
 * each channel standardised; FP16 [nsig][11][4096].
 * Net: circular 1-D convolutions, kernel 9, 11 -> 64 -> 64 -> 64 -> 2 channels, ReLU after
 * the first three, mean over groups of 8 bins: logits [B][form][512] (CONV, CONJ).  FP16
 * weights and activations, FP32 sums (the forward convolutions on the tensor cores);
 * parameters as one flat FP32 vector (W1 b1 W2 b2 W3 b3 W4 b4, W[out][in][9]) of
 * cyc_net_nparams() values.  The forward's bounded device waits report CYC_ETIMEDOUT from
 * cyc_net_forward, cyc_net_gradients, cyc_net_train_step and cyc_propose.
 * Training minimises the mean binary cross-entropy with logits (positives weighted by
 * pos_weight) against labels [B][form][512] in {0, 1}, with Adam (0.9, 0.999, 1e-8).
 * ====================================================================================== */
typedef struct cyc_net cyc_net;

/* params: cyc_net_nparams() FP32 values, or NULL for seeded He-normal weights, zero biases. */
CYC_API int cyc_net_create(const float* params, uint64_t seed, int device, cyc_net** out);
CYC_API int cyc_net_destroy(cyc_net* n);
CYC_API int cyc_net_nparams(void);
CYC_API int cyc_net_get_params(cyc_net* n, float* out);           /* host, nparams floats */
CYC_API int cyc_net_set_params(cyc_net* n, const float* params);  /* host; resets Adam state */

/* Features of nsig signals stored back to back in device memory (signal s at x + s*T
 * complex64 samples, T >= 65552; the first 65552 are used) into device FP16 `feats`. */
CYC_API int cyc_features(const void* x, int64_t T, int nsig, void* feats);

/* Logits of B feature sets (device pointers): logits [B][2][512] FP32. */
CYC_API int cyc_net_forward(cyc_net* n, const void* feats, int B, float* logits);

/* Loss and parameter gradients for a batch (device feats and labels); grads (host,
 * nparams floats) and loss (host) may be NULL.  No update. */
CYC_API int cyc_net_gradients(cyc_net* n, const void* feats, const float* labels, int B, float pos_weight,
                              float* grads, float* loss);

/* One Adam step on a batch; *loss (host, optional) receives the batch loss before the step. */
CYC_API int cyc_net_train_step(cyc_net* n, const void* feats, const float* labels, int B, float lr,
                               float pos_weight, float* loss);

/* Proposals for one signal (host or device, >= 65552 samples): the k most likely grid
 * cycle frequencies of each form into alphas_conv[k] and alphas_conj[k] (host), the
 * confidence (1 - the predicted probability of the most likely bin left out, the lower of
 * the two forms), and *used_fallback = 1 when the confidence is below tau: the caller
 * should then run the full grid. */
CYC_API int cyc_propose(cyc_net* n, const void* x, int64_t T, int on_device, int k, float tau,
                        double* alphas_conv, double* alphas_conj, float* conf, int* used_fallback);

/*
 * cyc_estimate_static: a one-shot estimate over x[0..T) that allocates no memory at all.
 * The paper has no counterpart; it exists for callers that cannot call cudaMalloc when
 * they need an estimate -- a real-time signal-processing callback that must not
 * allocate (device allocation can synchronise the whole device and take unbounded time),
 * or a plug-in whose host application has already reserved the device memory in its
 * own pool.
 *   x        device (or managed) memory of the current device, 8-byte aligned: T interleaved
 *            complex64 samples
 *   lags     non-negative lags (the signed lags of cyc_params are not accepted here:
 *            CYC_EINVAL); alphas, conj_flag, n0 as in cyc_params (host arrays, read before
 *            return)
 *   out      device (or managed) memory of the current device, 16-byte aligned,
 *            F * nalphas * nlags * 16 bytes: R as interleaved FP64 [form][alpha][lag] (same
 *            layout and value as cyc_read)
 *   n_eff    optional, receives T - max(lags) (or 0)
 *   cuda_stream   cudaStream_t the work is queued on (NULL = legacy default stream); the
 *            call returns once the work is queued -- the tables travel as kernel launch
 *            parameters, so no copy from host memory makes it wait for the stream --;
 *            synchronise that stream before reading `out`.
 * It runs the FP32 projection with its scratch -- the cycle-frequency and column tables
 * and the FP32 partial sums -- in one fixed file-scope device array of about 8.1 MiB,
 * which every GPU that loads it holds until the process exits.  CUDA loads the library's
 * device code lazily by default, so the array is brought onto a device, and its device
 * address looked up, by the first call on that device: a caller whose host application
 * later reserves the device memory, or that captures work into a CUDA graph, must make
 * one call (of any valid size) beforehand, or run with CUDA_MODULE_LOADING=EAGER.
 * Limits: nalphas <= 4096, nlags * F <= 2048 and nalphas * nlags * F <= 2^20; larger
 * requests fail with CYC_EINVAL and queue nothing.  Duplicate cycle frequencies are
 * computed separately.  Every call shares the array: calls whose GPU work can overlap
 * (different CUDA streams) race and give wrong results; calls on one stream are ordered
 * and safe.  CYC_ENODATA when T <= max(lags).
 */
CYC_API int cyc_estimate_static(const void* x, int64_t T, const int32_t* lags, int nlags,
                                const double* alphas, int nalphas, int conj_flag, int64_t n0,
                                double* out, int64_t* n_eff, void* cuda_stream);

/* Error text for a status code, and the calling thread's last detailed message. */
CYC_API const char* cyc_strerror(int code);
CYC_API const char* cyc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CYC_H */
