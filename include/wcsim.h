/*
 * wcsim.h -- C-ABI of the GB300 LArTPC signal-simulation library (libwcsim.so).
 *
 * The library computes the signal term of Eq. 1 (Sec. 2): electron clouds drift to a wire
 * plane (Fig. 2), each is rasterized into a small Gaussian patch over impact position x
 * time tick, the patches are scatter-added into the plane's grid S(t, x) (Sec. 2.1.1,
 * "rasterization" and "scatter adding"), and the grid is convolved with the detector
 * response in the frequency domain (Eq. 2) to give per-wire waveforms M(t, x).
 *
 * Conventions shared by every call
 *  - Units: mm, microseconds, electrons; diffusion constants in cm^2/s.
 *  - Arrays passed to compute calls are DEVICE pointers owned by the caller, except where a
 *    call says otherwise.  The plane object owns its response copy and all scratch.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls only enqueue
 *    work on it and never synchronize the host, so they return before the work is done.
 *  - Every call returns a wcsim_status and never aborts; wcsim_last_error() gives a
 *    thread-local message for the last failing call of the calling thread.
 *  - Depo values are checked on the device: a depo with a NaN/Inf field, negative drift time
 *    or negative charge contributes nothing and raises a flag that wcsim_plane_check()
 *    reports.  A depo that lies (partly or wholly) outside the grid contributes only its
 *    in-grid bins; that is not an error.
 *  - Layouts: grid S is float32 [n_wires * n_imp][n_ticks], row r = w * n_imp + j covering
 *    pitch coordinate [p0 + r d, p0 + (r+1) d), d = pitch / n_imp; tick k covers
 *    [t0 + k tick, t0 + (k+1) tick).  Waveforms are float32 [n_wires][n_ticks].  Response
 *    spectra are complex64 (interleaved re, im float32) [n_imp][n_fw][n_ft].
 */
#ifndef WCSIM_H
#define WCSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WCSIM_OK = 0,
    WCSIM_EINVAL = 1,        /* null pointer, NaN / out-of-range scalar parameter */
    WCSIM_ESHAPE = 2,        /* unsupported or inconsistent sizes */
    WCSIM_ENOMEM = 3,        /* a device allocation failed */
    WCSIM_ECUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    WCSIM_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    WCSIM_EDEVICE_CHECK = 6  /* the device flagged invalid depo values (see plane_check) */
} wcsim_status;

/* Opaque plane object: geometry, parameters, response (Hermitian half, pre-scaled) and
 * scratch.  Library-owned; create/destroy only. */
typedef struct wcsim_plane wcsim_plane;

/* Plane geometry (Sec. 2.1.1: patches on an impact-position x tick grid). */
typedef struct {
    int32_t n_wires;   /* wires in the plane, >= 1 */
    int32_t n_imp;     /* impact positions per wire pitch, >= 1 */
    int32_t n_ticks;   /* time ticks in the frame, >= 1 */
    int32_t reserved;  /* must be 0 */
    double pitch_mm;   /* wire pitch, > 0 */
    double p0_mm;      /* pitch coordinate of the lower edge of row 0 */
    double tick_us;    /* tick length, > 0 */
    double t0_us;      /* time of the lower edge of tick 0 */
} wcsim_geometry;

/* Drift, diffusion, lifetime, truncation and fluctuation parameters.  The paper gives no
 * formulas (Fig. 2 only); the library uses t_a = t + t_d, Q' = Q exp(-t_d / lifetime),
 * sigma_T = sqrt(2 D_T t_d) [mm], sigma_t = sqrt(2 D_L t_d) / v [us]. */
typedef struct {
    double v_mm_per_us;  /* drift speed, > 0 */
    double DL_cm2_s;     /* longitudinal diffusion constant, >= 0 */
    double DT_cm2_s;     /* transverse diffusion constant, >= 0 */
    double lifetime_us;  /* electron lifetime, > 0 (may be +inf) */
    double nsigma;       /* patch half-width in sigmas, > 0 */
    int32_t fluctuate;   /* per-bin charge fluctuation (Sec. 4.3.1, 4.3.2, Table 1): 0 the
                            mean; 1 the normal approximation to Binomial(Q', mean / Q');
                            2 the exact Binomial(rint Q', mean / Q') drawn by inversion of
                            its CDF (bins whose variance exceeds 65536 electrons^2 take the
                            normal approximation).  0, 1 or 2, else WCSIM_EINVAL */
    uint32_t plane_id;   /* 4th Philox counter word */
    uint64_t seed;       /* Philox key (lo, hi words) */
    int32_t renormalize; /* 1: each axis' weights divided by their sum over the n-sigma
                            window before it is clipped to the grid, so that a patch inside
                            the grid carries Q' exactly and charge beyond the grid's border
                            stays lost (the reductions of the paper's Sec. 4.3.2 hint at a
                            normalisation); 0: the truncated tails are lost.  0 or 1, else
                            WCSIM_EINVAL */
    int32_t reserved;    /* must be 0 */
} wcsim_drift_params;

/* Depos, structure of arrays, DEVICE pointers (8-byte aligned), n entries each. */
typedef struct {
    const double* p_mm;       /* pitch-direction position */
    const double* t_us;       /* deposition time */
    const double* tdrift_us;  /* drift time to this plane, >= 0 */
    const float* q;           /* charge (electrons), >= 0 */
    const uint32_t* id;       /* depo id; keys the fluctuation random stream */
    int64_t n;                /* number of depos, >= 0 */
} wcsim_depos;

/* Create a plane.  Defined by Eq. 2: `resp_c64` is the pre-calculated response
 * R(omega_t, omega_x) per impact position, DEVICE complex64 [n_imp][n_fw][n_ft]; it is
 * read during this call (stream-ordered) and not retained.  n_fw >= n_wires and
 * n_ft >= n_ticks set the FFT size (the frame is zero-padded; equal sizes give circular
 * convolution); 0 means "same as the frame".  Each of n_fw, n_ft must factor into 2, 3,
 * 5 and 7, n_ft <= 13500 and n_fw <= 8192.  Allocates device memory
 * (response half-spectrum, grid and spectrum scratch): WCSIM_ENOMEM if that fails.
 * On success *out receives the plane; on failure *out is set to NULL. */
wcsim_status wcsim_plane_create(const wcsim_geometry* geom, const void* resp_c64,
                                int32_t n_fw, int32_t n_ft, const wcsim_drift_params* params,
                                void* stream, wcsim_plane** out);

/* Replace the drift parameters (e.g. while fitting D_L, D_T, lifetime).  Host-only. */
wcsim_status wcsim_plane_set_params(wcsim_plane* plane, const wcsim_drift_params* params);

/* Replace the response spectra (same shape as at create), stream-ordered. */
wcsim_status wcsim_plane_set_response(wcsim_plane* plane, const void* resp_c64, void* stream);

/* Rasterization + scatter adding (Sec. 2.1.1): drift every depo, rasterize it into its
 * truncated Gaussian patch (bins meeting [mu - n sigma, mu + n sigma], weights from erf
 * bin-edge integrals, optional fluctuation) and ADD the patch into `grid` (DEVICE float32
 * [n_wires * n_imp][n_ticks]; the caller zeroes it).  Additions are atomic, so the
 * summation order, and the last bits of overlapping bins, vary from run to run. */
wcsim_status wcsim_rasterize(wcsim_plane* plane, const wcsim_depos* depos, float* grid,
                             void* stream);

/* Eq. 2: M = IFFT2( sum_j R_j . FFT2(S_j) ), S_j = rows j, j + n_imp, ... of `grid`
 * (DEVICE float32 [n_wires * n_imp][n_ticks], read only), real part, cropped to the frame,
 * written to `wave` (DEVICE float32 [n_wires][n_ticks]).  Uses the plane's scratch, so two
 * calls on one plane must not run concurrently. */
wcsim_status wcsim_convolve(wcsim_plane* plane, const float* grid, float* wave, void* stream);

/* Whole signal simulation: zero the plane's grid, rasterize `depos` into it, convolve into
 * `wave` (DEVICE float32 [n_wires][n_ticks]), plus the plane's noise (Eq. 1) if it has
 * one.  Same concurrency rule as wcsim_convolve. */
wcsim_status wcsim_run(wcsim_plane* plane, const wcsim_depos* depos, float* wave,
                       void* stream);

/* wcsim_run with the frame read out as ADC codes (Eq. 1 reads M as "an ADC value"; the paper
 * gives no digitizer): `adc` (DEVICE uint16 [n_wires][n_ticks]) receives
 * clamp(floor(fl(fl(gain M) + pedestal) + 1/2), 0, 2^bits - 1) with the plane's digitizer
 * settings, each step one correctly rounded FP32 operation on the float frame wcsim_run
 * would write.  WCSIM_EINVAL if no digitizer was set. */
wcsim_status wcsim_run_adc(wcsim_plane* plane, const wcsim_depos* depos, uint16_t* adc,
                           void* stream);

/* wcsim_run for a fit: `residual` (DEVICE float32 [n_wires][n_ticks]) receives M - target,
 * each value one FP32 subtraction of the frame wcsim_run would write from `target` (DEVICE
 * float32, same layout, read only), the dL/dM of L = 1/2 |M - target|^2 that
 * wcsim_run_backward takes; if `loss` (DEVICE double) is not NULL it is set to L (squares
 * summed in FP32 within each warp's share of two wires, those sums in FP64).  residual and target
 * must not overlap.  A forward like wcsim_run for wcsim_plane_set_reuse_forward.
 * WCSIM_EINVAL if target or residual is NULL. */
wcsim_status wcsim_run_residual(wcsim_plane* plane, const wcsim_depos* depos, const float* target,
                                float* residual, double* loss, void* stream);

/* Digitizer of wcsim_run_adc: gain (ADC counts per unit of M), pedestal (counts), bits in
 * 1..16.  WCSIM_EINVAL for bits out of range or a non-finite gain or pedestal. */
wcsim_status wcsim_plane_set_digitizer(wcsim_plane* plane, float gain, float pedestal,
                                       int32_t bits);

/* Bins each depo covers, as decided by wcsim_rasterize: `out` DEVICE int32 [n][4] =
 * (r_lo, r_hi, k_lo, k_hi) inclusive, or (-1, -1, -1, -1) when the depo covers nothing. */
wcsim_status wcsim_windows(wcsim_plane* plane, const wcsim_depos* depos, int32_t* out,
                           void* stream);

/* Per-depo and global gradients of a scalar loss L (see wcsim_run_backward).  Every
 * pointer is DEVICE memory and may be NULL (that output is then skipped).  Per-depo arrays
 * have n entries, float32; dglobal has 3 doubles.  Units follow the inputs: dq per
 * electron, dp per mm, dt per us, dsigma_L and dsigma_T per mm (sigma_L = sqrt(2 D_L t_d),
 * the longitudinal spread in mm before division by v; sigma_T = sqrt(2 D_T t_d)), and
 * dglobal = (dL/dD_L per cm^2/s, dL/dD_T per cm^2/s, dL/dlifetime per us). */
typedef struct {
    float* dq;
    float* dp;
    float* dt;
    float* dsigma_L;
    float* dsigma_T;
    double* dglobal;
} wcsim_depo_grads;

/* Adjoint of wcsim_convolve (Eq. 2): given G = dL/dM (DEVICE float32 [n_wires][n_ticks])
 * and the grid S the forward used (DEVICE float32 [n_wires * n_imp][n_ticks]), write
 * dgrid = dL/dS = Re IFFT2(conj(R_j) . FFT2(G)) per impact row (DEVICE float32, same shape
 * as S; may alias `grid`) and, if grad_resp is not NULL, dL/dR_j = conj(FFT2(S_j)) .
 * FFT2(G) / (n_fw n_ft) (DEVICE complex64 [n_imp][n_fw][n_ft], the PyTorch convention for
 * complex gradients: dL/dRe + i dL/dIm).  Any spectrum size the plane accepts (one warp per
 * time frequency for n_fw = 32 M with M in {4, 8, 15, 16, 20, 24, 25, 30}, the block-level
 * engine otherwise).  Uses the plane's scratch. */
wcsim_status wcsim_convolve_adjoint(wcsim_plane* plane, const float* grad_wave, const float* grid,
                                    float* dgrid, void* grad_resp_c64, void* stream);

/* Adjoint of rasterization + drift on the mean path (no fluctuation), with each depo's bin
 * window held fixed: given dgrid = dL/dS, write the gradients of L with respect to each
 * depo's charge, pitch position, time, sigma_L, sigma_T, and the sums over depos for D_L,
 * D_T and the lifetime (dglobal is overwritten).  sigma = 0 (t_d = 0) depos get zero sigma
 * and position gradients; D_L or D_T = 0 give no gradient for that constant (the
 * derivative of sqrt(2 D t) is unbounded there). */
wcsim_status wcsim_rasterize_adjoint(wcsim_plane* plane, const wcsim_depos* depos,
                                     const float* dgrid, wcsim_depo_grads* grads, void* stream);

/* Backward pass of wcsim_run for L with dL/dwave = grad_wave: recompute the grid on the
 * mean path (fluctuation off: the gradient is that of the expected waveform; skipped, with
 * the time-axis FFT of the grid, when wcsim_plane_set_reuse_forward applies), run
 * wcsim_convolve_adjoint and wcsim_rasterize_adjoint.  grad_resp_c64 as in
 * wcsim_convolve_adjoint (NULL skips it).  Uses the plane's scratch and grid. */
wcsim_status wcsim_run_backward(wcsim_plane* plane, const wcsim_depos* depos,
                                const float* grad_wave, wcsim_depo_grads* grads,
                                void* grad_resp_c64, void* stream);

/* enable = 1: wcsim_run_backward reuses the time-axis spectra of the grid (the FFT of S that
 * the forward of Eq. 2 computes) when the plane's previous compute call was a successful
 * wcsim_run or wcsim_run_adc on the same depo arrays (same pointers and count) with the same
 * parameters and fluctuate = 0, instead of recomputing the mean-path grid and its spectra.
 * The caller promises not to change the depo arrays between the two calls (as autograd keeps
 * a forward's activations for its backward): the arrays are recognised by their pointers and
 * count only, so arrays freed and reallocated at the same addresses with other contents would
 * be taken for the forward's.  Any other compute call on the plane drops the spectra.
 * enable = 2: as 1, and such a forward's wire pass also writes the 2D spectra of S (the wire
 * FFT of every impact's time-axis spectra, n_imp * n_fw * 4 ceil((n_ft / 2 + 1) / 4) complex
 * values, allocated here) when the plane runs the one-warp wire pass (n_fw = 32 M; otherwise
 * 2 acts as 1); a backward that wants dL/dR then reads them instead of transforming the
 * spectra of S again, which moves the cost of those transforms into one extra write in the
 * forward.  enable = 0 (the default): the backward always recomputes.  Calling it (with any
 * value) drops any kept spectra, and a value other than 2 frees the 2D spectra's buffer
 * (synchronising the device).  WCSIM_EINVAL for other values, WCSIM_ENOMEM if the buffer
 * cannot be allocated.  Host-only. */
wcsim_status wcsim_plane_set_reuse_forward(wcsim_plane* plane, int32_t enable);

/* Forward variant of wcsim_run / wcsim_run_adc.  fused = 0 (the default): the flow of Sec.
 * 2.1.1, rasterize and scatter-add into the plane's grid S, then Eq. 2 on the grid.
 * fused = 1: the depos are binned by wire, and each time-axis transform CTA rasterizes the
 * depos that reach its two grid rows straight into shared memory, so the grid is never
 * written to device memory (this pays on sparse frames, where the plain transform would read
 * a mostly empty grid; wcsim_plane_autotune times both).  Both give the same frame up to
 * floating-point summation order.  The exact binomial (fluctuate = 2) always takes the plain
 * flow.  The fused flow keeps depo binning scratch (about 230 bytes per depo), allocated by
 * the first wcsim_run with more depos than before.  WCSIM_EINVAL for fused outside 0..1.
 * Host-only. */
wcsim_status wcsim_plane_set_forward(wcsim_plane* plane, int32_t fused);

/* Rasterization tile of this plane (the autotuner's first choice, settable by hand):
 * depos_per_block depos per CTA of 256 threads, each rasterized by lanes_per_depo lanes.
 * Supported: (32, 8), (64, 8), (128, 8), (256, 8), (64, 16), (128, 16), (256, 16),
 * (64, 32), (128, 32), (256, 32); WCSIM_EINVAL otherwise.  Results are unchanged up to summation order.
 * Host-only. */
wcsim_status wcsim_plane_set_raster_tile(wcsim_plane* plane, int32_t depos_per_block,
                                         int32_t lanes_per_depo);

/* Choices and best times (ms) found by wcsim_plane_autotune. */
typedef struct {
    int32_t time_radix[8];     /* radices of the time-axis FFT plan, in pass order, 0-padded */
    int32_t rows_variant;      /* time-axis forward kernel: 0 direct loads, 1 bulk-staged */
    int32_t wire_variant;      /* wire pass: 0 one warp per time frequency, 1 block-level */
    int32_t depos_per_block;   /* rasterization tile: depos per CTA, 32..256 */
    int32_t candidates_timed;  /* configurations timed */
    float ms_rasterize, ms_rows, ms_wire;
    int32_t forward_fused;     /* forward variant kept (wcsim_plane_set_forward) */
    float ms_forward_plain, ms_forward_fused;   /* whole forward, each variant (0: not timed) */
    int32_t lanes_per_depo;    /* rasterization tile: lanes that rasterize one depo, 8..32 */
} wcsim_tune_report;

/* Time the kernel variants of this plane on `depos` (DEVICE) and keep the fastest: the
 * rasterization tile (depos per CTA, lanes per depo), the radices and order of the time-axis FFT plan (the cheapest
 * plans with the fewest passes), the time-axis forward kernel, the wire-pass kernel and the
 * forward variant (plain or fused, wcsim_plane_set_forward).
 * Results are unchanged up to floating-point rounding order.  Synchronizes `stream`,
 * allocates temporary plan tables, overwrites the plane's scratch; report may be NULL. */
wcsim_status wcsim_plane_autotune(wcsim_plane* plane, const wcsim_depos* depos, void* stream,
                                  wcsim_tune_report* report);

/* Maximum events of one wcsim_batch_run call. */
#define WCSIM_MAX_BATCH 64

/* Batched simulation of independent events (the planned all-device flow of Fig. 4 applied
 * to many events at once): event e runs wcsim_run on planes[e] with depos[e] (DEVICE SoA)
 * into waves[e] (DEVICE float32 [n_wires][n_ticks] of that plane), with the fluctuation
 * seed of planes[e] plus e.  Events that share a plane object are processed together: each
 * stage is one launch over all of them, and the wire pass reads each response tile once
 * for all of them.  A plane needs batch scratch for as many events as share it; it is grown
 * on demand (allocating) or beforehand with wcsim_plane_reserve_batch, after which the call
 * allocates nothing, synchronizes nothing and can be recorded in a stream capture.
 * 0 <= n_events <= WCSIM_MAX_BATCH; all planes on one device. */
wcsim_status wcsim_batch_run(int32_t n_events, wcsim_plane* const* planes,
                             const wcsim_depos* depos, float* const* waves, void* stream);

/* Reserve batch scratch for n_events (<= WCSIM_MAX_BATCH) events on this plane. */
wcsim_status wcsim_plane_reserve_batch(wcsim_plane* plane, int32_t n_events);

/* Wait for the plane's work on `stream`, then read and clear its device flags.
 * *flags (may be NULL) receives the bit set (bit 0: invalid depo values seen; bit 1: a
 * kernel's bounded wait for an asynchronous copy gave up, so its output is incomplete).
 * Returns WCSIM_ETIMEOUT if bit 1 is set, else WCSIM_EDEVICE_CHECK if bit 0 is set, else
 * WCSIM_OK. */
wcsim_status wcsim_plane_check(wcsim_plane* plane, void* stream, int32_t* flags);

/* Electronics noise N(t, x), the additive term of Eq. 1, for the waveforms of wcsim_run and
 * wcsim_batch_run (wcsim_convolve stays Eq. 2 alone).  The paper gives no noise model; this
 * is spectral noise per wire: the normalised inverse DFT over n_ft points of A(k) xi_w(k),
 * cropped to the frame, where amp (HOST, n_amp = n_ft / 2 + 1 values >= 0, extended as
 * A(n_ft - k) = A(k)) is the amplitude spectrum and xi_w(k) = (z_re + i z_im) / sqrt 2 are
 * complex Gaussians of unit mean square (z_re alone at k = 0 and, for even n_ft, at
 * n_ft / 2), z from Philox4x32-10 (counter = (k / 2, wire, 0x4E4F4953, plane id), key =
 * seed, plus the event index in a batch) and Box-Muller.  The noise is added to the wire
 * spectra as the inverse time FFT reads them (no extra memory pass).  amp == NULL or
 * n_amp == 0 turns it off.  Copies the spectrum once on `stream` and waits for the copy;
 * WCSIM_ESHAPE if n_amp is not n_ft / 2 + 1, WCSIM_EINVAL for a negative or non-finite
 * amplitude (the previous setting is kept).  No counterpart in the paper beyond Eq. 1's
 * term. */
wcsim_status wcsim_plane_set_noise(wcsim_plane* plane, const float* amp, int32_t n_amp,
                                   uint64_t seed, void* stream);

/* Limit, in ns of the device's global timer, of each device-side wait of this plane's
 * kernels for a bulk asynchronous copy (default 2e9: far above any legitimate wait).  A wait
 * that runs out sets flag bit 1 (reported by wcsim_plane_check as WCSIM_ETIMEOUT), lets the
 * copy it was waiting for land (bounded by the default limit) and ends its CTA, leaving that
 * CTA's output incomplete; the context stays usable.  0 makes every wait that is not
 * satisfied at once run out, which exercises that path (a diagnostic; no counterpart in the
 * paper).  Applies to the calls issued after it. */
wcsim_status wcsim_plane_set_wait_limit(wcsim_plane* plane, uint64_t ns);

/* Per-stage device time of the last compute calls on this plane (CUDA events), when
 * enabled with wcsim_plane_set_timing(plane, 1).  ms[0..n) receives, in order, the forward
 * stages of the last wcsim_run / rasterize / convolve: zero grid, rasterize+scatter,
 * time-axis forward FFT, wire-axis FFT x response x sum x inverse, time-axis inverse FFT;
 * then (n up to 12) the stages of the last wcsim_run_backward: zero grid, mean-path
 * rasterize, time-axis FFT of S, time-axis FFT of G, wire-axis adjoint, inverse time FFT of
 * dL/dS, per-depo adjoint (zeros if none was recorded).  Synchronizes on the events. */
wcsim_status wcsim_plane_set_timing(wcsim_plane* plane, int32_t enable);
wcsim_status wcsim_plane_stage_times(wcsim_plane* plane, float* ms, int32_t n);

/* Bytes of the static device scratch used by wcsim_convolve_noalloc (16 MiB). */
#define WCSIM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* The convolution of wcsim_convolve without any device allocation, for callers that may
 * not allocate: code running under an allocator it does not own (a framework's caching
 * allocator, a pool with a fixed budget) or a process that forbids allocation after
 * start-up.  The paper has no counterpart; it is a deployment variant of wcsim_convolve.
 * Inputs as in wcsim_plane_create + wcsim_convolve: geometry, DEVICE response complex64
 * [n_imp][n_fw][n_ft] (n_fw, n_ft = 0: the frame size), DEVICE grid float32
 * [n_wires * n_imp][n_ticks]; output DEVICE wave float32 [n_wires][n_ticks].  All
 * intermediate arrays (Hermitian response, spectra, twiddle tables) live in one static
 * device array of WCSIM_NOALLOC_SCRATCH_BYTES per device; frames whose scratch does not fit
 * (e.g. 128 wires x 10 impacts x 1024 ticks needs about 11 MiB) are rejected with
 * WCSIM_ESHAPE.  No cudaMalloc, cudaFree or allocating library call is made.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call shares the array and
 * overwrites what the previous call left: calls whose GPU work overlaps race on it, so the
 * caller must serialise them.  Stream-ordered; returns before the work is done. */
wcsim_status wcsim_convolve_noalloc(const wcsim_geometry* geom, const void* resp_c64,
                                    int32_t n_fw, int32_t n_ft, const float* grid, float* wave,
                                    void* stream);

/* Status of the last wcsim_convolve_noalloc call on the current device, without allocating:
 * waits for `stream` (the stream of that call), then copies the call's device flag word from
 * the static scratch to the host.  *flags (may be NULL) receives the bits (bit 1: a bounded
 * device-side wait for an asynchronous copy gave up, so part of that call's output was never
 * written).  Returns WCSIM_ETIMEOUT if bit 1 is set, else WCSIM_OK.  Like the entry point it
 * checks, it has no counterpart in the paper.  The next wcsim_convolve_noalloc call on the
 * device clears the word. */
wcsim_status wcsim_convolve_noalloc_check(void* stream, int32_t* flags);

/* Release the plane and everything it owns.  NULL is accepted. */
wcsim_status wcsim_plane_destroy(wcsim_plane* plane);

/* Message for the last failing call on this thread ("" if none). */
const char* wcsim_last_error(void);

/* Library version string. */
const char* wcsim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WCSIM_H */
