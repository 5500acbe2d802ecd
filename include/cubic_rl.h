/*
 * cubic_rl.h -- C ABI of the GB300 (sm_103a) 3D Richardson-Lucy deconvolution library.
 *
 * The operation is the Richardson-Lucy iteration of arXiv 2510.14143, Section 4
 * ("Richardson-Lucy deconvolution"): each iteration convolves the estimate with the
 * PSF, divides the observed image by that blurred estimate, correlates the ratio with
 * the PSF (convolution with the flipped PSF) and multiplies the estimate by the result.
 * The same section fixes the PSF to the image's ZYX size and does the convolutions with
 * FFTs.  Readings taken where the paper is silent:
 *   - boundaries are circular (same-size FFT convolution, no padding), except for plans
 *     made by cubic_rl_plan_linear (zero-padded "same"-mode convolution);
 *   - the PSF peak sits at index floor(n/2) on every axis;
 *   - the initial estimate is the constant max(mean(image), eps);
 *   - the ratio's denominator is clamped: image / max(blurred, eps).
 *
 * Conventions shared by every call:
 *   - Volumes are float32, C-order [nz][ny][nx] (x fastest), dense, in device memory,
 *     16-byte aligned.  dims[] is always {nz, ny, nx}.
 *   - Every axis length must be one the library has kernels for: the 5-smooth
 *     lengths (2^a 3^b 5^c) listed by cubic_rl_supported_length(); others give
 *     CUBIC_ERR_UNSUPPORTED_SIZE.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     validate their arguments on the host, then enqueue work on `stream` and return
 *     without synchronising; results are ready when the stream reaches that point.
 *   - On any error nothing is enqueued, the status is returned and a thread-local
 *     message is available from cubic_last_error().  Nothing aborts or prints.
 *   - A plan is used by one stream at a time (its scratch is shared by its calls).
 */
#ifndef CUBIC_RL_H
#define CUBIC_RL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CUBIC_API __attribute__((visibility("default")))
#else
#define CUBIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUBIC_OK = 0,
    CUBIC_ERR_INVALID_ARG = 1,
    CUBIC_ERR_UNSUPPORTED_SIZE = 2,
    CUBIC_ERR_ALIGNMENT = 3,
    CUBIC_ERR_OUT_OF_MEMORY = 4,
    CUBIC_ERR_CUDA = 5,
    CUBIC_ERR_TIMEOUT = 6,
    CUBIC_ERR_NOT_READY = 7
} cubic_status_t;

typedef struct cubic_rl_plan_s *cubic_rl_plan_t;

/* Human-readable name of a status code (static string). */
CUBIC_API const char *cubic_status_string(cubic_status_t s);

/* Detail of the last error raised on the calling host thread (thread-local, static
 * storage; valid until the next failing call on this thread). */
CUBIC_API const char *cubic_last_error(void);

/* 1 if an axis of length n is supported, else 0. */
CUBIC_API int cubic_rl_supported_length(int64_t n);

/* Create a plan for volumes of size dims = {nz, ny, nx} and PSF `psf` (device float32
 * [nz][ny][nx], peak at (nz/2, ny/2, nx/2), floor division).  In Section 4 of the paper
 * the PSF volume is as large as the image volume.  The plan moves the PSF peak to
 * the origin and keeps H = DFT3(psf shifted) / V (complex64, [nz][ny][nx/2+1] padded),
 * plus twiddle tables; the caller keeps owning `psf` and may free it once the stream
 * has passed this call.  flags: reserved, pass 0.
 * Errors: INVALID_ARG (null pointers, flags), UNSUPPORTED_SIZE, ALIGNMENT,
 * OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_plan(cubic_rl_plan_t *plan, const int64_t dims[3], const float *psf,
                             unsigned flags, void *stream);

/* Replace the PSF of an existing plan -- e.g. after a PSF-parameter step.  psf: device
 * float32 of the plan's PSF dims (the image dims, or psf_dims for a cubic_rl_plan_linear
 * plan), peak at floor(n/2), 16-byte aligned; the caller keeps owning it.  H is rebuilt on
 * `stream` and the point-symmetry check that selects the real-spectrum Z pass is redone
 * (one stream synchronisation).  Errors: INVALID_ARG (null pointers), ALIGNMENT,
 * OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_plan_update_psf(cubic_rl_plan_t plan, const float *psf, void *stream);

/* Release a plan and everything it allocated (synchronises the device first; a workspace
 * given by cubic_rl_set_workspace stays the caller's).  NULL is accepted and ignored. */
CUBIC_API cubic_status_t cubic_rl_plan_destroy(cubic_rl_plan_t plan);

/* Bytes of device scratch one deconvolution call of this plan needs (the complex
 * half-spectrum work array).  Errors: INVALID_ARG (null pointers). */
CUBIC_API cubic_status_t cubic_rl_workspace_bytes(cubic_rl_plan_t plan, size_t *bytes);

/* Give the plan caller-owned device scratch of at least cubic_rl_workspace_bytes()
 * bytes (256-byte aligned).  Without it the plan allocates its own on first use; a
 * workspace the plan allocated before is freed (after a device synchronisation).
 * The caller must keep the memory alive while the plan uses it.  Errors: INVALID_ARG
 * (null pointers, too small), ALIGNMENT. */
CUBIC_API cubic_status_t cubic_rl_set_workspace(cubic_rl_plan_t plan, void *dev_ptr, size_t bytes);

/* Richardson-Lucy deconvolution, Section 4 of the paper: n_iter iterations of
 *   b = psf (*) u;  r = image / max(b, eps);  q = psf (*)^T r;  u = u * q
 * from u0 = max(mean(image), eps), (*) circular convolution, (*)^T its adjoint
 * (correlation, i.e. convolution with the flipped PSF).
 * image: device float32 [nz][ny][nx] (read only).  out: device float32 [nz][ny][nx],
 * receives u_{n_iter}; must not overlap image.  n_iter >= 0 (0 gives u0).  eps > 0,
 * finite.  Errors: INVALID_ARG, ALIGNMENT, OUT_OF_MEMORY (workspace), CUDA. */
CUBIC_API cubic_status_t cubic_rl_deconvolve(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                   float *out, void *stream);

/* Batched Richardson-Lucy: the same deconvolution as cubic_rl_deconvolve for n volumes of
 * possibly different sizes, each with its own plan (plans must be distinct: a plan's scratch
 * serves one volume).  images[v], outs[v]: device float32 volumes of plans[v]'s dims.  For
 * each pass, the volumes whose length along that pass is one of the 5-smooth lengths 48 to
 * 160 share one kernel launch per length class (three classes by elements per thread, with
 * launch shapes fixed per length); the volumes of any other length share one launch per
 * length, whose launch shape (threads per line, lines or columns per CTA) is tuned the first
 * time the length appears: every candidate is timed on the call's own buffers and the
 * fastest is kept for the process.  A launch's blocks span every member volume.  The whole
 * n_iter sequence is captured once into a CUDA graph (first call with a given argument
 * set: tuning of new lengths, capture and instantiation, synchronous) and replayed on
 * `stream` by later calls with identical arguments (a few argument sets are cached).
 * 1 <= n <= 256.  Errors: INVALID_ARG, ALIGNMENT, OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_deconvolve_batched(const cubic_rl_plan_t *plans, int n,
                                                     const float *const *images, int n_iter, float eps,
                                                     float *const *outs, void *stream);

/* Kernel nodes in the graph the last cubic_rl_deconvolve_batched call replayed. */
CUBIC_API int64_t cubic_rl_batched_graph_nodes(void);

/* cubic_rl_deconvolve on host buffers: copies `image` (host, V floats; pinned memory makes
 * the copies asynchronous) to device memory owned by the plan, deconvolves there, and
 * copies the estimate back into `out` (host, V floats).  All three steps are enqueued on
 * `stream`; `out` is valid once the stream has passed this call.  The first call
 * allocates the two device staging volumes (released with the plan). */
CUBIC_API cubic_status_t cubic_rl_deconvolve_host(cubic_rl_plan_t plan, const float *image, int n_iter,
                                                  float eps, float *out, void *stream);

/* Create a plan with linear ("same"-mode, zero-padded) boundaries for images of size
 * dims = {nz, ny, nx} and a PSF box psf_dims = {kz, ky, kx} (device float32, peak at
 * floor(k/2) per axis), which may be smaller than the image.  The paper convolves
 * same-size arrays circularly; here the estimate and the image stay on their own box, the
 * blur sees zeros outside it, b(x) = sum_t p(t + c) u(x - t) with c = floor(k/2), and the
 * back-projection is its adjoint.  The transforms run on the smallest supported lengths
 * m >= max(n + floor(k/2), k) per axis, which is exact for this output.  The plan owns two
 * zero-padded copies of the image box (image and estimate).  Supported on such a plan:
 * cubic_rl_deconvolve, cubic_rl_deconvolve_host, cubic_rl_deconvolve_accel,
 * cubic_rl_deconvolve_auto, cubic_rl_deconvolve_monitor (the likelihood summed over the
 * image's voxels), cubic_rl_convolve, cubic_rl_plan_update_psf (psf of psf_dims),
 * cubic_rl_autotune and the plan queries.  Every other entry point returns INVALID_ARG
 * for it.  Errors: INVALID_ARG, UNSUPPORTED_SIZE (no supported length, or padded nz or
 * ny above 65535), ALIGNMENT, OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_plan_linear(cubic_rl_plan_t *plan, const int64_t dims[3],
                                              const int64_t psf_dims[3], const float *psf, unsigned flags,
                                              void *stream);

/* The image dims and the transform dims of a plan (equal unless it has linear
 * boundaries); either pointer may be NULL. */
CUBIC_API cubic_status_t cubic_rl_plan_dims(cubic_rl_plan_t plan, int64_t image[3], int64_t transform[3]);

/* Normalised anisotropic Gaussian PSF, psf = amp * g / sum(g) with
 * g = exp(-(dx^2 + dy^2) / (2 sigma_xy^2) - dz^2 / (2 sigma_z^2)), (dx, dy, dz) = index -
 * floor(n/2) per axis.  The paper models its PSF with a theoretical (Richards-Wolf)
 * model of the same ZYX size as the image (Section 4, "Dataset description"); this
 * parametric stand-in is the one whose parameters the differentiable path fits.
 * psf: device float32 [nz][ny][nx].  g in float32, sum(g) in double.  Uses a small
 * stream-ordered scratch allocation.  Errors: INVALID_ARG, ALIGNMENT, CUDA. */
CUBIC_API cubic_status_t cubic_psf_gaussian(const int64_t dims[3], float sigma_xy, float sigma_z, float amp,
                                            float *psf, void *stream);

/* Device-side status of the plan's kernels: synchronises `stream`, then returns
 * CUBIC_ERR_TIMEOUT (and clears the flag) if any kernel's bounded wait on an asynchronous
 * copy gave up since the last check, else CUBIC_OK.  Kernels that give up skip their
 * stores, so their outputs are then undefined. */
CUBIC_API cubic_status_t cubic_rl_stream_status(cubic_rl_plan_t plan, void *stream);

/* Limit, in nanoseconds of the GPU's global timer, of every bounded device wait made by
 * the plan's kernels (the waits on the asynchronous tile copies).  0 restores the default
 * of 2 s.  A wait that reaches the limit gives up as described for cubic_rl_stream_status.
 * Errors: INVALID_ARG for a null plan. */
CUBIC_API cubic_status_t cubic_rl_plan_set_wait_limit(cubic_rl_plan_t plan, uint64_t limit_ns);

/* Test support for the failure path of the bounded waits (no counterpart in the paper).
 * Arms a one-shot setting for the whole process: the next Y-pass launch that uses a
 * TMA-pipelined launch shape -- on any plan, or inside cubic_rl_deconvolve_noalloc -- waits
 * at most wait_ns per tile, and its first CTA does not issue the copy of its first tile.
 * That CTA's wait then runs out: it sets the device error word, waits for the copies it
 * did issue and returns, so no copy is left in flight and the context stays usable.  The
 * call that made the launch reports CUBIC_ERR_TIMEOUT through cubic_rl_stream_status (or
 * cubic_rl_noalloc_status) and its result is wrong by design.  wait_ns == 0 disarms a
 * setting that no launch has taken yet.  Always CUBIC_OK. */
CUBIC_API cubic_status_t cubic_test_skip_next_tile_copy(uint64_t wait_ns);

/* ---- launch shapes and autotuning ---- */

/* counts[3] = number of compiled launch-shape variants of the X, Y and Z passes for this
 * plan's lengths; chosen[3] = the variants in use.  Either pointer may be NULL. */
CUBIC_API cubic_status_t cubic_rl_plan_variants(cubic_rl_plan_t plan, int counts[3], int chosen[3]);

/* Select launch-shape variants explicitly (INVALID_ARG if out of range).  Every variant
 * computes the same transform; they differ in threads per line and lines per CTA. */
CUBIC_API cubic_status_t cubic_rl_plan_set_variants(cubic_rl_plan_t plan, int vx, int vy, int vz);

/* Process the Y-forward / Z / Y-inverse passes of each convolution in chunks of `columns`
 * spectrum columns (a multiple of 16; 0 = all columns in one launch per pass), so that a
 * chunk stays in L2 between the three passes.  Results do not depend on it. */
CUBIC_API cubic_status_t cubic_rl_plan_set_chunk(cubic_rl_plan_t plan, int64_t columns);

/* Current chunk setting (-1 for a NULL plan). */
CUBIC_API int64_t cubic_rl_plan_chunk(cubic_rl_plan_t plan);

/* Time every variant of each pass on this plan's own buffers (image read, `out` and the
 * workspace overwritten) and keep the fastest.  Synchronises the stream several times, so
 * do not call it while capturing a graph.  The choice is remembered for later plans of
 * the same dims in this process and, if the environment variable CUBIC_TUNE_CACHE names a
 * file, appended there and read back by later processes. */
CUBIC_API cubic_status_t cubic_rl_autotune(cubic_rl_plan_t plan, const float *image, float *out,
                                           void *stream);

/* Allocation-free deconvolution.  The paper has no counterpart: this is a service for
 * callers that cannot call cudaMalloc -- a framework whose device memory is fully
 * reserved by its own pool allocator, plug-in code whose host application does not let it
 * allocate, and latency-critical loops that cannot take cudaMalloc's implicit device-wide
 * synchronisation.  It computes what cubic_rl_plan + cubic_rl_deconvolve compute on
 * (psf, image), equal to float32 rounding: it always multiplies by the complex PSF
 * spectrum, because finding that a PSF is point-symmetric (which lets a plan use the
 * cheaper real spectrum) takes a host synchronisation.  Every internal buffer lives in one
 * fixed 8 MiB device array that each GPU loading this library holds until the process
 * exits; nothing is allocated or freed.
 * Limit: nz * ny * xp <= about 2^19 complex elements, xp = nx/2+1 rounded up to 16 (e.g.
 * 64x64x64 or 80x80x128); larger volumes get CUBIC_ERR_UNSUPPORTED_SIZE with the byte
 * counts.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make that first
 * call before any stream capture; the kept address does not survive a cudaDeviceReset.
 * All calls share the array, which keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and give wrong results;
 * serialise them.  A bounded device wait that runs out sets an error word in the array
 * that stays set until cubic_rl_noalloc_status reads it.  psf, image, out: device float32
 * [nz][ny][nx], 16-byte aligned; out must not overlap image.  Errors: INVALID_ARG,
 * UNSUPPORTED_SIZE, ALIGNMENT, CUDA. */
CUBIC_API cubic_status_t cubic_rl_deconvolve_noalloc(const int64_t dims[3], const float *psf,
                                                     const float *image, int n_iter, float eps,
                                                     float *out, void *stream);

/* Device-side status of the allocation-free calls on the current device: synchronises
 * `stream`, then returns CUBIC_ERR_TIMEOUT (and clears the word) if a bounded device wait
 * of any allocation-free call gave up since the last check, else CUBIC_OK.  Allocates
 * nothing.  The paper has no counterpart. */
CUBIC_API cubic_status_t cubic_rl_noalloc_status(void *stream);

/* Richardson-Lucy with metric-guided stopping.  The paper (Section 4) selects the
 * iteration count by monitoring an image-quality measure between consecutive iterations
 * against a threshold; Section 3 lists scale-invariant PSNR among its metrics.  Every
 * iteration k (the one that makes u_{k+1}) records three measures:
 *   delta_k   = ||u_{k+1} - u_k|| / ||u_k||;
 *   NLL(u_k)  = sum (c - d ln c), c = max(h * u_k, eps): the Poisson negative
 *               log-likelihood up to a constant, from iteration k's forward convolution;
 *   PSNR_k    = scale-invariant PSNR of u_{k+1} against reference: 20 log10(range / rmse)
 *               after the least-squares affine fit a u + b of the estimate to the reference,
 *               range = max - min of the reference (NaN without a reference).
 * The sums are compensated float32 on the GPU; the fit and the logarithms are finished on
 * the host in double precision.  At every check (k + 1 a multiple of check_every, or the
 * last iteration) the run stops when the chosen measure's improvement is under tol:
 *   CUBIC_METRIC_REL_CHANGE: delta_k < tol;
 *   CUBIC_METRIC_NLL:        k >= 1 and (NLL(u_{k-1}) - NLL(u_k)) / |NLL(u_k)| < tol;
 *   CUBIC_METRIC_PSNR:       k >= 1 and PSNR_k - PSNR_{k-1} < tol (decibels).
 * out receives the last estimate, *n_done the iterations done, history (host, may be NULL)
 * 3 * max_iter doubles: (delta, NLL, PSNR) per iteration done.  reference: device float32
 * [nz][ny][nx] or NULL (required for CUBIC_METRIC_PSNR).  Synchronous: it returns after the
 * last check.  Errors: INVALID_ARG, ALIGNMENT, OUT_OF_MEMORY, CUDA. */
enum { CUBIC_METRIC_REL_CHANGE = 0, CUBIC_METRIC_NLL = 1, CUBIC_METRIC_PSNR = 2 };
CUBIC_API cubic_status_t cubic_rl_deconvolve_monitor(cubic_rl_plan_t plan, const float *image,
                                                     const float *reference, int max_iter, float eps,
                                                     int metric, double tol, int check_every, float *out,
                                                     int *n_done, double *history, void *stream);

/* Accelerated Richardson-Lucy.  The paper (Section 2) cites the acceleration of Biggs and
 * Andrews (Applied Optics 36(8), 1997) for RL; this is their first-order vector
 * extrapolation.  Each RL step starts from a prediction along the last move:
 *   y_k = max(x_k + alpha_k (x_k - x_{k-1}), 0),  x_{k+1} = one RL iteration from y_k,
 *   g_k = x_{k+1} - y_k,  alpha_{k+1} = <g_k, g_{k-1}> / <g_{k-1}, g_{k-1}> clamped to [0, 1],
 * with x_0 = max(mean(image), eps), alpha_0 = alpha_1 = 0 and alpha = 0 for a zero
 * denominator.  The dot products are compensated float32 sums.  out receives x_{n_iter}.
 * alpha (device float[n_iter], may be NULL) receives alpha_0 .. alpha_{n_iter-1}.
 * image, out: device float32 [nz][ny][nx], 16-byte aligned, not overlapping.  The first
 * call allocates five volumes of plan-owned buffers.  Asynchronous on stream (alpha stays
 * on the device).  Errors: INVALID_ARG (null pointers, n_iter < 0, eps <= 0 or not finite,
 * overlap), ALIGNMENT, OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_deconvolve_accel(cubic_rl_plan_t plan, const float *image, int n_iter,
                                                   float eps, float *out, float *alpha, void *stream);

/* Richardson-Lucy with automatic stopping.  The paper (Section 4) stops the iteration when
 * the improvement between consecutive iterations falls under a threshold; it names neither
 * the measure nor the threshold.  Reading taken here: the improvement of iteration k is the
 * relative change of the estimate, delta_k = ||u_{k+1} - u_k||_2 / ||u_k||_2, accumulated
 * inside the update pass.  After every check_every-th iteration (and after max_iter) the
 * host reads delta_{k} (a stream synchronisation) and stops when delta_k < tol.
 * out receives the last estimate, *n_done the number of iterations done, history (host,
 * max_iter doubles, may be NULL) delta_0 .. delta_{n_done-1}.  Synchronous (returns after
 * the last check).  Errors: INVALID_ARG, ALIGNMENT, OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_rl_deconvolve_auto(cubic_rl_plan_t plan, const float *image, int max_iter,
                                                  float eps, float tol, int check_every, float *out,
                                                  int *n_done, double *history, void *stream);

/* Fourier Shell Correlation of two volumes of the plan's dims, the resolution metric the
 * paper evaluates deconvolution with (FRC/FSC, Sections 3 and 4):
 *   fsc[s] = Re sum_{k in s} A(k) conj B(k) / sqrt(sum |A|^2 sum |B|^2),
 * A, B the 3D DFTs of a and b (device float32 volumes).  Shell s = floor(2 n_shells rho)
 * for the normalised frequency radius rho = |(kz/nz, ky/ny, kx/nx)| (cycles per voxel,
 * decided exactly in integer arithmetic); frequencies beyond Nyquist (rho >= 1/2) are left
 * out; an empty shell gives 0.  fsc: device float32[n_shells].  1 <= n_shells <= 1024.
 * Uses the plan's workspace and a second spectrum it allocates on first use. */
CUBIC_API cubic_status_t cubic_fsc(cubic_rl_plan_t plan, const float *a, const float *b, int n_shells,
                                   float *fsc, void *stream);

/* Single-image FSC (the resolution measure of the paper's Section 4 "Evaluation metrics",
 * computed from one image after Koho et al. 2019).  image: device float32 of dims 2h =
 * {2 hz, 2 hy, 2 hx}; half_plan: a plan (circular) of dims h, whose PSF is not used.  The
 * image splits into its eight parity sub-volumes d(2z + a, 2y + b, 2x + c); the FSC of each
 * of the four pairs of opposite parity is taken on the half grid (shells of the half grid)
 * and fsc (device float[n_shells]) receives their mean.  No correction is made for the
 * half-voxel diagonal shift within a pair.  Uses a small stream-ordered scratch allocation.
 * Errors: INVALID_ARG, ALIGNMENT, OUT_OF_MEMORY, CUDA. */
CUBIC_API cubic_status_t cubic_fsc_split(cubic_rl_plan_t half_plan, const float *image, int n_shells, float *fsc,
                                         void *stream);

/* ---- differentiation (reverse mode through the iterations) ---- */

/* cubic_rl_deconvolve that also stores the estimate u_k at every k = 0, ckpt_every,
 * 2*ckpt_every, ... < n_iter into ckpts (device float32, ceil(n_iter/ckpt_every) volumes,
 * back to back) for cubic_rl_backward.  n_iter >= 1, ckpt_every >= 1; image, out and
 * ckpts must not overlap. */
CUBIC_API cubic_status_t cubic_rl_deconvolve_ckpt(cubic_rl_plan_t plan, const float *image, int n_iter,
                                                  float eps, int ckpt_every, float *ckpts, float *out,
                                                  void *stream);

/* Device scratch the backward keeps in the plan for this checkpoint spacing:
 * (4*ckpt_every + 4) volumes of floats, (2*ckpt_every + 1) half spectra and a small
 * reduction buffer. */
CUBIC_API cubic_status_t cubic_rl_backward_workspace_bytes(cubic_rl_plan_t plan, int ckpt_every,
                                                           size_t *bytes);

/* Gradient of a loss L(u_{n_iter}) through the n_iter iterations of the paper's RL step
 * (Section 4: forward convolution, ratio, flipped-PSF convolution, multiplicative
 * update), given grad_out = dL/du_{n_iter} (device float32 volume) and the checkpoints
 * of cubic_rl_deconvolve_ckpt for the same (plan, image, n_iter, eps, ckpt_every).
 * Writes grad_image = dL/dimage (through every ratio and through u0 = max(mean, eps));
 * grad_psf = dL/dpsf for the centred PSF (added to grad_psf when accumulate_psf != 0).
 * Either output may be NULL.  The derivative of max(b, eps) is taken as 1 where
 * b > eps, else 0.  Segments between checkpoints are recomputed; their iterates live in
 * plan-owned scratch (allocated on first use; cubic_rl_backward_workspace_bytes). */
CUBIC_API cubic_status_t cubic_rl_backward(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                           int ckpt_every, const float *ckpts, const float *grad_out,
                                           float *grad_image, float *grad_psf, int accumulate_psf,
                                           void *stream);

/* dL/d(sigma_xy, sigma_z, amp) of the Gaussian PSF of cubic_psf_gaussian given
 * grad_psf = dL/dpsf: writes three floats to grad_params (device memory).  The PSF's flux
 * sum is in double, the other five reductions in compensated float32. */
CUBIC_API cubic_status_t cubic_psf_gaussian_backward(const int64_t dims[3], float sigma_xy, float sigma_z,
                                                     float amp, const float *grad_psf, float *grad_params,
                                                     void *stream);

/* ---- launch accounting and per-kernel timing ---- */

/* Number of kernel kinds and the name of each (static strings). */
CUBIC_API int cubic_rl_kernel_kinds(void);
CUBIC_API const char *cubic_rl_kernel_name(int kind);

/* Reset the plan's launch counters; with enable != 0 also bracket every later launch by a
 * pair of CUDA events on its stream (up to max_events events, taken from a pool the plan
 * keeps), so that per-kernel device time can be read back.  Timing adds two event records
 * per launch to the stream. */
CUBIC_API cubic_status_t cubic_rl_profile(cubic_rl_plan_t plan, int enable, int max_events);

/* Per kernel kind (arrays of n_kinds entries, any may be NULL): summed event-timed device
 * time in ms and the number of timed launches (synchronises on the last recorded event),
 * the number of launches enqueued since cubic_rl_profile() and their algorithmic HBM bytes
 * (each array the kernel must read or write, counted once). */
CUBIC_API cubic_status_t cubic_rl_profile_read(cubic_rl_plan_t plan, int n_kinds, double *total_ms,
                                               int64_t *timed_launches, int64_t *launches, double *bytes);

/* ---- building blocks (the same kernels, exposed for the forward model and for tests) ---- */

/* Convolution with the plan's PSF (the blur step of Section 4 of the paper):
 * out = psf (*) in, circular, or zero-padded "same"-mode for a cubic_rl_plan_linear plan.
 * flipped != 0 gives the correlation with the PSF (a convolution with the mirrored PSF,
 * the step that carries the ratio back), the adjoint of the former.  in, out: device
 * float32 [nz][ny][nx] of the image dims; they may alias.  Uses the plan workspace. */
CUBIC_API cubic_status_t cubic_rl_convolve(cubic_rl_plan_t plan, const float *in, int flipped, float *out,
                                 void *stream);

/* Layout of the plan's half spectra: xh = nx/2+1 valid columns, row pitch xp >= xh
 * (complex64 elements); a spectrum is complex64 [nz][ny][xp]. */
CUBIC_API cubic_status_t cubic_rl_spectrum_layout(cubic_rl_plan_t plan, int64_t *xh, int64_t *xp);

/* Unnormalised forward 3D DFT, X[k] = sum_n x[n] exp(-2 pi i k.n / N), of a real volume
 * (device float32 [nz][ny][nx]) into a half spectrum (device complex64 [nz][ny][xp],
 * columns >= xh untouched).  `in` must not overlap `spec`. */
CUBIC_API cubic_status_t cubic_rl_fft3_forward(cubic_rl_plan_t plan, const float *in, void *spec, void *stream);

/* Inverse 3D DFT with the 1/V factor of a half spectrum back to a real volume.  The
 * imaginary parts of the self-conjugate x-bins (kx = 0 and kx = nx/2) are ignored, as in
 * any complex-to-real transform.  `spec` is overwritten (used as scratch). */
CUBIC_API cubic_status_t cubic_rl_fft3_inverse(cubic_rl_plan_t plan, void *spec, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CUBIC_RL_H */
