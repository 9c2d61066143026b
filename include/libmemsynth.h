/*
 * libmemsynth — non-gridding maximum-entropy image synthesis on one GB300.
 *
 * C ABI of the hot path of Carcamo et al., "Multi-GPU maximum entropy image
 * synthesis for radio astronomy" (arXiv:1703.02920): the measurement operator
 * of Eq. (1) evaluated as a direct (non-gridded) sum at every (u,v) sample,
 * its adjoint (the chi^2 gradient, Eq. chi2gradient / Appendix C), the entropy
 * term and its gradient (Eq. logentropy, Eq. Sgradient), the positivity bound
 * I >= G (Eq. minproblem) and the projected conjugate-gradient solve.
 *
 * Notation.  N = image side, pixels row-major [y][x] (index n*N + m) with
 * pixel coordinates x_m = (m - N/2) dx, y_n = (n - N/2) dy (radians; the pixel
 * origin of the gradient kernel in Section 2.5).  u, v in wavelengths.
 * Visibilities are interleaved (re, im).  A is the primary beam (Section 2.4,
 * step 1), B = A * I the attenuated image, w_k = 1 / sigma_k^2.
 *
 *   forward   V_k   = sum_{n,m} B[n][m] exp(-2 pi i (u_k x_m + v_k y_n))
 *   adjoint   G[n][m] = A[n][m] * sum_k Re( y_k exp(+2 pi i (u_k x_m + v_k y_n)) )
 *   chi^2     = 1/2 sum_k w_k |V_k - V^o_k|^2                      (Eq. phi2)
 *   entropy   S = - sum_i I_i log(I_i / G)                          (Eq. logentropy;
 *               the paper's (I/G) log(I/G) scale is folded into lambda)
 *   objective Phi = chi^2 - lambda S                                (Eq. phi3)
 *   gradient  grad Phi = A * Re(F^H (w r)) + lambda (1 + log(I/G)),  r = V - V^o
 *
 * Multi-channel data (Section 2.1, Eq. chi2-multi): visibilities of channel c
 * are the index range [vis_offsets[c], vis_offsets[c+1]); channel c has its
 * own primary beam A_c (C*N*N floats).  MEM_IMAGES_PER_CHANNEL treats each
 * channel as an independent image (a line cube, C*N*N floats per image
 * argument); MEM_IMAGE_SHARED fits one N*N image to all channels, chi^2
 * summed over channels as in Eq. chi2-multi.
 *
 * Ownership and threading.  The caller owns every pointer it passes.
 * mem_create copies the data into device memory owned by the context (the
 * data stays resident, Section 2.5 "keep most of the data in global memory").
 * Arguments named *_dev are device pointers the caller allocated (e.g. torch
 * tensors); work is enqueued on the stream given to mem_create and calls
 * returning scalars to the host synchronise that stream.  A context is used
 * from one host thread at a time and is not re-entrant.
 *
 * Errors.  Every call returns a mem_status; nothing is thrown across the ABI.
 * mem_last_error() gives a message for the last failing call of a context.
 * Device-side waits are bounded (mem_config.spin_limit); a wait that runs out
 * makes the call return MEM_ETIMEOUT without faulting the GPU.  The last wait
 * of a tensor-core kernel, for its own operations and copies already in
 * flight (they must finish before their memory is released), is bounded by
 * max(spin_limit, 2^24) polls.  A non-finite
 * objective returns MEM_ENUMERIC.  There is no CPU fallback: without a usable
 * sm_103a GPU, mem_create returns MEM_ECUDA.
 */
#ifndef LIBMEMSYNTH_H
#define LIBMEMSYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mem_ctx mem_ctx;

typedef enum {
    MEM_OK = 0,
    MEM_EINVAL = 1,    /* bad argument (null pointer, size, unsupported combination) */
    MEM_ENOMEM = 2,    /* device allocation failed or exceeded MEMSYNTH_MAX_BYTES */
    MEM_ECUDA = 3,     /* CUDA runtime error, or no sm_103a device */
    MEM_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    MEM_ENUMERIC = 5,  /* objective not finite */
    MEM_ENOTSUP = 6    /* form not available */
} mem_status;

/* Number format of the operator pair.  Every form computes the same sums
 * (Eq. 1 and Eq. chi2gradient); they differ in arithmetic.  Phase arguments
 * u x + v y are always reduced exactly (64-bit fixed-point turns obtained
 * from an FP64 reduction of u dx and v dy). */
typedef enum {
    MEM_PREC_FP64_DIRECT = 0,  /* one FP64 exponential per (visibility, pixel) pair */
    MEM_PREC_FP32_DIRECT = 1,  /* one FP32 (SFU) exponential per pair, FP64 partial sums */
    MEM_PREC_BF16X3 = 2,       /* separable phase tables generated on chip, tcgen05
                                  tensor-core contractions in 3-term split BF16 with FP32
                                  accumulation, compensated cross-tile reductions */
    MEM_PREC_FP16X3 = 3        /* as BF16X3 with a 3-term split FP16 (11-bit halves) and
                                  power-of-two operand scaling: same speed, ~8x smaller
                                  representation error */
} mem_precision;

typedef enum {
    MEM_IMAGES_PER_CHANNEL = 0,
    MEM_IMAGE_SHARED = 1
} mem_image_mode;

typedef struct {
    int32_t n;                   /* image side N, 16 <= N <= 4096, multiple of 16 */
    double dx, dy;               /* pixel size in radians, > 0 */
    int32_t n_channels;          /* C >= 1 */
    const int64_t *vis_offsets;  /* host, C+1 non-decreasing entries, [0] = 0, [C] = Z total */
    double lambda;               /* entropy weight (>= 0) in Phi = chi^2 + lambda sum I log(I/G) */
    double G;                    /* lower bound and entropy reference, > 0 (Jy/pixel) */
    int32_t precision;           /* mem_precision */
    int32_t image_mode;          /* mem_image_mode */
    uint64_t spin_limit;         /* bound on device-side wait iterations; 0 = default (2^26) */
} mem_config;

/* Per-call summary of mem_solve. */
typedef struct {
    int32_t iterations;    /* CG iterations completed (per image, max over images) */
    int32_t evaluations;   /* objective evaluations (forward passes), summed over images */
    int32_t status;        /* mem_status of the solve */
    int32_t stopped_early; /* 1 if an image stopped before n_iter (no descent / no decrease) */
    double phi, chi2, entropy;  /* final values summed over images */
} mem_solve_report;

/* Create a context: validates cfg, copies u, v (Z doubles each), vis_obs (2Z
 * doubles, interleaved re/im), sigma (Z doubles, > 0) and pb (C*N*N floats)
 * to the device, prepares per-visibility phase increments (FP64 reduction of
 * u dx, v dy to 64-bit fixed-point turns) and binds the context to `stream`
 * (a cudaStream_t; NULL = legacy default stream).  All host pointers.
 * Resident device data: 84 bytes per visibility (u, v, the fixed-point
 * phases, V° in FP64 and as FP32 hi/lo pairs, 1/sigma^2 in FP64 and FP32, the
 * weighted residual) and 4 bytes per beam pixel; the first evaluation adds
 * work buffers (operand planes, split-K partials: about 40 MB at N = 256). */
mem_status mem_create(const mem_config *cfg, const double *u, const double *v,
                      const double *vis_obs, const double *sigma, const float *pb,
                      void *stream, mem_ctx **out);

/* Waits for the context's stream, then frees everything the context owns:
 * device buffers, CUDA graphs, events and its pinned host words.  The
 * caller's stream is not destroyed.  NULL is ignored. */
void mem_destroy(mem_ctx *ctx);

/* Message for the last failing call on ctx (or a global one when ctx is NULL);
 * mem_status_string: a static name for a status code. */
const char *mem_last_error(const mem_ctx *ctx);
const char *mem_status_string(mem_status s);

/* Switch the number format used by later calls (same data, no re-upload). */
mem_status mem_set_precision(mem_ctx *ctx, int32_t precision);

/* Sizes: total visibilities; images (C in cube mode, 1 in shared mode). */
int64_t mem_num_vis(const mem_ctx *ctx);
int32_t mem_num_images(const mem_ctx *ctx);

/* Forward operator, Eq. (1): vis_dev[2k], vis_dev[2k+1] = Re, Im of
 * V_k = F_c(A_c * I_c) for k in channel c.  image_dev: C*N*N floats (cube)
 * or N*N (shared).  vis_dev: 2*Z floats. */
mem_status mem_forward(mem_ctx *ctx, const float *image_dev, float *vis_dev);

/* Adjoint, Eq. (chi2gradient) with the beam factor: img_dev = A_c *
 * Re(F_c^H y_c) per channel image (cube) or summed over channels (shared).
 * y_dev: 2*Z floats (re, im).  img_dev: C*N*N or N*N floats. */
mem_status mem_adjoint(mem_ctx *ctx, const float *y_dev, float *img_dev);

/* Objective and gradient at image_dev (all pixels must be > 0): writes
 * grad_dev (same shape as the image; NULL to skip) with grad Phi, or the
 * positively projected gradient when `projected` != 0 (components with
 * I <= G and grad > 0 set to 0).  out3_host (nullable) receives Phi, chi^2, S
 * summed over images; passing it synchronises the stream.  The last values
 * also stay on the device, see mem_scalars_dev. */
mem_status mem_objective_grad(mem_ctx *ctx, const float *image_dev, float *grad_dev,
                              int32_t projected, double *out3_host);

/* Same as mem_objective_grad with host buffers: copies image_host to the
 * device and grad_host back within the call (synchronous: one stream
 * synchronisation, which also reads the scalars and the status word back).
 * Page-locked host buffers let both copies run asynchronously on the stream;
 * pageable ones work too, through the driver's staging copies. */
mem_status mem_objective_grad_host(mem_ctx *ctx, const float *image_host, float *grad_host,
                                   int32_t projected, double *out3_host);

/* Device pointer to 3 doubles (Phi, chi^2, S) of the last objective call. */
const double *mem_scalars_dev(const mem_ctx *ctx);

/* Minimise Phi over I >= G (Eq. minproblem) from image_dev_inout (clipped to
 * G first), n_iter projected Polak-Ribiere CG iterations per image (beta
 * clipped at 0, steepest-descent restart every 50 iterations or when the
 * direction is not a descent one), each with a line search on
 * phi(alpha) = Phi(max(I + alpha d, G)): first trial step from the quadratic
 * model of chi^2 along d, bracketing, Brent's method (relative tolerance 1e-3,
 * at most 20 evaluations), then one Newton step on central differences.  Each
 * probe evaluates the change of Phi from the image difference, so its
 * rounding scales with the step.  Cube mode runs one independent CG per
 * channel image, all channels batched in every launch.  hist_host (nullable,
 * host) receives per image and iteration 0..n_iter the 6 doubles (Phi, chi^2,
 * S, alpha, beta, evaluations), laid out [image][iteration][6]; iterations
 * after an early stop repeat the last values. */
mem_status mem_solve(mem_ctx *ctx, float *image_dev_inout, int32_t n_iter,
                     mem_solve_report *rep, double *hist_host);

/* Wait for all work of ctx; returns MEM_ETIMEOUT / MEM_ECUDA if a kernel
 * reported a bounded-wait timeout or a CUDA error occurred. */
mem_status mem_sync(mem_ctx *ctx);

/* The paper's gridded approximation of Eq. (1) (Section 2.4, the steps of
 * the objective evaluation; Algorithm alg:chi2gpu): each channel's
 * attenuated image is zero-padded to M = pad * N (image centred), Fourier
 * transformed on the grid (cuFFT, real to complex, FP32), modulated so that
 * the phase centre is pixel (N/2, N/2), and the model visibility is
 * bilinearly interpolated at (u M dx, v M dy).  Not the exact operator the
 * other entry points evaluate: its error against Eq. (1) falls about as
 * 1/pad^2 (percent level at pad 2 on smooth images).  image_dev: device,
 * n_images x N x N float32; vis_dev: device, 2 * Z_total float32 (re, im);
 * pad in 1..8.  The padded images and spectra (C * M^2 * 4 bytes and about
 * twice that) stay allocated for the last pad used. */
mem_status mem_forward_gridded(mem_ctx *ctx, const float *image_dev, int32_t pad, float *vis_dev);

/* Natural-weights dirty image per channel (Appendix A, Eq. dirty, with the
 * measured visibilities in place of gridded ones) or, with psf != 0, the
 * PSF (Eq. PSF):
 *   I^D[c](X) = sum_k omega_k Re(V_k exp(+2 pi i U_k . X)),
 *   omega_k = (1/sigma_k^2) / sum over the channel's samples of 1/sigma^2,
 * with V_k = 1 for the PSF; no primary-beam factor.  Runs the context's
 * adjoint in its precision form.  out_dev: device, C x N x N float32. */
mem_status mem_dirty_image(mem_ctx *ctx, int32_t psf, float *out_dev);

/* Residual map: the natural-weights dirty image (as mem_dirty_image) of the
 * residual visibilities V°_k - V_k(I), with V(I) the forward operator (Eq. 1)
 * of the model image in the context's precision form.  After a solve it shows
 * what the model leaves unexplained.  image_dev: device, n_images x N x N
 * float32 (the image before the primary beam); out_dev: device, C x N x N
 * float32. */
mem_status mem_residual_image(mem_ctx *ctx, const float *image_dev, float *out_dev);

/* Mosaics (Section 2.4: one attenuation image per pointing, centred on its
 * field).  A pointing whose phase-tracking centre lies at (x_p, y_p)
 * (radians, relative to the image's phase centre, pixel (N/2, N/2)) measures
 * V_p = exp(+2 pi i (u x_p + v y_p)) F(A_p I).  The factor has unit modulus, so
 * its chi^2 equals that of the visibilities rotated to the image's phase
 * centre, vis *= exp(-2 pi i (u x_p + v y_p)).  This host function applies
 * that rotation in place (FP64, the phase reduced modulo one turn before the
 * sine and cosine).  With each pointing's rotated data and its beam (centred
 * on the pointing) as one channel of a MEM_IMAGE_SHARED context, the
 * context's objective, gradient and solve are the mosaic's.  u, v (n_vis,
 * wavelengths) and vis (2 * n_vis, interleaved re, im) on the host. */
mem_status mem_phase_rotate(int64_t n_vis, const double *u, const double *v, double x_p, double y_p,
                            double *vis_inout);

/* Elliptical Gaussian fitted to a PSF's main lobe (Appendix A: BMAJ, BMIN,
 * BPA).  Host function, no GPU.  The main lobe is the 4-connected region
 * around the centre pixel (n/2, n/2) where the PSF exceeds 0.35 of its value
 * there; ln(PSF / PSF0) is fitted by least squares to -(A x^2 + B x y + C y^2)
 * with x = (m - n/2) dx, y = (row - n/2) dy (radians).  out4 (host): BMAJ and
 * BMIN (FWHM, radians), BPA (degrees in (-90, 90], from the +y (row) axis
 * towards +x (column)), and the beam area in pixels, pi/(4 ln 2) BMAJ BMIN /
 * (dx dy), which converts Jy/beam to Jy/pixel.  MEM_ENUMERIC when the lobe is
 * not a peak. */
mem_status mem_beam_fit(const float *psf_host, int32_t n, double dx, double dy, double *out4);

/* Tensor-core tiling.  fwd_kernel selects the forward kernel:
 *   MEM_FWD_STREAM    the split image operand streams through shared memory
 *                     for every 64-visibility tile, in column blocks of
 *                     fwd_cols (a multiple of 32 dividing N, at most 256);
 *                     fwd_stages 3 or 4;
 *   MEM_FWD_RESIDENT  (N <= 256) each CTA keeps a 128-row slice of the split
 *                     image operand in shared memory and only the phase
 *                     tables stream; fwd_cols is N; fwd_stages 4 to 6 (as
 *                     shared memory allows).
 * adj_stages: adjoint pipeline depth, 2 or 3.  The two forward kernels round
 * differently (the resident one sums 128-row slices in FP64 and issues the
 * small correction products before the main ones); both meet the form's
 * tolerances; at a solve's final image the resident order halves the chi^2
 * error. */
typedef enum { MEM_FWD_STREAM = 0, MEM_FWD_RESIDENT = 1 } mem_fwd_kernel;

typedef struct {
    int32_t fwd_kernel;
    int32_t fwd_cols;
    int32_t fwd_stages;
    int32_t adj_stages;
} mem_tiling_t;

/* Autotune the tiling on this context's data (a no-op for the direct forms):
 * every valid (forward kernel, column block, stages) candidate, then the
 * adjoint depth, each timed over `reps` (0: 3) objective + gradient
 * evaluations at image_dev with per-kernel CUDA events.  The fastest is kept
 * in the context and appended to a cache file (MEMSYNTH_TUNE_CACHE, default
 * $HOME/.cache/libmemsynth_tune.txt) that mem_create reads back for the same
 * device, N, visibility-count octave, channel count and form.  choice_out:
 * nullable, host. */
mem_status mem_autotune(mem_ctx *ctx, const float *image_dev, int32_t reps, mem_tiling_t *choice_out);

/* Set the tiling explicitly (ranges above; fwd_cols is ignored for
 * MEM_FWD_RESIDENT).  Waits for the context's stream.  MEM_EINVAL for a
 * direct form or an invalid choice. */
mem_status mem_set_tiling(mem_ctx *ctx, const mem_tiling_t *tiling);

/* The tiling in use.  The direct forms report the defaults, which they do
 * not use.  Defaults (before mem_autotune or a cached choice): for N <= 128
 * MEM_FWD_RESIDENT with the deepest pipeline that fits (mem_autotune keeps
 * the resident kernel there: it is the more accurate one, see above), for
 * N >= 256 MEM_FWD_STREAM with 256 columns and 4 stages; adjoint 3 stages. */
mem_status mem_tiling(const mem_ctx *ctx, mem_tiling_t *out);

/* CUDA graphs (default on): every repeated launch sequence (objective +
 * gradient for given image / gradient pointers, and the solver's evaluation,
 * curvature and line-search probe sequences) is captured once, on a private
 * stream, and replayed on the context stream.  Disabled while profiling. */
mem_status mem_use_graphs(mem_ctx *ctx, int32_t enable);

/* Kernel launches issued by ctx since creation (for launch accounting). */
int64_t mem_launch_count(const mem_ctx *ctx);

/* Per-kernel timing for measurement: when enabled, every kernel launch of ctx
 * is bracketed by CUDA events recorded on the context stream.
 * mem_profile_read synchronises the stream, writes up to max_kernels entries
 * (names: 32 chars each, NUL-terminated; total milliseconds; launch counts),
 * clears the accumulators and returns the number of entries (-1 on error). */
mem_status mem_profile(mem_ctx *ctx, int32_t enable);
int32_t mem_profile_read(mem_ctx *ctx, int32_t max_kernels, char *names, double *ms_total,
                         int64_t *launches);

/* Adjoint without device allocation (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory: code running inside a
 * framework that owns all device memory through its own pool or arena and
 * forbids side allocations, or code that must not allocate after start-up.
 * They keep their inputs and outputs in device memory themselves; this call
 * needs nothing else and calls no cudaMalloc / cudaFree or allocating library
 * routine.
 *
 * Computes, for one channel with the split-BF16 tensor-core form,
 *   img_dev[n*N + m] = pb_dev[n*N + m] * sum_k Re( y_k exp(+2 pi i (u_k x_m + v_k y_n)) )
 * (the same operation as mem_adjoint).  All pointers are device pointers:
 * u_dev, v_dev (n_vis doubles, wavelengths), y_dev (2*n_vis floats, re/im,
 * 8-byte aligned), pb_dev and img_dev (N*N floats).  N must be 64, 128 or
 * 256; other sizes return MEM_EINVAL with a message in mem_last_error(NULL).
 *
 * Scratch lives in a fixed static device array of about 16 MB (split-K
 * partials for at most 64 CTAs plus the work list) that every GPU loading the
 * library holds until exit.  All calls share it: calls that overlap on the
 * GPU race and must be serialised by the caller.  The array keeps the last
 * call's contents; nothing in it needs clearing between calls.  The first
 * call on a device resolves the array's device address (cudaGetSymbolAddress,
 * with that device current) and keeps it for the life of the process, so the
 * call must not be used after cudaDeviceReset.  `stream` must belong to the
 * device current at the call.  Every call uploads its work list from host
 * memory and reads a device status word back, synchronising `stream`: never
 * make it while `stream` (or, in global capture mode, any stream of the
 * process) is being captured.  Returns MEM_ETIMEOUT if a bounded device-side
 * wait ran out. */
mem_status mem_adjoint_noalloc(int32_t n, double dx, double dy, int64_t n_vis,
                               const double *u_dev, const double *v_dev, const float *y_dev,
                               const float *pb_dev, float *img_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBMEMSYNTH_H */
