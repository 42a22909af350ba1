/*
 * hcgs.h — C ABI of libhcgs, the B300 (sm_103a) implementation of the
 * hologram render path of "Complex-Valued Holographic Radiance Fields"
 * (arXiv 2506.08350).
 *
 * The path renders, for each view, a complex hologram P (Sec. 3, problem
 * statement: P in C^{nx x ny}, pose r, pixel pitch dx) from N complex-valued
 * 3D Gaussians in four steps:
 *   1. project      (Sec. 3 Eq. gaussian_projection / gaussian_projection_2d,
 *                    Eq. hard_assignment)                      -> hcgs_project
 *   2. depth-sort and bin per plane into 64x64-pixel buckets, each bucket's
 *                    list in visiting order (Sec. 4.2, Algorithm 2
 *                    preprocessing)                          -> hcgs_project
 *   3. composite complex footprints into L plane fields (Sec. 4.1 per-plane
 *                    field equation, Algorithm 2)             -> hcgs_rasterize_planes
 *   4. propagate each plane by the band-limited angular spectrum method and
 *                    sum (Eq. band_limited_asm_transfer_function,
 *                    Eq. layer2plane_asm, Eq. sum_planes)     -> hcgs_asm_propagate
 * hcgs_render_view runs all four.  Every step has a _backward twin (Supp.
 * D.4, Eq. ste).  The training-step pieces are hcgs_focal_stack_loss
 * (Eq. plane2layer_asm, Eq. recon_loss) and hcgs_adam_step, and the paper's
 * own recipe: hcgs_paper_loss (L_recon + L_SSIM, Sec. 4.1) and hcgs_adan_step
 * (Sec. 5); Algorithm 1's densification is hcgs_densify_accumulate / _plan /
 * _apply with hcgs_philox for its noise; the phase-only conversion of Sec. 6
 * is hcgs_phase_only_loss; the learned initialisation network is
 * hcgs_mlp_forward / hcgs_mlp_backward.  Options select the zero-padded
 * propagation (hcgs_optics.padding), the FP16x2 / BF16x2 footprint tiers and the dense
 * plane-weight gradient (hcgs_raster_opts.footprint, .rho_grad).
 *
 * Conventions (all entry points):
 *  - Memory: every array argument marked "device" is a device pointer owned
 *    by the caller; arrays marked "host" are host memory read during the call.
 *    The library allocates device memory only for its own scratch (the
 *    context workspace and the buffers held by an hcgs_saved), grows it on
 *    demand, and frees it in hcgs_saved_release / hcgs_ctx_destroy.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Work is enqueued asynchronously.  hcgs_project synchronises `stream`
 *    once to read the number of tile instances (it sizes the instance list).
 *  - Complex numbers are interleaved (re, im) float pairs, i.e. the layout of
 *    torch.complex64.  An upstream gradient of a real loss w.r.t. a complex
 *    array z is passed as g = dL/dRe(z) + j dL/dIm(z) (Supp. D.4 uses the
 *    separate dL/dreal, dL/dimag).
 *  - Units: metres for wavelengths, pitch, plane distances, means and scales;
 *    pixels for intrinsics.  Pixel (row i, col j) has its centre at x = j,
 *    y = i.  Camera axes: x right, y down, z forward (world -> camera 4x4,
 *    row-major).
 *  - Errors: every call returns an hcgs_status; no exception crosses the ABI.
 *    Arguments are validated before any launch.  CUDA errors map to
 *    HCGS_ERR_CUDA and the message is kept for hcgs_last_error.
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef HCGS_H
#define HCGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HCGS_OK = 0,
    HCGS_ERR_INVALID_ARG = -1,     /* null pointer, bad size, bad option            */
    HCGS_ERR_CUDA = -2,            /* a CUDA runtime call failed                    */
    HCGS_ERR_CAPACITY = -3,        /* scratch could not be allocated                */
    HCGS_ERR_UNSUPPORTED_SIZE = -4,/* FFT length with a prime factor other than 2,3,5,
                                      or larger than 4096                           */
    HCGS_ERR_DEVICE_CHECK = -5,    /* a kernel's own bounds check fired             */
    HCGS_ERR_TIMEOUT = -6,         /* a bounded device wait ran out in an earlier
                                      launch of the context (reported at the
                                      next hcgs_project / hcgs_render_view)    */
    HCGS_ERR_STATE = -7            /* saved state missing or from another shape     */
} hcgs_status;

typedef struct hcgs_ctx hcgs_ctx;     /* scratch workspace, transfer-function cache */
typedef struct hcgs_saved hcgs_saved; /* forward state that the backward reuses     */

/* Hologram-plane sampling and depth planes (Sec. 3 problem statement:
 * q = (r, dx, nx, ny); Sec. 4.1 layer construction: L planes parallel to the
 * hologram, each sampled on the hologram grid). */
typedef struct {
    int H, W;                 /* ny, nx: rows and columns of every plane        */
    int C;                    /* number of wavelengths (colour channels), 1..4  */
    int L;                    /* number of depth planes, 1..16                  */
    double pitch_x, pitch_y;  /* pixel pitch (m)                                */
    const double* wavelength; /* host [C] (m)                                   */
    const double* plane_z;    /* host [L] (m): Z_l, distance plane l -> hologram */
    int band_limit;           /* 0: Eq. band_limited_asm_transfer_function as
                                 printed (evanescent cut f^2 <= 1/lambda^2);
                                 1: also the band limit of Matsushima and
                                 Shimobaba, the reference the paper cites for
                                 the method: with du = 1/(n pitch) on an n-sample
                                 axis, H is kept only where |f| <= 1/(lambda
                                 sqrt((2 du z)^2 + 1)) on both axes (inactive
                                 at 8 um pitch for the paper-shaped grids);
                                 other values: HCGS_ERR_INVALID_ARG            */
    int padding;              /* 0: circular convolution on the H x W grid (the
                                 DFTs of the equations taken on the grid as is);
                                 1: linear convolution: every propagation runs on
                                 a 2H x 2W grid with the field at rows H/2 ..
                                 H/2 + H - 1, columns W/2 .. W/2 + W - 1 and zeros
                                 elsewhere, H_z (and the band limit) on that
                                 grid's frequencies, the same window cropped
                                 back; 2H and 2W must be supported FFT lengths.
                                 Not available in hcgs_asm_propagate_noalloc. */
} hcgs_optics;

/* Rasterizer options.  Values the paper leaves unstated (Algorithm 2 names
 * eps_plane and eps_T without values) default to the 3DGS constants. */
typedef struct {
    int tile;                 /* must be 16 (Sec. 4.2: 16x16 tiles)             */
    float alpha_min;          /* skip a Gaussian at a pixel when alpha < this (1/255) */
    float alpha_max;          /* alpha = min(alpha_max, o G) (0.99); the min is
                                 taken for Gaussians whose opacity exceeds
                                 alpha_max (1 - 2^-10), below which o G <= o
                                 cannot reach it up to rounding               */
    float T_eps;              /* stop a pixel once T < T_eps, after the add (1e-4) */
    float cov2d_dilation;     /* added to the diagonal of Sigma' (0.3 px^2)     */
    float near_z;             /* cull when camera-space z < near_z (0.2 m)      */
    float clip_factor;        /* clamp of x/z, y/z in J (1.3; <= 0: no clamp)   */
    float ste_tau;            /* softmax temperature of Eq. ste (1e-3)          */
    int order;                /* 0 front-to-back (nearest first), 1 back-to-front */
    int footprint;            /* 0 FP32 footprint; 1 FP16x2 and 2 BF16x2 footprint
                                 (in the footprint's normalised frame the part
                                 of the exponent that varies along a pixel
                                 column and its exp() in packed half / bfloat16
                                 precision, the part constant along the column
                                 in FP32) with FP32 accumulation               */
    int rho_grad;             /* 0: only the assigned plane's rho gets gradient
                                 (the forward skips the other planes);
                                 1: dense plane-weight gradient: every plane's
                                 logit also receives dL/drho_l of compositing
                                 with continuous weights (alpha_eff = alpha
                                 rho_l) at the one-hot argmax weights, through
                                 the same straight-through rule; costs an
                                 all-plane binning and an extra pass that walks
                                 every plane against every Gaussian of a tile  */
} hcgs_raster_opts;

/* Gaussian parameters k = (c, x, R, S, alpha, phi, rho') (Sec. 4.1), device,
 * float32, structure of arrays. */
typedef struct {
    const float* means;          /* [N][3] world position (m)                    */
    const float* log_scales;     /* [N][3] S = diag(exp(log_scales))             */
    const float* quats;          /* [N][4] rotation (w, x, y, z), any norm > 0   */
    const float* opacity_logits; /* [N]    alpha_base = sigmoid(logit)           */
    const float* amplitude;      /* [N][C] c_n, wave amplitude per wavelength    */
    const float* phase;          /* [N][C] phi_n (rad) per wavelength            */
    const float* plane_logits;   /* [N][L] rho'_n; rho_n = OneHot(argmax rho'_n) */
    int N;
} hcgs_gaussians;

/* Gradients w.r.t. the arrays of hcgs_gaussians, device float32, same shapes.
 * Overwritten, or added to when `accumulate` is non-zero. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *amplitude, *phase, *plane_logits;
} hcgs_gaussian_grads;

/* ---------------- context ---------------- */
/* Creates a context on `device` (made current for the call).  Destroying it
 * (and releasing a saved state) first waits for the work the context's
 * launches enqueued, on every stream they used (not for the whole device),
 * then frees its buffers. */
hcgs_status hcgs_ctx_create(hcgs_ctx** ctx, int device);
void hcgs_ctx_destroy(hcgs_ctx* ctx);
const char* hcgs_status_string(hcgs_status s);
/* Message of the last failing call on this context (empty if none). */
const char* hcgs_last_error(hcgs_ctx* ctx);
/* Bytes of device scratch the context and its saved states hold. */
size_t hcgs_ctx_bytes(hcgs_ctx* ctx);
/* Creates an empty forward state; hcgs_project and hcgs_render_view fill it
 * and reuse its buffers when called again with the same handle. */
hcgs_status hcgs_saved_create(hcgs_ctx* ctx, hcgs_saved** saved);
hcgs_status hcgs_saved_release(hcgs_ctx* ctx, hcgs_saved* saved);

/* Per-kernel timing.  While enabled, every kernel launch of this context is
 * bracketed by two CUDA events on its stream.  hcgs_profile_summary waits
 * for the recorded events, writes for up to `max` kernels (in first-launch
 * order) the name (static strings owned by the library), the summed device
 * time in ms and the number of launches, sets *n_out, and clears the record. */
/* Self-test of the bounded waits: launches, on `stream`, one kernel that
 * waits on a shared-memory barrier nothing completes.  Its wait gives up
 * after about one second of SM clock and sets the context's status word, as
 * the FFT row passes and the SSIM passes of hcgs_paper_loss /
 * hcgs_paper_loss_intensities / hcgs_phase_only_loss do when a bulk or tensor
 * copy never arrives (they leave without writing); the next hcgs_project or
 * hcgs_render_view on the context then returns HCGS_ERR_TIMEOUT (and clears
 * the word), and the calls after it work again.  Returns HCGS_OK once the
 * kernel is launched; HCGS_ERR_INVALID_ARG for a null context. */
hcgs_status hcgs_selftest_wait_timeout(hcgs_ctx* ctx, void* stream);

/* ---------------- bounds-checked build (no counterpart in the paper) ---------------- */
/* libhcgs_checked.so is the same library compiled with HCGS_CHECKED: device
 * kernels check the indices they take from data (bucket-list entries, strip
 * lengths, visiting ranks, instance offsets) before using them and skip an
 * access whose check fails, the projection checks that every Gaussian
 * parameter is finite (a non-finite Gaussian is reported and culled), and
 * every buffer the library grows carries a 256-byte guard band after its
 * capacity.  A failed check sets the context's status word.
 * hcgs_is_checked_build: 1 in libhcgs_checked.so, 0 in libhcgs.so.
 * hcgs_check_status: synchronises `stream`, verifies the guard bands of this
 *   device's library buffers (checked build; a damaged band is reported and
 *   filled again), reads and clears the status word.  Returns
 *   HCGS_ERR_DEVICE_CHECK if a check failed since the last report,
 *   HCGS_ERR_TIMEOUT if a bounded device wait ran out, else HCGS_OK; the
 *   context stays usable.  (hcgs_project / hcgs_render_view also report the
 *   word at their own readback, which follows the projection: a non-finite
 *   Gaussian makes that very call return HCGS_ERR_DEVICE_CHECK.)
 * hcgs_selftest_device_check: checked build only (else HCGS_ERR_STATE).
 *   kind 0 launches a kernel whose index check fails (the index is outside
 *   the checked range but inside its buffer); kind 1 writes one byte into
 *   the guard band of a context buffer (inside the allocation).  The next
 *   hcgs_check_status returns HCGS_ERR_DEVICE_CHECK.  No access leaves its
 *   allocation in either case. */
int hcgs_is_checked_build(void);
hcgs_status hcgs_check_status(hcgs_ctx* ctx, void* stream);
hcgs_status hcgs_selftest_device_check(hcgs_ctx* ctx, int kind, void* stream);

hcgs_status hcgs_profile_enable(hcgs_ctx* ctx, int on);
hcgs_status hcgs_profile_summary(hcgs_ctx* ctx, int max, int* n_out, const char** names, double* ms,
                                 int64_t* launches);

/* ---------------- step 1+2: projection, depth sort, tile binning ---------------- */
/* Projects the N Gaussians for V views (Eq. gaussian_projection:
 * Sigma' = J W Sigma W^T J^T, mu = projection of the mean; Eq. hard_assignment
 * for the plane), culls (z < near_z), sorts by camera-space depth (the
 * depth z of the mean formed in FP64 from the FP32 inputs and rounded once
 * to FP32; equal keys by index) and bins every Gaussian into the 64x64-pixel
 * buckets of its plane that the 16x16 tiles its support
 * {p : o G(p) >= alpha_min} can touch lie in; the compositing tests the tile
 * rectangle and the support again per 16x8 strip.
 *   viewmats   device [V][4][4] world -> camera, row-major
 *   intrinsics device [V][4]    (f_x, f_y, c_x, c_y) in pixels
 * The result lives in `saved` (must come from hcgs_saved_create). */
hcgs_status hcgs_project(hcgs_ctx* ctx, const hcgs_gaussians* g, int V, const float* viewmats,
                         const float* intrinsics, const hcgs_optics* optics,
                         const hcgs_raster_opts* opts, hcgs_saved* saved, void* stream);

/* ---------------- step 3: complex multi-plane compositing ---------------- */
/* Composites every plane of every view (Sec. 4.1 per-plane field equation;
 * Algorithm 2): per pixel and plane, in depth order, alpha = min(alpha_max,
 * o exp(-power)); skip if alpha < alpha_min; U += c e^{j phi} alpha T;
 * T *= 1 - alpha; stop once T < T_eps.
 *   U          device [V][L][C][H][W] complex64 (output)
 *   T_final    device [V][L][H][W] float, nullable (output)
 *   n_contrib  device [V][L][H][W] int32, nullable: number of Gaussians that
 *              added to the pixel (output)
 * Requires a prior hcgs_project on `saved`. */
hcgs_status hcgs_rasterize_planes(hcgs_ctx* ctx, hcgs_saved* saved, float* U, float* T_final,
                                  int32_t* n_contrib, void* stream);

/* ---------------- step 4: band-limited ASM ---------------- */
/* Two forms (B = batch of views; H_z of Eq. band_limited_asm_transfer_function,
 * formed in FP64 and reduced mod 2 pi, applied in FP32; unnormalised forward
 * DFT, 1/(H W) on the inverse; no padding):
 *   sign = +1, reduce_planes = 1 (forward recording, Eq. layer2plane_asm +
 *     Eq. sum_planes):  in [B][L][C][H][W] -> out [B][C][H][W],
 *     out = sum_l IDFT(H_{Z_l} DFT(in_l))
 *   sign = -1, reduce_planes = 0 (inverse propagation, Eq. plane2layer_asm):
 *     in [B][C][H][W] -> out [B][L][C][H][W], out_l = IDFT(H_{-Z_l} DFT(in))
 * `in` is not modified; `out` must not alias `in`. */
hcgs_status hcgs_asm_propagate(hcgs_ctx* ctx, const float* in, int B, const hcgs_optics* optics,
                               int sign, int reduce_planes, float* out, void* stream);
/* Adjoint of hcgs_asm_propagate with the same (sign, reduce_planes):
 * g_out has the shape of `out`, g_in the shape of `in`; for the forward form
 * g_in_l = IDFT(conj(H_{Z_l}) DFT(g_out)). */
hcgs_status hcgs_asm_propagate_backward(hcgs_ctx* ctx, const float* g_out, int B,
                                        const hcgs_optics* optics, int sign, int reduce_planes,
                                        float* g_in, void* stream);

/* ---------------- all four steps ---------------- */
/*   hologram  device [V][C][H][W] complex64 (output)
 *   planes    device [V][L][C][H][W] complex64, nullable (output of step 3)
 *   saved     nullable: with a handle, the forward state is kept for
 *             hcgs_render_view_backward; with NULL an internal one is used. */
hcgs_status hcgs_render_view(hcgs_ctx* ctx, const hcgs_gaussians* g, int V, const float* viewmats,
                             const float* intrinsics, const hcgs_optics* optics,
                             const hcgs_raster_opts* opts, float* hologram, float* planes,
                             hcgs_saved* saved, void* stream);

/* ---------------- adjoints ---------------- */
/* Adjoint of step 3 (Supp. D.4; backward walks each pixel's contributors in
 * reverse and recovers T by division, Sec. 4.2).  gU device [V][L][C][H][W]
 * complex64.  The per-Gaussian 2D gradients stay in `saved`. */
hcgs_status hcgs_rasterize_planes_backward(hcgs_ctx* ctx, hcgs_saved* saved, const float* gU,
                                           void* stream);
/* Adjoint of steps 1-2 (Supp. D.4 chain to q, x, S, c, phi, alpha_base; Eq. ste
 * for rho': dL/drho' = dL/drho * softmax(rho'/tau), elementwise).  Sums over
 * the views of `saved`.  `g` must be the parameters hcgs_project saw. */
hcgs_status hcgs_project_backward(hcgs_ctx* ctx, hcgs_saved* saved, const hcgs_gaussians* g,
                                  const hcgs_gaussian_grads* grads, int accumulate, void* stream);
/* Adjoint of hcgs_render_view: g_hologram device [V][C][H][W] complex64. */
hcgs_status hcgs_render_view_backward(hcgs_ctx* ctx, hcgs_saved* saved, const hcgs_gaussians* g,
                                      const float* g_hologram, const hcgs_gaussian_grads* grads,
                                      int accumulate, void* stream);

/* ---------------- training step ---------------- */
/* Focal-stack intensity loss (Eq. plane2layer_asm, I_l = |U_{P->l}|^2,
 * Eq. recon_loss as a mean over planes, channels and pixels):
 *   hologram device [B][C][H][W] complex64
 *   I_gt     device [B][L][C][H][W] float
 *   loss     device float[1] (output)
 *   g_hologram device [B][C][H][W] complex64, nullable: dL/dP (output)
 *   I_out    device [B][L][C][H][W] float, nullable (output) */
hcgs_status hcgs_focal_stack_loss(hcgs_ctx* ctx, const float* hologram, const float* I_gt, int B,
                                  const hcgs_optics* optics, float* loss, float* g_hologram,
                                  float* I_out, void* stream);
/* The paper's training objective on one batch of views (Sec. 4.1, loss):
 * the focal stack I_l = |V_l|^2, V_l = ASM(P, -z_l) (Eq. plane2layer_asm),
 * against the targets, with L = L_recon + L_SSIM averaged over views:
 *   L_recon = mean over (b, l, c, pixel) of d^2 (1 + M + I_gt^2), d = I - I_gt
 *             (the sum |I - I_gt|^2 + |I M - I_gt M|^2 + |I I_gt - I_gt I_gt|^2
 *             for a binary M);
 *   L_SSIM  = lambda_ssim mean over (b, l, c) of (1 - SSIM(I, I_gt)), SSIM
 *             with an 11 x 11 Gaussian window (sigma 1.5, zeros outside the
 *             image), C1 = 0.01^2, C2 = 0.03^2, averaged over the pixels.
 *   hologram device [B][C][H][W] complex64
 *   I_gt     device [B][L][C][H][W] float
 *   masks    device [B][L][H][W] float (0 or 1: pixels whose depth falls on
 *            plane l), nullable = all zero
 *   lambda_ssim >= 0 (the paper's lambda_1 = 0.005)
 *   loss     device [1] float (output)
 *   g_hologram device [B][C][H][W] complex64, nullable: dL/dP (output)
 *   I_out    device [B][L][C][H][W] float, nullable (output)
 * Scratch: 2 B C H W + 2 B L C H W complex and 4 B L C H W floats (3 when
 * I_out is given), held by the context. */
hcgs_status hcgs_paper_loss(hcgs_ctx* ctx, const float* hologram, const float* I_gt, const float* masks, int B,
                            const hcgs_optics* optics, float lambda_ssim, float* loss, float* g_hologram,
                            float* I_out, void* stream);
/* The same objective on given intensities I device [B][L][C][H][W] float (any
 * H, W >= 1; B L C H W < 2^29): loss device [1] and g_I = dL/dI device
 * [B][L][C][H][W] float (outputs); I_gt and masks as in hcgs_paper_loss. */
hcgs_status hcgs_paper_loss_intensities(hcgs_ctx* ctx, const float* I, const float* I_gt, const float* masks,
                                        int B, int L, int C, int H, int W, float lambda_ssim, float* loss,
                                        float* g_I, void* stream);
/* One Adan update (Xie et al., Algorithm 1; the optimiser of Sec. 5) of count
 * float32 parameters in place, with decay factors b1 (first moment), b2
 * (gradient difference) and b3 (second moment).  Sec. 5 gives two values,
 * 0.9 and 0.99, read as b1 and b3; it is silent on b2, for which Adan's own
 * default 0.92 is the usual choice:
 *   step 1: m = g, v = 0, n = g^2;  step 2: v = g - g_prev;
 *   then m = b1 m + (1-b1) g, v = b2 v + (1-b2)(g - g_prev),
 *        n = b3 n + (1-b3)(g + b2 (g - g_prev))^2  (m, n also at step 2);
 *   p = (p - lr (m + b2 v) / (sqrt(n) + eps)) / (1 + weight_decay lr);
 *   g_prev = g.
 * All arrays device [count] float; g_prev, m, v, n are the caller's state
 * (any contents at step 1). */
hcgs_status hcgs_adan_step(hcgs_ctx* ctx, float* p, const float* g, float* g_prev, float* m, float* v,
                           float* n, int64_t count, int step, float lr, float beta1, float beta2, float beta3,
                           float eps, float weight_decay, void* stream);
/* One bias-corrected Adam update of n float32 parameters in place:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr m^ / (sqrt(v^) + eps),
 * m^ = m/(1-b1^step), v^ = v/(1-b2^step).  All arrays device [n]. */
hcgs_status hcgs_adam_step(hcgs_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n,
                           int step, float lr, float beta1, float beta2, float eps, void* stream);
/* hcgs_adam_step on k parameter arrays in one launch (0 <= k <= 16): array a
 * is p[a], g[a], m[a], v[a] (device [count[a]] float) with learning rate
 * lr[a]; the pointer tables p, g, m, v and count, lr are host [k] arrays,
 * read during the call.  Each element is updated exactly as by
 * hcgs_adam_step.  The arrays must not overlap.  Errors as hcgs_adam_step;
 * k outside [0, 16] -> HCGS_ERR_INVALID_ARG. */
hcgs_status hcgs_adam_step_multi(hcgs_ctx* ctx, int k, float* const* p, const float* const* g, float* const* m,
                                 float* const* v, const int64_t* count, const float* lr, int step, float beta1,
                                 float beta2, float eps, void* stream);
/* hcgs_adan_step on k parameter arrays in one launch (0 <= k <= 16), tables
 * as in hcgs_adam_step_multi (g_prev, n: the Adan state of each array);
 * each element is updated exactly as by hcgs_adan_step with lr[a]. */
hcgs_status hcgs_adan_step_multi(hcgs_ctx* ctx, int k, float* const* p, const float* const* g, float* const* g_prev,
                                 float* const* m, float* const* v, float* const* n, const int64_t* count,
                                 const float* lr, int step, float beta1, float beta2, float beta3, float eps,
                                 float weight_decay, void* stream);

/* ---------------- learned initialisation network (no counterpart in the paper) ---------------- */
/* 4-layer ReLU MLP, width 128, BF16 operands with FP32 accumulation:
 * 16 -> 128 -> 128 -> 128 -> 16 (last layer linear).
 *   x   device [N][16] bf16 (features: mean 3, log-scale 3, quaternion 4,
 *       opacity logit 1, RGB 3, padding 2)
 *   W1  device [128][16], W2, W3 [128][128], W4 [16][128] bf16 (row = output)
 *   b1, b2, b3 device [128], b4 [16] float
 *   y   device [N][16] float (output)
 * 0 <= N <= 2^30 (row indices stay in 32-bit arithmetic), else
 * HCGS_ERR_INVALID_ARG; the same bound holds for hcgs_mlp_backward. */
hcgs_status hcgs_mlp_forward(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* W1,
                             const uint16_t* W2, const uint16_t* W3, const uint16_t* W4,
                             const float* b1, const float* b2, const float* b3, const float* b4,
                             float* y, void* stream);
/* Reverse mode of hcgs_mlp_forward for upstream gy device [N][16] float.
 * Writes (overwrites) gW1..gW4 (float, shapes of W1..W4) and gb1..gb4. */
hcgs_status hcgs_mlp_backward(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* W1,
                              const uint16_t* W2, const uint16_t* W3, const uint16_t* W4,
                              const float* b1, const float* b2, const float* b3, const float* b4,
                              const float* gy, float* gW1, float* gW2, float* gW3, float* gW4,
                              float* gb1, float* gb2, float* gb3, float* gb4, void* stream);

/* Training of the network (no counterpart in the paper): mean squared error
 * of the first K (1..16) of the 16 output columns against target, both device
 * [N][16] float; writes loss (device float[1]) and gy = dL/dy (device
 * [N][16] float, zero in the unused columns). */
hcgs_status hcgs_mlp_mse_loss(hcgs_ctx* ctx, const float* y, const float* target, int N, int K, float* loss,
                              float* gy, void* stream);
/* Rounds n device floats to bfloat16 (nearest, ties to even): the network's
 * FP32 master weights -> the BF16 operands of hcgs_mlp_forward. */
hcgs_status hcgs_cast_bf16(hcgs_ctx* ctx, const float* src, uint16_t* dst, int64_t n, void* stream);

/* Marshalling of the network's data (no counterpart in the paper).
 * hcgs_init_features: x device [N][16] bf16 = (mean 3, (log_scale + 4)/0.5 3,
 *   unit quaternion 4, opacity logit 1, rgb 3, 0, 0) from g and rgb device [N][3].
 * hcgs_init_targets: target device [N][16] float = (a_c cos phi_c, a_c sin phi_c)
 *   for c < C, zero after, from amplitude/phase device [N][C].
 * hcgs_init_apply: amplitude = |w_c|, phase = arg w_c from y device [N][16]. */
hcgs_status hcgs_init_features(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* rgb, uint16_t* x,
                               void* stream);
hcgs_status hcgs_init_targets(hcgs_ctx* ctx, const float* amplitude, const float* phase, int N, int C,
                              float* target, void* stream);
hcgs_status hcgs_init_apply(hcgs_ctx* ctx, const float* y, int N, int C, float* amplitude, float* phase,
                            void* stream);

/* ---------------- allocation-free inverse propagation ---------------- */
/* The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, for example an application whose device memory is
 * all owned by its own pool allocator (an allocation from inside a library
 * would fail or fragment that pool), or a display loop that allocates at
 * start-up and must not stall on cudaMalloc/cudaFree (they synchronise the
 * device) mid-frame.  It needs no context and allocates nothing.
 * Result: the same as hcgs_asm_propagate(ctx, in, B, optics, -1, 0, out,
 * stream), i.e. out[b][l][c] = IDFT(H_{-Z_l} DFT(in[b][c])):
 *   in   device [B][C][H][W] complex64, not modified
 *   out  device [B][L][C][H][W] complex64, must share no byte with `in`
 * Working memory (column spectrum, transfer-function table, twiddles) lives
 * in one static device array of 4 Mi complex64 values (32 MiB) that every GPU
 * loading the library holds until exit.  Requests needing more, i.e.
 *   B*C*H*W + C*L*(H/2+1)*S + H + W (each rounded up to 64) > 4194304, with
 *   S = W/2 + 1 rounded up to even (the table's row stride),
 * return HCGS_ERR_CAPACITY before any launch.  The first call on a device
 * (and again the first after that device's context was destroyed and made
 * anew, e.g. by cudaDeviceReset) looks up that device's address of the array
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (each call rewrites what it reads), so
 * calls whose kernels overlap on the GPU race: serialise them.  Errors:
 * HCGS_ERR_INVALID_ARG (NULL pointers, `in` and `out` overlapping, B < 1,
 * bad optics),
 * HCGS_ERR_UNSUPPORTED_SIZE (H or W not 2^a 3^b 5^c <= 4096),
 * HCGS_ERR_CAPACITY (too large), HCGS_ERR_CUDA (a CUDA call failed). */
hcgs_status hcgs_asm_propagate_noalloc(const float* in, int B, const hcgs_optics* optics, float* out,
                                       void* stream);

/* ---------------- phase-only hologram conversion (Sec. 6) ---------------- */
/* Objective of the conversion of a complex hologram P = A e^{j phi} into a
 * phase-only one e^{j phi_opt}: both are propagated to the planes,
 * U_l = IDFT(H_{-Z_l} DFT(P)) (the target, given) and U_phi,l the same of
 * e^{j phase}, and
 *   L = mean over (b, l, c, part, pixel) of (part(U_phi) - part(U))^2
 *       + lambda_ssim mean over (b, l, c, part) of (1 - SSIM(part(U_phi), part(U))),
 * part = the real and the imaginary component (the SSIM of hcgs_paper_loss).
 *   U_target device [B][L][C][H][W] complex64 (e.g. hcgs_asm_propagate with
 *            sign -1, reduce_planes 0, of the complex hologram)
 *   phase    device [B][C][H][W] float (rad)
 *   loss     device [1] float (output)
 *   g_phase  device [B][C][H][W] float, nullable: dL/dphase (output) */
hcgs_status hcgs_phase_only_loss(hcgs_ctx* ctx, const float* U_target, const float* phase, int B,
                                 const hcgs_optics* optics, float lambda_ssim, float* loss, float* g_phase,
                                 void* stream);
/* phase[i] = arg(hologram[i]) in (-pi, pi]: hologram device [n] complex64,
 * phase device [n] float (the starting point of the conversion). */
hcgs_status hcgs_hologram_phase(hcgs_ctx* ctx, const float* hologram, int64_t n, float* phase, void* stream);
/* out[i] = s x[i] for n floats (device; out may equal x), e.g. to normalise
 * a complex hologram's RMS amplitude to 1 before the conversion. */
hcgs_status hcgs_scale(hcgs_ctx* ctx, const float* x, int64_t n, float s, float* out, void* stream);
/* hologram[i] = e^{j phase[i]}: phase device [n] float, hologram device [n]
 * complex64 (the phase-only hologram an SLM displays). */
hcgs_status hcgs_phase_hologram(hcgs_ctx* ctx, const float* phase, int64_t n, float* hologram, void* stream);

/* ---------------- densification (Algorithm 1, Supp. D.2) ---------------- */
/* The 3DGS densification rules that Sec. 5 adopts (period: 300 steps),
 * with phase-aware copies (Supp. D.2: copies and children get a small random
 * phase perturbation). */
typedef struct {
    float grad_threshold; /* densify when the mean NDC gradient norm of the 2D mean >= this (2e-4) */
    float split_scale;    /* split when the largest scale exp(log_scale) > this (m), else clone  */
    float prune_opacity;  /* prune when sigmoid(opacity_logit) < this (0.005)                 */
    float prune_scale;    /* prune when the largest scale > this (m); <= 0: no size pruning   */
    float split_shrink;   /* children's scales are the parent's / split_shrink (1.6)          */
    float phase_noise;    /* standard deviation of the phase perturbation (rad)               */
} hcgs_densify_opts;
#define HCGS_DENSIFY_MAX_EXTRA 32

/* Adds the last backward pass's screen-space statistics: for every view of
 * `saved` in which Gaussian n is visible, accum[n] += |(dL/dmu_x W/2,
 * dL/dmu_y H/2)| (the gradient w.r.t. the 2D mean in normalised device
 * coordinates) and denom[n] += 1.  accum, denom device [N] float (in/out).
 * Needs hcgs_rasterize_planes_backward (or hcgs_render_view_backward) on
 * `saved` first (HCGS_ERR_STATE otherwise). */
hcgs_status hcgs_densify_accumulate(hcgs_ctx* ctx, hcgs_saved* saved, float* accum, float* denom, void* stream);
/* Decides every Gaussian's fate and sizes the output: action device [N]
 * int32 (out: 0 keep, 1 prune, 2 clone, 3 split), offsets device [N + 1]
 * uint32 (out: exclusive prefix sum of 1 / 0 / 2 / 2 outputs per Gaussian;
 * offsets[N] = the new count), *n_out (host, out) the new count.  Decisions
 * in FP32: prune if sigmoid(logit) < prune_opacity or (prune_scale > 0 and
 * the largest scale > prune_scale); otherwise densify if denom > 0 and
 * accum / denom >= grad_threshold, splitting when the largest scale >
 * split_scale.  Synchronises `stream` once to read the count. */
hcgs_status hcgs_densify_plan(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* accum, const float* denom,
                              const hcgs_densify_opts* opts, int32_t* action, uint32_t* offsets,
                              int64_t* n_out, void* stream);
/* Writes the new Gaussians: output offsets[n] onward receives, for a kept
 * Gaussian, its copy; for a clone, the original then a copy with phases
 * phi + phase_noise noise[n][0][3 + c]; for a split, two children k = 0, 1
 * with means mu + R diag(exp(log_scales)) noise[n][k][0:3] (R of the
 * normalised quaternion), log-scales - log(split_shrink), phases phi +
 * phase_noise noise[n][k][3 + c], the rest copied; pruned Gaussians write
 * nothing.  noise device [N][2][3 + C] float standard normals (e.g.
 * hcgs_philox).  g_out: the output arrays (device, n_out rows; the struct of
 * writable arrays), must not alias g_in.  extra_in / extra_out: host arrays
 * of n_extra (<= HCGS_DENSIFY_MAX_EXTRA) device pointers to per-Gaussian
 * float arrays of extra_width[e] columns (optimiser state): copied for kept
 * Gaussians and clone originals, zero for copies and children. */
hcgs_status hcgs_densify_apply(hcgs_ctx* ctx, const hcgs_gaussians* g_in, int C, int L, const int32_t* action,
                               const uint32_t* offsets, const float* noise, const hcgs_densify_opts* opts,
                               const hcgs_gaussian_grads* g_out, int n_extra, const float* const* extra_in,
                               float* const* extra_out, const int* extra_width, void* stream);
/* Counter-based random numbers (Philox4x32-10 of Salmon et al., SC'11): word
 * block b of stream (seed, stream_id) is Philox(counter (b, stream_id, 0, 0),
 * key (seed low 32 bits, seed high 32 bits)), four uint32 words per block.
 * kind 0: out device [n] uint32, the words in order; kind 1: out device [n]
 * float standard normals, each word pair (a, b) giving, with u = (a + 1/2)
 * 2^-32, v = (b + 1/2) 2^-32, sqrt(-2 ln u) (cos 2 pi v, sin 2 pi v);
 * kind 2: out device [n] float uniforms (w + 1/2) 2^-32 in (0, 1). */
hcgs_status hcgs_philox(hcgs_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, int kind, void* out,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HCGS_H */
