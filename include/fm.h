/*
 * fm.h -- C ABI of the GB300 regularised field-map estimator.
 *
 * Method: Lin & Fessler, "Efficient Regularized Field Map Estimation in 3D MRI"
 * (arXiv 2005.08661).  Given multi-echo (optionally multi-coil) images y_clj, coil
 * maps s_cj and echo times t_l (Sec. II, Eq. 1), it minimises
 *     Psi(w) = Phi(w) + beta/2 ||C w||^2                                   (Eq. 5)
 *     Phi(w) = sum_j sum_{m,n} sum_{c,d} |r_cdmnj| (1 - cos(angle r_cdmnj + w_j (t_m - t_n)))
 *                                                                          (Eq. 2, r: Eq. 3)
 * with C the 3-D first-order finite differences between 6-neighbours inside the
 * support mask, by preconditioned Polak-Ribiere nonlinear CG with the monotonic
 * line search (Algorithm box, Sec. III-C, Eq. 13-16) and an IC(0) preconditioner
 * of H = diag(d) + beta C'C (Sec. III-B, Eq. 9-12).
 *
 * Conventions shared by every entry point
 *   - Volumes are nx * ny * nz voxels, x fastest: voxel (x, y, z) is element
 *     x + nx * (y + ny * z).  Arrays are dense and contiguous; no strides.
 *   - Precision (fm_opts.precision): FM_FP32 -> voxel arrays are float and images
 *     are complex64 (interleaved float re, im); FM_FP64 -> double / complex128.
 *     In FM_FP32 mode every global sum (cost, dot products, line-search sums) and
 *     the IC(0) pivot recurrence are carried in double.
 *   - "device" pointers are CUDA device (or managed) memory of the context's
 *     device; "host" pointers are ordinary host memory.  Caller arrays are
 *     borrowed for the duration of the call only; the context owns everything it
 *     allocates.
 *   - Work is enqueued on the context's stream.  Calls that return a host value
 *     (cost, cost history) synchronise that stream; the others return once the
 *     work is enqueued, except that every call reports errors found by earlier
 *     kernels of the same context at its next synchronisation.
 *   - Field maps are in radians per unit of the echo times (echo times in ms ->
 *     rad/ms).  Voxels outside the mask are not unknowns and are returned as 0.
 *   - Every function returns FM_OK (0) or a negative FM_ERR_* code and never
 *     aborts.  After an error the context can still be destroyed; FM_ERR_CUDA
 *     after a sticky device fault leaves the context unusable.
 */
#ifndef FM_H
#define FM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FM_API __attribute__((visibility("default")))
#else
#define FM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FM_OK 0
#define FM_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad option) */
#define FM_ERR_STATE (-2)     /* call order wrong, e.g. a solve before fm_set_data */
#define FM_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define FM_ERR_NOT_PD (-4)    /* an IC(0) pivot was <= 0 (H not positive definite) */
#define FM_ERR_TIMEOUT (-5)   /* a device-side wait exceeded fm_opts.spin_limit polls */
#define FM_ERR_NONFINITE (-6) /* a global reduction (cost, dot, step) was not finite */
#define FM_ERR_OOM (-7)       /* device or host allocation failed */
#define FM_ERR_SIZE (-8)      /* problem larger than a fixed-size buffer of the call allows */
#define FM_ERR_FILL (-9)      /* FM_PC_ICT: the drop tolerance keeps fill at more grid offsets
                                 than the factor can hold (see FM_PC_ICT) */

#define FM_FP64 0
#define FM_FP32 1

#define FM_PC_IC0 0  /* IC(0) of H in natural order (Sec. III-B, Eq. 12): the paper's L_0 */
#define FM_PC_DIAG 1 /* diag(H): the paper's NCG-MLS-D comparison (Sec. IV) */
#define FM_PC_NONE 2 /* identity: the paper's NCG-MLS comparison (Sec. IV) */
#define FM_PC_RB 3   /* IC(0) in red-black order (x + y + z even first): a labelled multicolour
                        variant, two parallel stencil passes instead of the wavefronts */
#define FM_PC_ICT 4  /* IC with a drop tolerance (Sec. III-B, the paper's L_t, and its
                        NCG-MLS-IC): natural order, every off-diagonal factor entry (fill-in
                        included) smaller in magnitude than tau = droptol * H_max is set to
                        zero, H_max being the largest |H_jk| of each outer iteration's H.  The
                        factor is held on a set of grid offsets: IC(0)'s plus the level-1 fill
                        offsets (x+1, y-1, z), (x+1, y, z-1), (x, y+1, z-1) at first; a check
                        after every factorisation finds any entry the tolerance keeps outside
                        the set, and the calls that factor (fm_ic_factor, fm_solve,
                        fm_adjoint_solve, fm_batch_solve) then add those offsets and run again
                        from the same start, so the result is the exact drop-tolerance factor
                        (these calls synchronise).  FM_ERR_FILL remains only for a pattern of
                        more than 64 offsets.  The sweeps run level by level (x + B y + C z,
                        B = 2, C = 3 for the initial set), slower than IC(0)'s. */

#define FM_CURV_LITERAL 0  /* d_j summed over every (c, d, m, n) term (Eq. 10) */
#define FM_CURV_COMBINED 1 /* d_j from the coil-combined pair weights (labelled variant) */

#define FM_MAX_ECHO 8
#define FM_MAX_COIL 32

typedef struct fm_ctx fm_ctx; /* opaque, owned by the library */

typedef struct fm_opts {
    int precision;       /* FM_FP32 (default) or FM_FP64 */
    int nls;             /* monotonic line-search steps per outer iteration (N_i), >= 1; default 5 */
    int precond;         /* FM_PC_IC0 (default) | FM_PC_DIAG | FM_PC_NONE | FM_PC_RB | FM_PC_ICT */
    int curvature;       /* FM_CURV_LITERAL (default) | FM_CURV_COMBINED */
    long long spin_limit;/* polls before a device-side wait gives up with FM_ERR_TIMEOUT (a poll
                            is one memory round trip, a barrier check or one bounded hardware
                            wait step, each about a microsecond at most); default 1<<21 (a
                            few seconds at most) */
    int use_graph;       /* 1: replay the outer iteration as a captured CUDA graph (default 1) */
    double droptol;      /* FM_PC_ICT only: tolerance relative to H_max, finite, >= 0; default 1e-3 */
} fm_opts;

/* Fill *opts with the defaults listed above.  opts must not be NULL. */
FM_API void fm_default_opts(fm_opts *opts);

/*
 * Create a context for one nx*ny*nz volume with ncoil coils and necho echoes
 * (Sec. II: N_c >= 1, L >= 2).  opts may be NULL (defaults).  device is a CUDA
 * device ordinal; cuda_stream is a cudaStream_t of that device or NULL for the
 * legacy default stream.  Allocates every device buffer the solver needs (about
 * (8 N_c L + 80) bytes per voxel in FM_FP32 mode).  *out is NULL on failure.
 * Errors: FM_ERR_ARG (sizes < 1, ncoil > FM_MAX_COIL, necho outside 2..FM_MAX_ECHO,
 * bad option), FM_ERR_CUDA, FM_ERR_OOM.
 */
FM_API int fm_create(fm_ctx **out, int nx, int ny, int nz, int ncoil, int necho, const fm_opts *opts,
              int device, void *cuda_stream);

/*
 * Load one acquisition and precompute everything the iterations share (Algorithm
 * box: "precompute r_cdmnj by Eq. 3 and t_m - t_n"; Sec. III-B).
 *   y     device, complex [necho][ncoil][nz][ny][nx] (complex64 in FM_FP32 mode,
 *         complex128 in FM_FP64 mode), the images y_clj of Eq. 1.
 *   smap  device, complex [ncoil][nz][ny][nx] of the same type, the coil maps
 *         s_cj; NULL means s = 1 and requires ncoil == 1 (Sec. II).
 *   te    host double [necho], the echo times t_l (any unit; w is rad per unit).
 *   mask  device uint8 [nz][ny][nx], nonzero = unknown voxel (Sec. IV mask); NULL
 *         means every voxel is an unknown.
 *   beta  the regularisation weight of Eq. 5, >= 0.
 * Also computes the Eq. 6 initial field map used by fm_solve(init_from_data = 1).
 * Errors: FM_ERR_ARG (NULL y, NULL smap with ncoil > 1, beta < 0 or not finite,
 * non-finite te, t_2 == t_1), FM_ERR_CUDA.
 */
FM_API int fm_set_data(fm_ctx *ctx, const void *y, const void *smap, const double *te,
                const uint8_t *mask, double beta);

/*
 * Write the Eq. 6 initial field map to omega (device [nz][ny][nx], float or double by
 * precision).  Requires fm_set_data.
 */
FM_API int fm_init_omega(fm_ctx *ctx, void *omega);

/*
 * Evaluate at the field map omega (device [nz][ny][nx]):
 *   cost  host double*, nullable: Psi(omega) (Eq. 5 with Phi of Eq. 2, literal
 *         constant terms included), accumulated in double;
 *   grad  device [nz][ny][nx], nullable: grad Psi (Eq. 8, with the first power of
 *         t_m - t_n, the derivative of Eq. 2);
 *   curv  device [nz][ny][nx], nullable: d_j of Eq. 10-11 (Huber curvature,
 *         angle wrapped into [-pi, pi]).
 * Outside the mask grad and curv are 0 and omega is ignored.  A non-NULL cost
 * synchronises the stream.  Errors: FM_ERR_STATE before fm_set_data, FM_ERR_ARG.
 */
FM_API int fm_cost_grad(fm_ctx *ctx, const void *omega, double *cost, void *grad, void *curv);

/*
 * Form H = diag(d(omega)) + beta C'C (Eq. 9) and its IC(0) factor (Eq. 12), natural
 * x-fastest order (red-black order when fm_opts.precond is FM_PC_RB), zero fill-in:
 * L = (Pi + E) Pi^{-1/2} with E the strict lower triangle of H in that order and pivots
 * pi_j = H_jj - sum_k E_jk^2 / pi_k.  With FM_PC_ICT it is instead the drop-tolerance
 * factor of FM_PC_ICT (tau = droptol * H_max(omega)), with pi_j = L_jj^2.  The factor
 * is kept in the context for fm_ic_apply.  inv_pivot (device [nz][ny][nx] of the voxel
 * type, nullable) receives 1/pi_j (0 outside the mask).  Pivots are computed in double.
 * Errors: FM_ERR_STATE, FM_ERR_NOT_PD (some pivot <= 0; reported at the next
 * synchronising call), FM_ERR_TIMEOUT, FM_ERR_FILL (FM_PC_ICT only; also reported at
 * the next synchronising call).
 */
FM_API int fm_ic_factor(fm_ctx *ctx, const void *omega, void *inv_pivot);

/*
 * fm_ic_factor from a given curvature instead of the field map: the factor of
 * H = diag(curv) + beta C'C (Eq. 9, 12) with the mask and beta of fm_set_data.  curv: device
 * [nz][ny][nx] of the voxel type (read at mask voxels only).  inv_pivot as for fm_ic_factor.
 * Errors: as fm_ic_factor.
 */
FM_API int fm_ic_factor_curv(fm_ctx *ctx, const void *curv, void *inv_pivot);

/*
 * The drop-tolerance factor (FM_PC_ICT) as the context holds it: *n_offsets receives the
 * number nh of held offsets; offsets (host int [3 nh], nullable) their (dx, dy, dz), each
 * pointing from a voxel to an earlier one in natural order; planes (host double
 * [nh + 1][nz][ny][nx], nullable; requires a factor) plane 0 = 1 / L_ii, plane 1 + h =
 * L_{i, i + offset h} (0 where dropped, outside the grid or outside the mask).  The held
 * pattern starts as IC(0)'s offsets plus the level-1 fill offsets and grows, inside the
 * calls that factor, until the drop tolerance keeps nothing outside it (at most 64 offsets).
 * Synchronises when planes is non-NULL.  Errors: FM_ERR_ARG, FM_ERR_STATE.
 */
FM_API int fm_ict_pattern(fm_ctx *ctx, int *n_offsets, int *offsets, double *planes);

/*
 * fm_ic_factor for the IC(0) preconditioner with the inverse pivots returned in double:
 * inv_pivot (device double [nz][ny][nx]) receives 1/pi_j as the recurrence carries it --
 * IEEE double in FM_FP64 mode; in FM_FP32 mode the sum hi + lo of the float pair the
 * forward sweep keeps (about 46 significant bits; the sweeps themselves apply the float hi).
 * The first FM_FP32 call allocates a float [nz][ny][nx] buffer kept by the context.
 * Errors: as fm_ic_factor; FM_ERR_STATE for another preconditioner.
 */
FM_API int fm_ic_factor64(fm_ctx *ctx, const void *omega, double *inv_pivot);

/*
 * p = (L L')^{-1} g with the factor of the last fm_ic_factor (Sec. III-B, the
 * "precondition" step of the Algorithm box): a forward then a back substitution.
 * g, p: device [nz][ny][nx], distinct.  Errors: FM_ERR_STATE if no factor exists.
 */
FM_API int fm_ic_apply(fm_ctx *ctx, const void *g, void *p);

/*
 * Run niter outer iterations of preconditioned NCG with the monotonic line search
 * (Algorithm box; Eq. 13-16) from omega (device [nz][ny][nx], in/out), or from the
 * Eq. 6 initial map when init_from_data != 0.  Per iteration: g = grad Psi, p =
 * P^{-1} g (IC(0) by default), mu = 0 at i = 0 else (g_i - g_{i-1})'p_i /
 * (g_{i-1}'p_{i-1}), z = -p + mu z, then nls steps alpha <- alpha - f'(alpha) /
 * (sum_j z_j^2 d_j(w + alpha z) + beta ||C z||^2) from alpha = 0, and w <- w + alpha z.
 * cost_hist (host double [niter + 1], nullable) receives Psi(w^0) .. Psi(w^niter);
 * a non-NULL cost_hist synchronises the stream and reports the solve's device errors.
 * Without it the call returns once the solve is enqueued, and its device errors are
 * reported by the next synchronising call (e.g. fm_synchronize).  Errors: FM_ERR_STATE,
 * FM_ERR_ARG (niter < 0), FM_ERR_NOT_PD, FM_ERR_TIMEOUT, FM_ERR_NONFINITE.
 */
FM_API int fm_solve(fm_ctx *ctx, void *omega, int init_from_data, int niter, double *cost_hist);

/* ---------------------------------------------------------------------------------
 * Host-buffer form of the problem statement (Sec. II): images, coil maps and mask in host
 * memory in, field map in host memory out.  The library owns two staging sets of device
 * inputs (allocated by the first fm_set_data_host: about (8 N_c (L + 1) + 1) bytes per
 * voxel each in FM_FP32 mode, twice that in FM_FP64 mode) and copies into them on its own
 * copy stream, so the upload of one acquisition runs while the previous one is solved.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) is needed for that overlap;
 * pageable memory works, but its copies complete before the call returns.
 * ------------------------------------------------------------------------------- */

/*
 * fm_set_data with host arrays: y (host, complex [necho][ncoil][nz][ny][nx] of the image
 * type), smap (host, complex [ncoil][nz][ny][nx] or NULL as for fm_set_data), te (host
 * double [necho]), mask (host uint8 [nz][ny][nx] or NULL), beta.  The copies run on the
 * library's copy stream; the precompute runs on the context's stream after them and after
 * everything enqueued there before (a solve in flight keeps its own data).  Returns once
 * both are enqueued: y, smap and mask must stay unchanged until the next synchronising call
 * on ctx.  Errors: as fm_set_data, and FM_ERR_OOM / FM_ERR_CUDA for the staging buffers.
 */
FM_API int fm_set_data_host(fm_ctx *ctx, const void *y, const void *smap, const double *te,
                            const uint8_t *mask, double beta);

/*
 * fm_solve with a host field map: omega (host [nz][ny][nx] of the voxel type) is read as
 * the start point when init_from_data == 0 and receives the result.  Enqueued on the
 * context's stream (the result is in omega after the next synchronising call, e.g.
 * fm_synchronize, or at return when cost_hist is non-NULL).  Errors: as fm_solve.
 */
FM_API int fm_solve_host(fm_ctx *ctx, void *omega, int init_from_data, int niter, double *cost_hist);

/* Wait for all work of ctx (its stream and its copy stream) and report device errors of
 * earlier asynchronous calls.  Errors: FM_ERR_CUDA and the device-side codes. */
FM_API int fm_synchronize(fm_ctx *ctx);

/*
 * Copy the step sizes alpha^(N_i) and Polak-Ribiere factors mu of the last fm_solve
 * (host double [n] each, nullable; n <= that solve's niter).  Synchronises.
 */
FM_API int fm_get_history(fm_ctx *ctx, double *alpha_hist, double *mu_hist, int n);

/* ---------------------------------------------------------------------------------
 * Water-fat model (Sec. II: x_l = m_w + m_f sum_p a_p e^{i 2 pi f_p t_l}; Eq. gamma).
 * ------------------------------------------------------------------------------- */

/*
 * Select the water-fat model for the next fm_set_data: npeak fat peaks with relative
 * amplitudes rel_amp (host double [npeak]; the paper's sum to 1) and frequency offsets
 * freq (host double [npeak], cycles per unit of the echo times: kHz when te is in ms).
 * fm_set_data then uses Gamma = gamma (gamma^H gamma)^{-1} gamma^H with gamma = [1, phi],
 * phi_l = sum_p rel_amp_p e^{i 2 pi freq_p t_l}, in Eq. 3 instead of 1/L; cost, gradient,
 * curvature, IC(0) and the solver are unchanged in form.  npeak = 0 restores the
 * field-map model.  Invalidates the loaded data: call fm_set_data again.
 * Errors: FM_ERR_ARG (npeak outside 0..64, NULL arrays, non-finite values); fm_set_data
 * returns FM_ERR_ARG if phi is collinear with the ones vector at the echo times.
 */
FM_API int fm_set_fat_model(fm_ctx *ctx, int npeak, const double *rel_amp, const double *freq);

/*
 * Voxel-wise initialisation of the water-fat case (Sec. III-A): for every mask voxel,
 * Phi_j (Eq. 2) at nsweep equally spaced values w_lo + (w_hi - w_lo) q / (nsweep - 1),
 * q = 0 .. nsweep - 1; the first value with the smallest cost goes to omega_tilde (device
 * [nz][ny][nx], voxel type; 0 outside the mask).  The paper sweeps 100 values over
 * [-|Delta_f / 2|, |Delta_f / 2|] (in rad per unit of te: pi |f| for a peak at f).
 * Errors: FM_ERR_ARG (nsweep < 1, non-finite bounds), FM_ERR_STATE.
 */
FM_API int fm_wf_sweep(fm_ctx *ctx, int nsweep, double w_lo, double w_hi, void *omega_tilde);

/*
 * The paper's sweep range for fm_wf_sweep under the current fat model (Sec. III-A:
 * [-|Delta_f / 2|, |Delta_f / 2|]), with Delta_f read as the frequency of the fat peak of
 * largest relative amplitude (the first such peak on a tie): *w_lo = -pi |f|, *w_hi = pi |f|
 * in rad per unit of te.  Errors: FM_ERR_ARG (NULL pointers), FM_ERR_STATE (no fat model).
 */
FM_API int fm_wf_sweep_range(const fm_ctx *ctx, double *w_lo, double *w_hi);

/*
 * PWLS initialisation (Eq. w0_wf): niter conjugate-gradient iterations (no preconditioner;
 * the paper uses 10) on (2 diag(rho) + beta C'C) w = 2 rho omega_tilde, starting from
 * omega_tilde, with rho_j = sum_{c,d,m,n} |r_cdmnj| from fm_set_data.  omega_tilde, omega0:
 * device [nz][ny][nx] of the voxel type (may alias).  Dot products in double.
 * Overwrites the solver's work buffers (and drops an fm_ic_factor result).  Synchronises.
 * Errors: FM_ERR_ARG, FM_ERR_STATE, FM_ERR_NOT_PD, FM_ERR_NONFINITE.
 */
FM_API int fm_pwls_init(fm_ctx *ctx, const void *omega_tilde, int niter, void *omega0);

/*
 * Water and fat components at the field map omega by the closed form of Eq. wf:
 * [m_w, m_f]_j = ((gamma diag(e^{i w_j t})) kron s_j)^+ y_j.  y and smap are the arrays
 * given to fm_set_data (smap NULL only with one coil); water and fat: device complex
 * [nz][ny][nx] of the image type (0 outside the mask and where sum_c |s_c|^2 = 0).
 * Errors: FM_ERR_ARG, FM_ERR_STATE (no fat model, or fm_set_data missing).
 */
FM_API int fm_wf_amplitudes(fm_ctx *ctx, const void *y, const void *smap, const void *omega, void *water,
                            void *fat);

/* ---------------------------------------------------------------------------------
 * Differentiation of the converged field map.  The paper has no counterpart; these
 * calls rest on its first-order condition at the solution, grad Psi(w^) = 0 (Eq. 5, 8).
 * Differentiating that identity gives, for a scalar loss l(w^) with b = dl/dw^,
 *     lambda = H_true^{-1} b,          H_true = diag(h(w^)) + beta C'C,
 *     dl/dbeta = -lambda' C'C w^,      dl/dy = -(d grad Phi / dy)' lambda,
 * where h is the exact second derivative of Phi (below), not the Huber majoriser d of
 * Eq. 10-11.  The gradient with respect to w of Psi itself is fm_cost_grad's grad.
 * ------------------------------------------------------------------------------- */

/*
 * h_j = d^2 Phi_j / dw_j^2 = sum_{c,d,m,n} |r| (t_m - t_n)^2 cos(angle r + w_j (t_m - t_n))
 * (the derivative of Eq. 8) at omega, into h (device [nz][ny][nx], voxel type; 0 outside
 * the mask).  h can be negative where a phase residual exceeds pi/2.
 * Errors: FM_ERR_ARG, FM_ERR_STATE before fm_set_data.
 */
FM_API int fm_true_curv(fm_ctx *ctx, const void *omega, void *h);

/*
 * Solve H_true lambda = rhs on the mask voxels by conjugate gradients preconditioned with
 * the IC(0) factor of the majoriser H(omega_hat) = diag(d) + beta C'C (Eq. 9, 12), the
 * factor the solver uses.  omega_hat, rhs, lambda: device [nz][ny][nx] of the voxel type
 * (rhs outside the mask is ignored; lambda is 0 there).  Stops when ||r|| <= tol ||rhs||
 * (the recursively updated residual; dot products in double) or after maxiter iterations;
 * iters and relres (host, nullable) receive the count and ||r|| / ||rhs||.  Reaching
 * maxiter is not an error: check relres.  Leaves the preconditioner factor of omega_hat in
 * the context (as fm_ic_factor would) and overwrites the solver's work buffers.
 * Synchronises.  Errors: FM_ERR_ARG (tol < 0, maxiter < 0), FM_ERR_STATE, FM_ERR_NOT_PD
 * (p' H_true p <= 0: omega_hat is not a strict local minimum), FM_ERR_NONFINITE,
 * FM_ERR_TIMEOUT.
 */
FM_API int fm_adjoint_solve(fm_ctx *ctx, const void *omega_hat, const void *rhs, void *lambda, double tol,
                            int maxiter, int *iters, double *relres);

/*
 * Given lambda from fm_adjoint_solve, the derivatives of the loss through the solution:
 *   dl_dy    device complex [necho][ncoil][nz][ny][nx] (nullable; the image type): the
 *            real-pair gradient d l / d Re y + i d l / d Im y, 0 outside the mask;
 *   dl_dbeta host double (nullable; synchronises): -lambda' C'C omega_hat.
 * y and smap must be the arrays given to fm_set_data (smap NULL only with one coil).
 * Errors: FM_ERR_ARG, FM_ERR_STATE (also: dl_dy under the water-fat model, not
 * implemented).
 */
FM_API int fm_implicit_grad(fm_ctx *ctx, const void *y, const void *smap, const void *omega_hat,
                            const void *lambda, void *dl_dy, double *dl_dbeta);

/* ---------------------------------------------------------------------------------
 * Batched form: many independent volumes (possibly of different sizes and coil counts)
 * solved together.  Each volume is its own context (same options) on its own stream;
 * fm_batch_solve captures one outer iteration of every volume as parallel branches of a
 * single CUDA graph (the two-iteration ping-pong body, as in fm_solve) and replays it, so
 * one graph launch advances all volumes and their kernels fill the GPU together.  The
 * per-volume arithmetic is exactly fm_solve's.
 * ------------------------------------------------------------------------------- */
typedef struct fm_batch fm_batch;

/* Create a batch of n volumes; dims is a host int array [n][5] of (nx, ny, nz, ncoil,
 * necho).  opts as for fm_create (shared by every volume).  cuda_stream: the stream the
 * batch orders itself after and completes on (NULL: legacy default stream).
 * Errors: FM_ERR_ARG (n < 1, bad sizes or options), FM_ERR_CUDA, FM_ERR_OOM. */
FM_API int fm_batch_create(fm_batch **out, int n, const int *dims, const fm_opts *opts, int device,
                           void *cuda_stream);

/* fm_set_data for volume k (same argument rules).  Errors: FM_ERR_ARG (k out of range). */
FM_API int fm_batch_set_data(fm_batch *b, int k, const void *y, const void *smap, const double *te,
                             const uint8_t *mask, double beta);

/* fm_solve on every volume: omega is a host array of n device pointers (in/out, each of its
 * volume's size and voxel type); cost_hist is a host array of n host pointers (each
 * [niter + 1] doubles) or NULL.  Synchronises.  Errors: as fm_solve; the first failing
 * volume's status is returned. */
FM_API int fm_batch_solve(fm_batch *b, void *const *omega, int init_from_data, int niter,
                          double *const *cost_hist);

/* Choose, by timing short solves of niter_probe iterations, the launch schedule of the
 * volumes running side by side: the fraction of its own full-GPU grid each volume's kernels
 * use (candidates 1, 1/2, 1/4, 1/8), the order in which the IC(0) forward wavefront claims
 * its tiles (weights (X + Y) : Z of 2 : 1, 1 : 1, 3 : 2; any positive weights keep the
 * dependency order), and then, at the best of those, the back-substitution wavefront's blocks
 * per SM (1, 2 or 3, as its occupancy allows).  best_ms (host, nullable) receives the winning
 * probe time.  Requires fm_batch_set_data on every volume.  The schedule stays in effect
 * until changed (fm_batch_schedule and fm_batch_bwd_blocks report it). */
FM_API int fm_batch_autotune(fm_batch *b, int niter_probe, double *best_fraction, double *best_ms);

/* Set the grid fraction directly (0 < fraction <= 1). */
FM_API int fm_batch_set_fraction(fm_batch *b, double fraction);

/* The schedule in effect: grid fraction and the forward tile order weights (host, nullable). */
FM_API int fm_batch_schedule(const fm_batch *b, double *fraction, int *order_wxy, int *order_wz);

/* The back-substitution wavefront's blocks per SM in effect (before the grid fraction). */
FM_API int fm_batch_bwd_blocks(const fm_batch *b, int *blocks_per_sm);

/* Context of volume k (for fm_cost_grad, fm_get_history, ...; owned by the batch). */
FM_API fm_ctx *fm_batch_ctx(fm_batch *b, int k);

/* Release the batch and its contexts.  NULL-safe. */
FM_API int fm_batch_destroy(fm_batch *b);

/*
 * Change the bound on device-side waits (fm_opts.spin_limit) of an existing context, >= 1.
 * A wait that exceeds it gives up with FM_ERR_TIMEOUT; the context stays usable and the
 * next call starts from a clean barrier state.  Errors: FM_ERR_ARG.
 */
FM_API int fm_set_spin_limit(fm_ctx *ctx, long long spin_limit);

/* Kernel classes timed by fm_kernel_times. */
#define FM_K_GRAD 0   /* data term + stencil gradient pass (fused update of the previous step) */
#define FM_K_IC_FWD 1 /* IC(0) pivots + forward substitution wavefront */
#define FM_K_IC_BWD 2 /* back substitution wavefront + g'p, g_prev'p */
#define FM_K_DIR 3    /* (no longer launched on its own: the direction is FM_K_LS's first phase) */
#define FM_K_LS 4     /* persistent kernel: Polak-Ribiere direction, then the line search */
#define FM_K_H2D 5    /* fm_set_data_host: host-to-device copy of one acquisition's inputs */
#define FM_K_D2H 6    /* fm_solve_host: device-to-host copy of the field map */
#define FM_NKERNEL 7

/*
 * Turn per-kernel timing on or off (off by default).  While on, fm_solve brackets
 * every kernel of the outer iteration with CUDA events on the context's stream (they
 * are part of the captured graph), which adds a few microseconds per iteration.
 */
FM_API int fm_set_profiling(fm_ctx *ctx, int on);

/*
 * Average device duration in milliseconds of each kernel class over the most recent
 * profiled outer iterations (the last graph replay, or the last iteration without a
 * graph): avg_ms and count are host arrays of FM_NKERNEL entries (count: launches
 * averaged, 0 if that class did not run).  Synchronises.
 */
FM_API int fm_kernel_times(fm_ctx *ctx, double *avg_ms, int *count);

/*
 * fm_cost_grad without a context and without allocating any device memory.  The paper
 * has no counterpart: this is a deployment convenience for callers that cannot call
 * cudaMalloc -- for example code that runs while another component captures a CUDA
 * graph on the device, real-time pipelines that must not allocate after start-up, or
 * plug-ins whose host runtime owns every device buffer and only passes pointers in.
 *
 * It evaluates, at omega, the same cost, gradient and curvature as fm_cost_grad, directly
 * from the raw inputs (same layouts and types as fm_set_data / fm_cost_grad; opts
 * supplies precision and curvature, NULL = defaults; beta >= 0).  cost (host) receives
 * Psi(omega) and synchronises the stream when non-NULL; grad and curv (device) are
 * nullable.  cuda_stream: a stream of `device`, or NULL for the legacy default stream.
 *
 * Scratch: the per-block FP64 partial costs live in one fixed array of about 128 KB
 * inside the library (a file-scope __device__ variable), which every GPU that loads the
 * library keeps until the process exits.  Limit: nx*ny*nz <= 67,108,864 voxels
 * (16,384 blocks of 4,096 voxels); larger volumes return FM_ERR_SIZE before any device
 * work.  The first call on a device looks up that array's device address (once per
 * device); make that first call before any stream capture.  The address is kept for the
 * life of the process, so cudaDeviceReset between calls is not supported (the array may
 * move when the library's module is loaded again).  Every call reuses the same array and
 * clears its counter at the start, so calls whose kernels overlap on the GPU (different
 * streams or threads without ordering) race and must not be issued.
 * Errors: FM_ERR_ARG, FM_ERR_SIZE, FM_ERR_CUDA, FM_ERR_NONFINITE (cost requested and not
 * finite, as fm_cost_grad reports a non-finite value inside the mask; the outputs are
 * still written).
 */
FM_API int fm_cost_grad_noalloc(int nx, int ny, int nz, int ncoil, int necho, const fm_opts *opts,
                                const void *y, const void *smap, const double *te, const uint8_t *mask,
                                double beta, const void *omega, double *cost, void *grad, void *curv,
                                int device, void *cuda_stream);

/* Release every resource of ctx.  NULL-safe.  Returns FM_OK. */
FM_API int fm_destroy(fm_ctx *ctx);

/* Static description of a status code. */
FM_API const char *fm_strerror(int status);

/* Description of the last error on ctx ("" if none); valid until the next call on ctx. */
FM_API const char *fm_last_error(const fm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FM_H */
