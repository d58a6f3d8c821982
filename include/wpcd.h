/*
 * wpcd.h -- C ABI of libwpcd, a GB300 (sm_103a) implementation of the
 * wave-packet continuum discretisation (WPCD) of the nucleon-nucleon
 * Lippmann-Schwinger equation (Miller, Ekstrom, Forssen, arXiv:2106.00454).
 *
 * Per partial-wave channel and parameter sample the library
 *   (a) projects the momentum-space potential onto free wave packets (FWP),
 *   (b) forms H = H0 + V (N_WP x N_WP uncoupled, 2N_WP x 2N_WP coupled) and
 *       diagonalises it,
 *   (c) evaluates the on-shell T-matrix at every requested energy through the
 *       energy-averaged resolvent of the scattering wave packets (SWP), and
 *   (d) turns T into phase shifts and the np total cross section.
 *
 * Conventions (all calls):
 *   - Every call returns a wpcd_status; nothing throws across the ABI.
 *   - Pointers named *_dev are device pointers owned by the caller and must
 *     stay valid until the work queued on the context stream has finished.
 *     Pointers named *_host are host pointers, read or written before the call
 *     returns (the *_host entry points synchronise the stream).
 *   - Handles (mesh, vset, eig ids) are owned by the context and live until
 *     wpcd_release or wpcd_destroy.
 *   - Work is queued on the context's CUDA stream; a call returns after
 *     queueing unless stated otherwise.  Errors that only the device can see
 *     (an energy outside the mesh, a solve that did not converge) are recorded
 *     in a device status word and returned by the next wpcd_sync.
 *   - Units: momenta fm^-1, lab energies MeV, T-matrix fm^2 (partial-wave
 *     normalisation <k'|k> = delta(k'-k)/(k'k), Sec. 2), angles in degrees,
 *     cross sections in mb.
 *   - Kinematics: p^2 = m_N T_lab / 2 with m_N = 938.918309 MeV and
 *     hbar c = 197.3269804 MeV fm (nonrelativistic; the paper leaves this open).
 */
#ifndef WPCD_H
#define WPCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wpcd_ctx wpcd_ctx; /* opaque; owns all device-resident state */

typedef enum {
    WPCD_OK = 0,
    WPCD_ERR_ARG = -1,        /* bad argument (null pointer, size out of range, energy outside the mesh) */
    WPCD_ERR_NOMEM = -2,      /* device or host allocation failed */
    WPCD_ERR_BUDGET = -3,     /* the request would exceed the context's HBM budget */
    WPCD_ERR_NOCONVERGE = -4, /* an eigensolve hit its sweep cap (per-solve status says which) */
    WPCD_ERR_TIMEOUT = -5,    /* a bounded wait ran out */
    WPCD_ERR_CUDA = -6,       /* a CUDA runtime call failed */
    WPCD_ERR_NOTREADY = -7,   /* serving: the ticket is still in flight */
    WPCD_ERR_HANDLE = -8      /* unknown or released handle / ticket */
} wpcd_status;

/* Arithmetic of the eigensolve.  FP64: H assembled and diagonalised in FP64
 * (parallel Jacobi).  MIXED: H diagonalised in FP32 (the same Jacobi with a
 * relative rotation threshold), then two FP64 refinement iterations of the
 * eigenpairs (Ogita-Aishima: Y = HX, S = X^T Y, G = X^T X, X <- X(I + E)) as
 * batched FP64 products; everything after the eigensolve (resolvent logs, T,
 * S, phases) is FP64 on both paths. */
typedef enum { WPCD_PREC_FP64 = 0, WPCD_PREC_MIXED = 1 } wpcd_precision;

/* Resolvent used for the on-shell T (App. B).
 * FREE_BIN: the SWP resolvent averaged over the free bin that holds the
 *   on-shell energy (the averaging of Sec. 3.2, "resolvent energy averaging";
 *   App. B closed form with the sign of W corrected).  T per free bin,
 *   converted at the bin midpoint; phases interpolated between midpoints.
 * SWP_INDEX: the App. B formula as printed, averaging over SWP bin i of the
 *   channel's single branch instead of free bin i.  Defined for uncoupled
 *   channels without bound states: a vset with a coupled channel is refused
 *   (WPCD_ERR_ARG); a solve that has a bound state gets NaN outputs and
 *   wpcd_sync reports WPCD_ERR_ARG.
 * POINT: no averaging; the point resolvent of App. B,
 *   g_s(E) = [ln|(E - B_s)/(E - B_s+1)| - i pi 1{E in [B_s, B_s+1]}] / dB_s
 *   (1/(E - e_b) for a bound state), evaluated at each requested energy, with
 *   the continuum conversion, S and the phases at p(E) itself (no
 *   interpolation).  An energy exactly on an SWP boundary gives a non-finite T. */
typedef enum { WPCD_AVG_FREE_BIN = 0, WPCD_AVG_SWP_INDEX = 1, WPCD_POINT = 2 } wpcd_resolvent;

/* Partial-wave channel.  Uncoupled: l = lp.  Coupled (K = 2): l = J-1,
 * lp = J+1 and the channel is the 2x2 block pair on degenerate FWP copies
 * (Sec. 3.1).  tz = 0 is np; only tz = 0 channels enter the np cross section. */
typedef struct { int s, J, l, lp, coupled, tz; } wpcd_channel;

/* Potential generators for wpcd_project. */
enum {
    WPCD_GEN_FINE = -1,     /* caller-supplied fine-grid values (v_fine_dev) */
    WPCD_GEN_YAMAGUCHI = 0, /* params {lambda (fm^2), beta (fm^-1)}: V = lambda g(p')g(p), g = 1/(p^2+beta^2); 1 term */
    WPCD_GEN_YUKAWA = 1     /* 19 params (masses m1..m3, regulator Lambda, 14 V0 strengths, 1S0 tz!=0 contact); 15 terms */
};

/* Options (wpcd_set_option).  WPCD_OPT_EXEC: one launch per size bucket
 * (BATCHED) or one launch per (sample, channel) solve (PLAIN, the baseline
 * execution).  WPCD_OPT_REFINE: engine of the mixed path's FP64 refinement
 * products -- TENSOR (BF16 tensor cores with Ozaki splitting, FP64-accurate) or
 * FP64 (FP64 CUDA cores).  WPCD_OPT_AUTOTUNE (1 = on, the default): on the first
 * batched eigensolve of each (matrix size, precision) the context times CTA
 * sizes 64/128/256/512 (and 1024 for the FP32 kernel) on about two full waves
 * of that bucket and keeps the
 * fastest (wpcd_tuning reports the choices); 0 = fixed 256 threads.
 * WPCD_OPT_GRAPH (1 = on, the default): batched wpcd_solve / wpcd_solve_host
 * calls are replayed from CUDA graphs (see wpcd_solve); 0 = every call
 * launches its kernels one by one.  WPCD_OPT_BIG_SLOTS: CTAs (each with its
 * own scratch copy of the matrix and eigenvectors) of the global-memory
 * eigensolver used above the shared-memory size; 0 (the default) = every
 * CTA that can be resident at once.  WPCD_OPT_ROTATE (1 = on, the default;
 * mixed path with the tensor refinement engine): the FP32 eigensolve starts
 * from C0^T H C0, C0 the FP64 eigenvectors of the projected set's diag(H0) + V0
 * (built once per set, on its first mixed solve), which is nearly diagonal for
 * samples near the mean and takes fewer Jacobi sweeps; the refined
 * eigenvectors are rotated back with FP64-accurate products.  0 = the FP32
 * eigensolve starts from H itself.  WPCD_OPT_REFINE_ITERS (1..4, default 2):
 * FP64 refinement iterations of the mixed path; each squares the eigenvector
 * error.  Measured on the 16384-sample N_WP = 150 workload against the FP64
 * path: two iterations leave phase errors below 1e-6 deg and cross-section
 * errors near 1e-6 mb; one iteration leaves phase errors up to ~6e-4 deg but
 * cross-section errors up to ~0.02 mb, outside the 0.01 mb bar, so it is only
 * an opt-in for callers that need the phases alone.  WPCD_OPT_REFINE_DIGITS
 * (4..6, default 6; tensor refinement engine): balanced 8-bit digits per operand
 * of the refinement's digit products -- 6 gives FP64-accurate products (21 digit
 * pairs), 5 and 4 about 39 and 31 bits (15 and 10 pairs), trading the refined
 * accuracy for product time. */
enum { WPCD_EXEC_BATCHED = 0, WPCD_EXEC_PLAIN = 1 };
enum { WPCD_REFINE_TENSOR = 0, WPCD_REFINE_FP64 = 1 };
enum { WPCD_OPT_EXEC = 1, WPCD_OPT_REFINE = 2, WPCD_OPT_AUTOTUNE = 3, WPCD_OPT_GRAPH = 4, WPCD_OPT_BIG_SLOTS = 5,
       WPCD_OPT_ROTATE = 6, WPCD_OPT_REFINE_ITERS = 7, WPCD_OPT_REFINE_DIGITS = 8 };

/* ---- context --------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = no cap).  cuda_stream: a cudaStream_t on
 * that device (NULL = the legacy default stream); the context does not own it.
 * Errors: WPCD_ERR_ARG (null out pointer, bad device), WPCD_ERR_CUDA. */
wpcd_status wpcd_create(wpcd_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Wait for the stream, free every handle and the context.  NULL is ignored. */
void wpcd_destroy(wpcd_ctx *ctx);

/* Static, human-readable text for a status code. */
const char *wpcd_strerror(wpcd_status st);

/* Interpolation point (Sec. 5.1.1, Eq. "interpolation point"): the point
 * q_i = k_i + frac (k_{i+1} - k_i) of each free bin at which the averaged
 * resolvents' T is converted to the continuum (wpcd_tmatrix) and the bin's
 * phase shift is placed for the linear interpolation (wpcd_observables);
 * frac = n/m of the paper, 0 < frac < 1, default 0.5 (the bin midpoint).
 * Applies to calls queued afterwards (served batches included); the point
 * resolvent ignores it.  Errors: WPCD_ERR_ARG (frac outside (0, 1)). */
wpcd_status wpcd_set_interp_point(wpcd_ctx *ctx, double frac);

/* Set an execution option (see WPCD_OPT_*).  Errors: WPCD_ERR_ARG. */
wpcd_status wpcd_set_option(wpcd_ctx *ctx, int key, int value);

/* Synchronise the context stream and return (then clear) the first error
 * recorded by device code since the last wpcd_sync, else WPCD_OK. */
wpcd_status wpcd_sync(wpcd_ctx *ctx);

/* Device bytes currently held by the context. */
size_t wpcd_bytes_in_use(const wpcd_ctx *ctx);

/* ---- (a0) free-wave-packet mesh: Sec. 3.2 step 1 ------------------------------------------------
 * Builds N+1 momentum boundaries k_0 = 0 < ... < k_N and n_quad Gauss-Legendre
 * points per bin on the device.  kind 0: tan^t map on a uniform angle grid that
 * ends at kmax_fm (k_j = alpha tan^t(j theta_max / N), theta_max =
 * atan((kmax/alpha)^(1/t))); kind 1: the paper's Chebyshev distribution
 * k_j = alpha tan^t((2j-1) pi / (4N)), k_0 = 0 (kmax ignored).
 * wp_kind 0: momentum packets f(k) = 1, N_i = dk_i; 1: energy packets
 * f(k) = sqrt(k/mu), N_i = dE_i (Sec. 3.1, definition of the free wave packet).
 * Constraints: 4 <= n_wp <= 512, 1 <= n_quad <= 16, alpha, t > 0.
 * Errors: WPCD_ERR_ARG, WPCD_ERR_NOMEM, WPCD_ERR_BUDGET, WPCD_ERR_CUDA. */
wpcd_status wpcd_mesh(wpcd_ctx *ctx, int n_wp, int kind, double alpha_fm, double t, double kmax_fm,
                      int n_quad, int wp_kind, int *mesh_id);

/* Copy a mesh to the host (synchronises): kb_host[n_wp+1], kq_host/wq_host[n_wp*n_quad]
 * (any of them may be NULL).  Errors: WPCD_ERR_HANDLE. */
wpcd_status wpcd_mesh_get(wpcd_ctx *ctx, int mesh_id, double *kb_host, double *kq_host, double *wq_host);

/* ---- (a1) projection of the potential terms: Sec. 3.2, Eq. "WP potential matrix identity" ------
 *   V_ij = (N_i N_j)^-1/2 int_{D_i} int_{D_j} k'k dk'dk f(k') f(k) v(k', k)
 * for every term t of the potential (t = 0 is V0, t >= 1 the terms that the
 * per-sample coefficients multiply), evaluated with the mesh's fine rule.
 * The partial-wave projection of a built-in generator uses a 96-point
 * Gauss-Legendre rule in the scattering angle.  Each channel c has its own
 * mesh (mesh_ids[c]); its matrix is n x n, n = K N_WP, l-blocks ordered
 * (l = J-1, l = J+1) for coupled channels.  Result: a vset handle holding
 * the FP64 matrices [term][n][n] per channel, resident on the device.
 * gen_params_host: the generator's parameters (see WPCD_GEN_*).
 * v_fine_dev (WPCD_GEN_FINE only): per channel c, term t, the fine-grid values
 * v(k_a, k_b) as a [K*NQ][K*NQ] row-major FP64 block (NQ = n_wp*n_quad),
 * channels one after another, terms inner: offset(c, t) = sum_{c'<c}
 * n_terms (K' NQ')^2 + t (K NQ)^2.  Read during the call's device work.
 * Errors: WPCD_ERR_ARG (n_ch < 1, unknown generator, n_terms out of range
 * 1..16, a generator that does not define the channel), WPCD_ERR_HANDLE,
 * WPCD_ERR_NOMEM, WPCD_ERR_BUDGET, WPCD_ERR_CUDA. */
wpcd_status wpcd_project(wpcd_ctx *ctx, const int *mesh_ids, const wpcd_channel *channels, int n_ch,
                         int generator_id, const double *gen_params_host, int n_gen_params,
                         const double *v_fine_dev, int n_terms, int *vset_id);

/* wpcd_project with a precision for the built-in Yukawa + contact generator
 * (the other generators ignore it): WPCD_PREC_FP64 is wpcd_project;
 * WPCD_PREC_MIXED forms the 96-point angle integrals I_L[m](k_a, k_b) of every
 * fine pair as a contraction on the tensor cores: the angle integrand is
 * evaluated in FP32, every row of it and every column of the w_x P_L(x) table
 * scaled by a power of two and cut into four balanced 8-bit digits (exact in
 * BF16), and the ten digit pairs of weight <= 3 accumulated in FP32 as exact
 * integers; the potential terms and the bin reduction follow in FP64 as for
 * wpcd_project.  The projected terms then differ from the FP64 ones by a few
 * 1e-6 of each term's largest element (the FP32 integrand), which keeps the
 * mixed path within 1e-3 deg and 0.01 mb of the FP64 oracle.  Errors as
 * wpcd_project; a device timeout of the tensor-core contraction is reported
 * by wpcd_sync. */
wpcd_status wpcd_project_prec(wpcd_ctx *ctx, const int *mesh_ids, const wpcd_channel *channels, int n_ch,
                              int generator_id, const double *gen_params_host, int n_gen_params,
                              const double *v_fine_dev, int n_terms, wpcd_precision prec, int *vset_id);

/* Copy the projected matrices of one channel to the host (synchronises):
 * out_host[n_terms][n][n].  Errors: WPCD_ERR_HANDLE, WPCD_ERR_ARG. */
wpcd_status wpcd_vset_get(wpcd_ctx *ctx, int vset_id, int channel, double *out_host);

/* ---- (a2, a3) parameter sum and eigendecomposition: Sec. 3.2 step 2, Eq. "eigendecomposition
 * Hamiltonian" -----------------------------------------------------------------------------------
 * For every sample s and channel c: H = diag(H0) + V0 + sum_{a>=1} c[s][a-1] V_a
 * (H0_ii = <x_i|h0|x_i> exactly, repeated on both l-blocks of a coupled
 * channel), then H = C D C^T with eigenvalues ascending.  coeffs_dev:
 * [n_samples][n_terms-1] FP64 (may be NULL when n_terms == 1).  The eigenpairs
 * stay on the device under the returned eig handle.  prec: WPCD_PREC_FP64 or
 * WPCD_PREC_MIXED (see wpcd_precision).  Every size uses the parallel cyclic
 * Jacobi method (App. C): matrices that fit one CTA's shared memory (FP64 up to
 * n ~ 230, FP32 up to n = 304) are held there; larger ones, up to n = 1024, are
 * held in global memory (L2-resident while a CTA works on them).
 * Per-solve convergence status: wpcd_diag_status.
 * Errors: WPCD_ERR_ARG, WPCD_ERR_HANDLE, WPCD_ERR_NOMEM, WPCD_ERR_BUDGET, WPCD_ERR_CUDA. */
wpcd_status wpcd_diag(wpcd_ctx *ctx, int vset_id, const double *coeffs_dev, int n_samples,
                      wpcd_precision prec, int *eig_id);

/* Per-solve status into status_dev[n_samples][n_ch] (int32): the number of
 * Jacobi sweeps taken, or -1 if the sweep cap was hit.  Queued on the stream. */
wpcd_status wpcd_diag_status(wpcd_ctx *ctx, int eig_id, int *status_dev);

/* Copy the eigenpairs of one solve to the host (synchronises):
 * eps_host[n], C_host[n][n] row-major (column s = eigenvector s). */
wpcd_status wpcd_eig_get(wpcd_ctx *ctx, int eig_id, int sample, int channel, double *eps_host, double *C_host);

/* ---- (a4-a7) on-shell T: Sec. 3.2 steps 3-5, App. B -----------------------------------------------
 * For every sample, channel and requested energy: the SWP boundaries of
 * Eq. "pseudostate wave packet boundaries", the resolvent of App. B chosen by
 * res (default: averaged over the free bin D_i holding p(E)), and
 *   T_ab(i) = V_(a,i),(b,i) + sum_s (VC)_(a,i),s gbar_s (VC)_(b,i),s,
 * converted to the continuum at q = the bin midpoint (Eq. "operator in cont and
 * disc representation").  e_lab_dev: [n_E] MeV, ascending, each inside the
 * channel meshes.  t_out_dev: complex128 (re, im interleaved)
 * [n_samples][n_ch][n_E][2][2] fm^2 (uncoupled channels fill [0][0], zeros
 * elsewhere).  Errors: WPCD_ERR_ARG, WPCD_ERR_HANDLE, WPCD_ERR_NOMEM, WPCD_ERR_CUDA;
 * an energy outside a mesh is reported by wpcd_sync as WPCD_ERR_ARG. */
wpcd_status wpcd_tmatrix(wpcd_ctx *ctx, int eig_id, const double *e_lab_dev, int n_E, wpcd_resolvent res,
                         double *t_out_dev);

/* ---- (a7, a8) phase shifts and total cross section: App. A, Sec. 5.1.1 ------------------------------
 * Phase shifts at the bin midpoints (S = 1 - 2 pi i mu p T; Stapp for coupled
 * channels), interpolated linearly in p between consecutive midpoints to each
 * requested energy (Eq. "linear interpolation"), and the np total cross section
 * sigma = pi/(2p^2) sum_ch (2J+1) sum_l Re(1 - S_ll) from the interpolated
 * parameters.  delta_dev: [n_samples][n_ch][n_E][3] degrees (delta or delta_-,
 * delta_+, eps_J; zeros where undefined); sigma_dev: [n_samples][n_E] mb.
 * Either output may be NULL.  Errors as wpcd_tmatrix. */
wpcd_status wpcd_observables(wpcd_ctx *ctx, int eig_id, const double *e_lab_dev, int n_E, double *delta_dev,
                             double *sigma_dev);

/* wpcd_observables with another resolvent (wpcd_observables uses FREE_BIN).
 * POINT gives the phases at each p(E) directly, without interpolation. */
wpcd_status wpcd_observables_res(wpcd_ctx *ctx, int eig_id, const double *e_lab_dev, int n_E, wpcd_resolvent res,
                                 double *delta_dev, double *sigma_dev);

/* ---- the whole hot path in one call --------------------------------------------------------------
 * wpcd_diag + wpcd_tmatrix + wpcd_observables for one batch, with the
 * eigenpairs kept in context scratch instead of a handle.  Outputs may be NULL.
 * CUDA graphs (WPCD_OPT_GRAPH on, batched execution, profiling off): the first
 * call with a given (vset, pointers, sizes, precision, resolvent) launches its
 * kernels one by one (and autotunes and sizes the workspaces); the second
 * captures the same launch sequence into a graph on a private stream; that and
 * every later identical call launch the graph on the context stream.  A graph
 * is dropped when anything it baked in may have changed (a workspace grew or
 * was reallocated, an option or the tuning table changed); the next identical
 * call then runs one by one again.  Results are the same either way: the graph
 * holds the same kernels with the same arguments. */
wpcd_status wpcd_solve(wpcd_ctx *ctx, int vset_id, const double *coeffs_dev, int n_samples,
                       const double *e_lab_dev, int n_E, wpcd_precision prec, wpcd_resolvent res,
                       double *t_out_dev, double *delta_dev, double *sigma_dev);

/* Same as wpcd_solve with every buffer on the host: inputs are copied to the
 * device and outputs back inside the call, which synchronises and returns the
 * device status as wpcd_sync would.  The copies go straight from and into the
 * caller's buffers; page-locked (pinned) buffers move at the link's full rate,
 * pageable ones are accepted too. */
wpcd_status wpcd_solve_host(wpcd_ctx *ctx, int vset_id, const double *coeffs_host, int n_samples,
                            const double *e_lab_host, int n_E, wpcd_precision prec, wpcd_resolvent res,
                            double *t_out_host, double *delta_host, double *sigma_host);

/* ---- spin observables: App. A -----------------------------------------------------------------------
 * From phase shifts delta_dev [n_samples][n_ch][n_E][3] (degrees, the layout
 * wpcd_observables writes, channels as passed here) at lab energies
 * e_lab_dev [n_E] (MeV): the M-matrix partial-wave expansion with the
 * incoming momentum along z and phi = 0,
 *   M^s_{m'm} = sqrt(4 pi)/(2 i p) sum_{J,l,l'} sqrt(2l+1) C(l' (m-m') s m' | J m)
 *               C(l 0 s m | J m) (S_{l'l} - delta_{l'l}) Y_{l'}^{m-m'}(theta, 0),
 * over the np channels (tz = 0; every channel once, S from the Stapp phases),
 * then the Saclay amplitudes as the coefficients of
 *   M = [(a+b) + (a-b)(s1.n)(s2.n) + (c+d)(s1.m)(s2.m) + (c-d)(s1.l)(s2.l) + e(s1+s2).n] / 2
 * (l, m, n along p + p', p - p', p x p'; the e term along n, the parity-even
 * form) and dsigma/dOmega = Tr(M M^+)/4 = (|a|^2+|b|^2+|c|^2+|d|^2+|e|^2)/2.
 * theta_dev [n_theta] radians.  Outputs (device, either may be NULL):
 * abcde_dev [n_samples][n_E][n_theta][5] complex (re, im) in fm;
 * dsig_dev [n_samples][n_E][n_theta] mb/sr.  Synchronises.  Errors:
 * WPCD_ERR_ARG, WPCD_ERR_NOMEM, WPCD_ERR_CUDA. */
wpcd_status wpcd_saclay(wpcd_ctx *ctx, const wpcd_channel *channels, int n_ch, const double *delta_dev,
                        int n_samples, const double *e_lab_dev, int n_E, const double *theta_dev, int n_theta,
                        double *abcde_dev, double *dsig_dev);

/* ---- MI comparison method: Sec. 2.1 (matrix inversion), Sec. 6 (interpolation) ---------------------
 * The LS equation solved directly on a momentum grid: N_Q Gauss-Legendre
 * points mapped by k = c tan(pi (1 + x) / 4) plus the on-shell point p, with
 * the Haftel-Tabakin pole subtraction
 *   D_j = w_j k_j^2 2 mu / (p^2 - k_j^2),  D_N = -2 mu p^2 sum_j w_j / (p^2 - k_j^2),
 *   (1 - V D) K = V,  T = (1 + i pi mu p K)^-1 K,  S = 1 - 2 pi i mu p T.
 * wpcd_mi_prepare evaluates the built-in potential's terms (generator_id
 * WPCD_GEN_YAMAGUCHI or WPCD_GEN_YUKAWA, parameters as for wpcd_project) on
 * the grid for the channels; n_quad = N_Q in [4, 100] (both l-blocks of a
 * coupled channel, 2 (N_Q + 1) rows, are factorised in one CTA's shared
 * memory), c_map_fm = c > 0.  Errors: WPCD_ERR_ARG, WPCD_ERR_NOMEM,
 * WPCD_ERR_BUDGET, WPCD_ERR_CUDA.  The handle is freed by wpcd_release. */
wpcd_status wpcd_mi_prepare(wpcd_ctx *ctx, const wpcd_channel *channels, int n_ch, int generator_id,
                            const double *gen_params_host, int n_gen_params, int n_terms, int n_quad,
                            double c_map_fm, int *mi_id);

/* Solve at the n_I >= 2 interpolation energies e_int_dev (MeV, ascending,
 * device) for every sample (coeffs_dev [n_samples][n_terms-1], device) and
 * channel, then interpolate the phase shifts linearly in T_lab to the requested
 * energies e_lab_dev [n_E] (the end segments extended; delta moved by
 * multiples of 180 deg to within 90 deg of the segment start) and form the np
 * total cross section as wpcd_observables does.  Each system is factorised in
 * FP32 (partial pivoting) and its solution refined with FP64 residuals until
 * it converges (below).  Outputs (device, any may be
 * NULL but not all): k_out_dev [n_samples][n_ch][n_I][2][2] the on-shell K
 * (fm^2, uncoupled channels in [0][0]); delta_dev [n_samples][n_ch][n_E][3]
 * degrees; sigma_dev [n_samples][n_E] mb; status_dev (may be NULL)
 * [n_samples][n_ch] int, the most refinement steps any energy of that
 * (sample, channel) took (31: solved by the FP64 fallback below), or -1.  A
 * system whose refinement neither reaches a correction below 1e-14 of the
 * solution nor stagnates below 1e-9 of it (the accuracy floor of an FP64
 * factorisation, ~cond u_64) within 30 steps is solved again by FP64
 * Gauss-Jordan elimination with partial pivoting; only an exactly singular
 * system is reported, by wpcd_sync, as WPCD_ERR_NOCONVERGE.  Errors: WPCD_ERR_ARG,
 * WPCD_ERR_HANDLE, WPCD_ERR_NOMEM, WPCD_ERR_BUDGET, WPCD_ERR_CUDA. */
wpcd_status wpcd_mi_solve(wpcd_ctx *ctx, int mi_id, const double *coeffs_dev, int n_samples, const double *e_int_dev,
                          int n_I, const double *e_lab_dev, int n_E, double *k_out_dev, double *delta_dev,
                          double *sigma_dev, int *status_dev);

/* Free a mesh, vset, eig or MI handle.  Errors: WPCD_ERR_HANDLE. */
wpcd_status wpcd_release(wpcd_ctx *ctx, int id);

/* ---- tracing ---------------------------------------------------------------------------------
 * Kernel phases for the per-launch event timing of wpcd_profile. */
enum {
    WPCD_PHASE_MESH = 0,        /* Gauss-Legendre rules and meshes */
    WPCD_PHASE_PROJECT = 1,     /* projection of the potential terms */
    WPCD_PHASE_EIGEN = 2,       /* parameter sum + eigensolve */
    WPCD_PHASE_PLAN = 3,        /* energy -> bin plan */
    WPCD_PHASE_TMATRIX = 4,     /* SWP boundaries, resolvent, T, phases at the bins */
    WPCD_PHASE_GATHER = 5,      /* T at the requested energies */
    WPCD_PHASE_OBSERVABLES = 6, /* interpolation and cross section */
    WPCD_PHASE_REFINE = 7,      /* FP64 refinement of the mixed path's eigenpairs */
    WPCD_PHASE_MI = 8,          /* the MI comparison method */
    WPCD_PHASE_COUNT = 9
};

/* Batched square products C_b = op(A_b) B_b (op(A) = A^T if trans_a) for `items`
 * n x n row-major FP64 matrices stored back to back, queued on the context
 * stream -- the refinement products of the mixed path, exposed for reuse and
 * testing.  engine WPCD_REFINE_TENSOR: each row of op(A) and column of B is
 * scaled by a power of two, rounded to 47 bits and split into six balanced
 * 8-bit digits (exact in BF16); digit products are summed exactly in FP32 on
 * the tensor cores (k <= 256 per sum) and combined in FP64 (Ozaki, Ogita,
 * Oishi, Rump, "Error-free transformations of matrix multiplication", 2012).
 * Error <~ 2^-48 (max_k|op(A)_ik| sum_k|B_kj| + sum_k|op(A)_ik| max_k|B_kj|).
 * engine WPCD_REFINE_FP64: FP64 FMA.
 * n <= 1024.  Errors: WPCD_ERR_ARG, WPCD_ERR_NOMEM, WPCD_ERR_CUDA. */
wpcd_status wpcd_batched_dgemm(wpcd_ctx *ctx, int n, int items, int trans_a, const double *A_dev,
                               const double *B_dev, double *C_dev, int engine);

/* The autotuner's table: up to max_entries (n, precision, chosen CTA size) and,
 * in ms_out[5 k + j], the measured time per solve of candidate j (64, 128, 256,
 * 512, 1024 threads; 1024 only for the FP32 kernel; negative = not run).
 * Returns the number of entries. */
int wpcd_tuning(wpcd_ctx *ctx, int max_entries, int *n_out, int *prec_out, int *threads_out, float *ms_out);

/* Number of kernels this context has launched since creation (host count;
 * a graph launch counts the kernels it holds). */
unsigned long long wpcd_kernel_launches(const wpcd_ctx *ctx);

/* The natural logarithm the resolvent kernel uses (table-driven after Tang,
 * ACM TOMS 16, 1990; about 1 ulp for positive normal arguments, the CUDA
 * library log for zero, subnormal, infinite and NaN ones), applied to n device
 * doubles x_dev into y_dev on the context stream: a test hook for comparing it
 * with other implementations.  Errors: WPCD_ERR_ARG, WPCD_ERR_CUDA. */
wpcd_status wpcd_device_log(wpcd_ctx *ctx, const double *x_dev, double *y_dev, int n);

/* CUDA-graph use of wpcd_solve: graphs captured and graph launches since the
 * context was created, and graphs currently cached.  Either pointer may be NULL.
 * Errors: WPCD_ERR_ARG (null context). */
wpcd_status wpcd_graph_stats(wpcd_ctx *ctx, unsigned long long *captures, unsigned long long *replays,
                             int *cached);

/* Turn per-launch CUDA-event timing on (1) or off (0); either call clears the
 * accumulated totals.  Timing adds two events per launch on the context stream. */
wpcd_status wpcd_profile(wpcd_ctx *ctx, int enable);

/* Synchronise and return the summed device time (ms) and the launch count of
 * one phase since profiling was enabled.  Errors: WPCD_ERR_ARG. */
wpcd_status wpcd_profile_read(wpcd_ctx *ctx, int phase, double *ms_total, long *launches);

/* Number of channels and matrix size of channel c in a vset. */
wpcd_status wpcd_vset_info(wpcd_ctx *ctx, int vset_id, int *n_ch, int *n_terms, int channel, int *n);

/* ---- serving: continuous batching -----------------------------------------------------------
 * wpcd_serve_start builds, for every N_WP in n_wp_list, the default mesh
 * (tan^2 map to 8 fm^-1, 8 points per bin, momentum packets) and the projected
 * potential of the channel set, keeps them resident, and starts a worker
 * thread with n_slots executors (each its own CUDA stream and workspaces).
 * Requests queue FIFO; whenever a slot is free the worker takes the oldest
 * request and every queued request with the same (N_WP, precision), up to
 * max_batch, and runs the whole hot path for that batch on the slot's stream
 * (each request keeps its own energy list), so batches overlap on the device
 * and new requests join as slots free up.  Admission: wpcd_submit refuses with
 * WPCD_ERR_BUDGET when max_queue requests wait, or when the context has an HBM
 * budget and the queued requests' working memory would exceed what is left.
 * Results (delta [n_ch][n_E][3] deg, sigma [n_E] mb, T [n_ch][n_E][2][2]
 * complex, host memory) belong to the context until wpcd_release_result;
 * latency_us is submit -> results ready on the host.  No counterpart in the
 * paper (its GPU code ran one prediction at a time). */
typedef struct {
    const double *coeffs; /* [n_terms] host: the sample's coefficients (n_terms = model terms - 1) */
    int n_terms;
    const double *e_lab;  /* [n_E] host, MeV */
    int n_E;
    int n_wp;             /* one of the served N_WP */
    wpcd_precision prec;
} wpcd_request;

typedef struct {
    wpcd_status status;
    int n_E, n_ch;
    const double *delta;
    const double *sigma;
    const double *T;
    double latency_us;
} wpcd_result;

wpcd_status wpcd_serve_start(wpcd_ctx *ctx, const wpcd_channel *channels, int n_ch, int generator_id,
                             const double *gen_params_host, int n_gen_params, int n_terms, const int *n_wp_list,
                             int n_nwp, int max_batch, int n_slots, int max_queue);
/* Drain the queue, stop the worker and free the serving state. */
wpcd_status wpcd_serve_stop(wpcd_ctx *ctx);
/* Copy a request (the caller may reuse its buffers afterwards).  Errors:
 * WPCD_ERR_ARG (no server, unserved N_WP, an energy that is not positive or
 * whose momentum is not below the mesh's top boundary -- checked here, with the
 * energy plan's own test, so that it never reaches a batch), WPCD_ERR_BUDGET
 * (admission refused).  A result's status is its own: WPCD_ERR_NOCONVERGE when
 * one of its solves hit the sweep cap, whatever the other requests of its
 * batch did; an error of the batch's launch or layout fails every request of
 * that batch. */
wpcd_status wpcd_submit(wpcd_ctx *ctx, const wpcd_request *req, uint64_t *ticket);
/* WPCD_OK and the result, WPCD_ERR_NOTREADY while in flight, WPCD_ERR_HANDLE for an unknown ticket. */
wpcd_status wpcd_poll(wpcd_ctx *ctx, uint64_t ticket, wpcd_result *out);
/* As wpcd_poll, blocking up to timeout_ms; WPCD_ERR_TIMEOUT if still in flight. */
wpcd_status wpcd_wait(wpcd_ctx *ctx, uint64_t ticket, int timeout_ms, wpcd_result *out);
/* Free a finished request's results (no-op while it is in flight). */
void wpcd_release_result(wpcd_ctx *ctx, uint64_t ticket);
/* Requests finished, batches launched, requests waiting. */
wpcd_status wpcd_serve_stats(wpcd_ctx *ctx, unsigned long long *completed, unsigned long long *batches,
                             unsigned long long *queued);

/* ---- the per-channel hot path without device allocation -------------------------------------
 * No counterpart in the paper: this entry point exists for callers that cannot
 * call cudaMalloc -- an application that owns all device memory through its own
 * pool and forbids libraries from allocating, or a latency-critical loop that
 * cannot take cudaMalloc's implicit device synchronisation.
 *
 * For one channel and n_samples parameter samples it runs what wpcd_solve runs
 * for that channel: builds the mesh (same arguments as wpcd_mesh), forms
 * H = diag(H0) + V0 + sum_a c_a V_a, diagonalises it (FP64 Jacobi), and
 * writes T at every requested energy (t_out_dev, layout of wpcd_tmatrix with
 * n_ch = 1) and the interpolated phase shifts (delta_dev, layout of
 * wpcd_observables with n_ch = 1; no cross section, which sums channels).
 * V_dev: the channel's projected terms [n_terms][n][n] FP64 (n = K n_wp), e.g.
 * from wpcd_vset_get; coeffs_dev: [n_samples][n_terms-1] (NULL if n_terms == 1).
 * Either output may be NULL, not both.  status_dev (optional, caller-zeroed
 * int on the device) receives the first device-side error code (1 = an energy
 * outside the mesh, 2 = no convergence).  Work is queued on cuda_stream (NULL =
 * legacy default stream) and the call returns without synchronising.
 *
 * It allocates nothing: every intermediate lives in one file-scope device
 * array of 16 MiB, held by every GPU that loads the library until exit.  A
 * problem whose intermediates do not fit (roughly n_samples * (K n_wp)^2 * 8
 * bytes plus small terms) is rejected with WPCD_ERR_ARG.  The first call on
 * each device looks up the array's device address with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after cudaDeviceReset (or anything else that
 * recreates the device's primary context) the array may move, so do not call
 * this entry point on a device that was reset.  All calls share the array:
 * calls whose work overlaps on the GPU race on it and must be serialised by
 * the caller (one stream, or events).
 * Errors: WPCD_ERR_ARG, WPCD_ERR_CUDA. */
wpcd_status wpcd_channel_solve_noalloc(int n_wp, int mesh_kind, double alpha_fm, double t, double kmax_fm,
                                       int n_quad, int wp_kind, wpcd_channel channel, const double *V_dev,
                                       int n_terms, const double *coeffs_dev, int n_samples,
                                       const double *e_lab_dev, int n_E, double *t_out_dev, double *delta_dev,
                                       int *status_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* WPCD_H */
