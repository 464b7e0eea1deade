/*
 * tbs.h -- C ABI of the GB300 traditional Born series (TBS) library.
 *
 * The library evaluates the Born series of the 2D inhomogeneous Helmholtz
 * equation (arxiv 2507.13754, Section 2.2):
 *
 *     lap(psi) + k0^2 psi = -S - V psi                         (Eq. 13)
 *     psi = sum_n u_n,  u_0 = G S,  u_{n+1} = G (V u_n)        (Eqs. 18-20)
 *
 * G is the convolution with the outgoing free-space Green's function
 * g(r) = (i/4) H0^(1)(k0 r) (Eq. 16 with epsilon -> 0), averaged over each
 * grid cell and applied as a zero-padded FFT convolution of size M (the
 * smallest power of two >= 2N - 1, at least 16), so that the result equals the
 * linear convolution on the N x N grid: (G f)[m] = dx^2 sum_n Gc[m - n] f[n].
 *
 * Conventions shared by every entry point:
 *   - Grids are N x N, row-major: element (iy, ix) at iy * N + ix.
 *   - Complex values are interleaved float pairs (re, im), i.e. complex64.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Work is enqueued on it; device pointers must stay valid until the
 *     stream reaches the enqueued work.
 *   - Pointers documented as "device" must be device (or managed) memory of
 *     the current device; "host" pointers are read before the call returns.
 *   - Every call returns a tbs_status.  On failure nothing is enqueued and
 *     tbs_last_error() returns a message for the calling thread.
 *   - A plan is not thread-safe; distinct plans are independent.
 *
 * Time convention exp(-i omega t): absorption gives Im(k) > 0.
 */
#ifndef TBS_H
#define TBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes of the API calls ------------------------------------- */
typedef enum tbs_status {
    TBS_OK = 0,
    TBS_ERR_INVALID_ARG = 1,      /* bad pointer, size, or parameter value     */
    TBS_ERR_UNSUPPORTED_SIZE = 2, /* N outside [2, TBS_MAX_N]                  */
    TBS_ERR_OOM = 3,              /* device allocation failed                  */
    TBS_ERR_CUDA = 4,             /* a CUDA runtime call failed                */
    TBS_ERR_STATE = 5             /* call out of order (e.g. adjoint w/o terms) */
} tbs_status;

/* ---- per right-hand-side outcome of a solve (data, not an error) -------- */
enum {
    TBS_CONVERGED = 0,  /* residual fell below tol                            */
    TBS_MAX_TERMS = 1,  /* max_terms summed (the fixed-term mode ends here)   */
    TBS_DIVERGED = 2,   /* growth rule fired (see tbs_plan_desc.div_*)        */
    TBS_NONFINITE = 3,  /* a norm became NaN or Inf                           */
    TBS_WAIT_TIMEOUT = 4, /* a kernel's bounded wait for a copy ran out; the
                           * field is invalid (never expected; see the fault
                           * injection hook tbs_debug_set)                    */
    TBS_COPY_CHECK_FAILED = 5 /* a copy failed the kernel's alignment self-check
                               * and was skipped; the field is invalid        */
};

/* ---- stop tests -------------------------------------------------------- */
enum {
    /* r_n = |u_n|_2 / |psi_n|_2 over the whole N x N grid, sums in FP64      */
    TBS_STOP_L2 = 0,
    /* r_n = sum_x |u_n(row, x)| / sum_x |psi_{n-1}(row, x)| on one row, FP64:
     * the error of Eq. 30 (Section 3.1); evaluated from n = 1 on            */
    TBS_STOP_L1_ROW = 1
};

/* ---- plan flags -------------------------------------------------------- */
enum {
    /* keep every term u_n of the last solve on the device, as the adjoint
     * needs them ([n_rhs][max_terms][N][N] complex64)                       */
    TBS_FLAG_KEEP_TERMS = 1u << 0,
    /* launch the solve as individual kernels instead of a cached CUDA graph */
    TBS_FLAG_NO_GRAPH = 1u << 1,
    /* with TBS_FLAG_KEEP_TERMS: keep only every K-th term (K = ceil(sqrt(
     * max_terms))) and recompute the others, a segment of K at a time, during
     * tbs_solve_adjoint -- term memory ceil(max_terms / K) + K instead of
     * max_terms fields per RHS (plus one N x M intermediate per RHS), for
     * about one more forward pass of work.  The gradient is bitwise that of
     * the stored-terms adjoint (the recomputation runs the same kernels).  */
    TBS_FLAG_CHECKPOINT_TERMS = 1u << 2,
    /* The paper's own discretisation (Section 2.2 with finite epsilon,
     * Section 3.1, Algorithm 1): a periodic N x N grid without padding
     * (N a power of two, 16 .. TBS_MAX_N_PERIODIC), the spectral Green's
     * function g~(p) = 1 / (|p|^2 - k0^2 - i eps) with eps = eps_factor k0^2
     * formed in the column pass (no table is built), V = U - i eps (the
     * plan subtracts i eps from tbs_set_medium's and tbs_set_potential's
     * U), and the iteration on the field itself,
     *   psi^0 = G S,   psi^{l+1} = A . G (V psi^l + S),
     * A the absorbing layer of abl_width cells (Eq. 29: the sigmoid
     * 1/(1 + exp(-abl_zeta (x - mu/2))) at distance x from the nearer edge,
     * mu = abl_width dx; the two axes' profiles multiply).  A solve "term"
     * is one iteration: info.terms counts psi^0 .. psi^{terms-1}, the stop
     * test compares psi^{l+1} with psi^l (L1 row: Eq. 30; L2: whole grid).
     * Not combinable with TBS_FLAG_KEEP_TERMS; tbs_get_ghat and
     * tbs_solve_adjoint return STATE. */
    TBS_FLAG_PERIODIC = 1u << 3,
    /* With TBS_FLAG_PERIODIC: the paper's absorbing-dispersive medium (Eq. 24,
     * Algorithm 1 case II) as a k-space potential,
     *   VV(p) = eta |p|^(nu+1) - i (tau omega |p|^nu + eps),
     *   tau = -2 alpha0 c0^(nu-1),  eta = 2 alpha0 c0^nu tan(pi nu / 2),
     * alpha0 = kspace_alpha0 [Np (rad/s)^-nu m^-1], nu = kspace_nu, applied to
     * the field's spectrum: psi^0 = G S, psi^{l+1} = A . F^-1 g~ (VV F psi^l +
     * F S) (computed as A . (F^-1 g~ VV F psi^l + psi^0)).  The spatial
     * potential is not used (the paper's case II is homogeneous).  With
     * kspace_absorption_only = 1, eta = 0 (absorption without dispersion). */
    TBS_FLAG_KSPACE_ABSORPTION = 1u << 4,
    /* With TBS_FLAG_PERIODIC (not with the k-space potential): the convergent
     * Born series preconditioner (Osnabrugge, Leedumrongwatthanakun and
     * Vellekoop, J. Comput. Phys. 322, 2016; the paper names the method as
     * future work, Section 5) on the periodic iteration,
     *   psi^{l+1} = A . (psi^l + gamma (G (V psi^l + S) - psi^l)),
     *   gamma = i V / eps,
     * which converges for any medium once eps >= max |U| (U = V + i eps the
     * unshifted potential): set eps_factor >= max |U| / k0^2, or
     * eps_factor = 0 to let the plan choose eps = 1.01 max |U| from each
     * medium (tbs_set_medium and tbs_set_potential then read max |U| back
     * from the device: they synchronize their stream; tbs_plan_eps reports
     * the choice).  The fixed point without a layer is the plain
     * iteration's. */
    TBS_FLAG_CBS = 1u << 5
};

#define TBS_MAX_N 2048        /* largest grid side (M = 4096)             */
#define TBS_MAX_N_PERIODIC 4096 /* largest side of a periodic grid (M = N) */
#define TBS_MAX_TERMS_CAP 4096

typedef struct tbs_plan_desc {
    int32_t n;            /* grid side N, 2 <= N <= TBS_MAX_N                 */
    int32_t n_rhs;        /* right-hand sides solved together (share V), >= 1 */
    double dx;            /* cell size [m], > 0                              */
    double freq_hz;       /* solve frequency f [Hz], > 0                      */
    double c0;            /* background sound speed [m/s]; k0 = 2 pi f / c0  */
    int32_t max_terms;    /* number of terms cap, 1 .. TBS_MAX_TERMS_CAP      */
    double tol;           /* stop threshold; 0 = always sum max_terms terms  */
    int32_t stop_mode;    /* TBS_STOP_L2 or TBS_STOP_L1_ROW                   */
    int32_t l1_row;       /* row of the L1 test; < 0 selects N/2              */
    int32_t div_grace;    /* growth test starts at term index div_grace (8)   */
    int32_t div_window;   /* that many consecutive growing |u_n| => DIVERGED (4) */
    double div_factor;    /* |u_n| > div_factor |u_0| => DIVERGED (1e6)       */
    uint32_t flags;       /* TBS_FLAG_*                                       */
    /* periodic grid only (TBS_FLAG_PERIODIC): */
    double eps_factor;    /* eps = eps_factor * k0^2 (0.8, Section 3.1), > 0
                           * (0 with TBS_FLAG_CBS: chosen from the medium)   */
    int32_t abl_width;    /* absorbing-layer width in cells, 0 .. N/2 (0: none) */
    double abl_zeta;      /* its steepness zeta [Np/m] (> 0 when abl_width > 0) */
    double kspace_alpha0; /* TBS_FLAG_KSPACE_ABSORPTION: alpha0 (>= 0)          */
    double kspace_nu;     /* and nu (0 < nu < 3)                               */
    int32_t kspace_absorption_only; /* 1: drop the dispersive eta term (the
                             * paper's "absorbing" case, Table 2); 0: Eq. 24 */
} tbs_plan_desc;

/* Outcome of one right-hand side, written by tbs_solve. */
typedef struct tbs_solve_info {
    int32_t terms;        /* terms summed into psi (u_0 .. u_{terms-1})       */
    int32_t status;       /* TBS_CONVERGED / MAX_TERMS / DIVERGED / NONFINITE */
    double residual;      /* last residual r_n evaluated (FP64)               */
    double term_norm_max; /* max_n |u_n|_2                                    */
    double psi_norm;      /* |psi|_2 at stop                                  */
} tbs_solve_info;

typedef struct tbs_plan_s *tbs_plan_t;

/* Fill *d with defaults (tol 1e-6, L2 stop, div_grace 8, div_window 4,
 * div_factor 1e6, max_terms 64, n_rhs 1, no flags, eps_factor 0.8, no
 * absorbing layer); the caller then sets n, dx, freq_hz and c0. */
void tbs_plan_desc_init(tbs_plan_desc *d);

/* Create a plan: allocates the plan's device buffers on the current device
 * and builds the spectrum of the cell-averaged Green's table,
 *   Gc[d] = (1/dx^2) * integral over cell d of (i/4) H0^(1)(k0 |r|) d^2r
 *   (Section 2.2, Eq. 16; G = F^-1 g~ F as below Eq. 17),
 * wrapped into M x M, transformed in FP64 and stored as complex64 scaled by
 * dx^2/M^2.  The plan owns its memory until tbs_destroy.  The call is
 * synchronous (it waits for the table build on `stream`).
 * Errors: INVALID_ARG (NULL pointers, dx/f/c0 <= 0, n_rhs < 1, bad
 * max_terms, tol < 0, bad stop mode or row), UNSUPPORTED_SIZE, OOM, CUDA. */
tbs_status tbs_plan(const tbs_plan_desc *d, void *stream, tbs_plan_t *out);

/* Device bytes of a plan's fixed-size buffers (Ghat quadrant, twiddles, V,
 * medium, sources, the two N x M intermediates per RHS, psi, norms, state;
 * the stored terms with TBS_FLAG_KEEP_TERMS), each at a 256-byte aligned
 * offset: what tbs_plan allocates in one block, and the workspace size
 * tbs_plan_with_workspace needs.  No allocation, no device work. */
tbs_status tbs_plan_device_bytes(const tbs_plan_desc *d, size_t *bytes);

/* As tbs_plan, but the fixed-size buffers are carved from the caller's
 * device memory `workspace` (256-byte aligned, >= tbs_plan_device_bytes(d)
 * bytes; e.g. a tensor from a framework's caching allocator).  The caller
 * owns it: it must stay allocated, on the plan's device and unused by
 * anything else until tbs_destroy, which does not free it.  Only the
 * point-source lists of tbs_set_sources (12 bytes per point and RHS) are
 * still allocated by the plan.  Errors: as tbs_plan; INVALID_ARG also for a
 * NULL, host, misaligned or too small workspace.  This entry point has no
 * counterpart in the paper: it lets a caller's allocator own plan memory. */
tbs_status tbs_plan_with_workspace(const tbs_plan_desc *d, void *workspace, size_t workspace_bytes,
                                   void *stream, tbs_plan_t *out);

/* Padded FFT size M of the plan. */
int32_t tbs_plan_padded_size(tbs_plan_t plan);

/* Set the medium and build V = p^2 - k0^2 on the device (Eq. 13; Eq. 25 for
 * a scatterer), with the power-law absorption and dispersion of Eqs. 3, 4
 * and 7 to first order in alpha:
 *     p = omega / c + alpha * (tan(pi y / 2) * delta + i),
 *     delta = 1 - (f_ref / f)^(y - 1)   (delta = 1 when f_ref <= 0).
 * c: device float[N*N] phase speed [m/s] at f_ref (> 0 everywhere).
 * alpha: device float[N*N] absorption [Np/m] at the solve frequency, or NULL
 *        for a lossless medium.
 * The plan copies c and alpha (the adjoint needs them); the caller may
 * reuse its buffers once the stream has passed this call.
 * Errors: INVALID_ARG on NULL plan/c. */
tbs_status tbs_set_medium(tbs_plan_t plan, const float *c, const float *alpha,
                          double y_pow, double f_ref_hz, void *stream);

/* Set V directly: device complex64 [N*N] (the adjoint then has no dV/dc). */
tbs_status tbs_set_potential(tbs_plan_t plan, const float *V, void *stream);

/* Point sources (Section 3.1, Algorithm 1's source table): the source of
 * right-hand side r is S_r = sum_j amp[r][j] delta_{(ix[j], iy[j])} / dx^2,
 * a discrete delta of unit integral, so an isolated element radiates
 * amp * Gc.  Elements sharing a cell add.
 * ix, iy: host int32[n_pts], 0 <= ix, iy < N.
 * amp: host complex64 [n_rhs][n_pts].
 * Errors: INVALID_ARG (n_pts < 0, index outside the grid, NULL). */
tbs_status tbs_set_sources(tbs_plan_t plan, int32_t n_pts, const int32_t *ix,
                           const int32_t *iy, const float *amp, void *stream);

/* Dense source field: device complex64 [n_rhs][N][N] (copied). */
tbs_status tbs_set_source_field(tbs_plan_t plan, const float *S, void *stream);

/* Second-harmonic source of the sum-term series (Eq. 28b, Eq. 11):
 *     S2 = -(1/2) xi (2 omega)^2 psi1^2,   xi = beta / (rho c^4),
 * written as the dense source of `plan` (whose frequency is 2 omega/2pi).
 * psi1: device complex64 [n_rhs][N][N], the fundamental field.
 * beta, rho, c: device float[N*N] (beta = 1 + B/2A).
 * omega_fundamental: 2 pi f of the fundamental.
 * Errors: INVALID_ARG on NULL pointers. */
tbs_status tbs_set_harmonic2_source(tbs_plan_t plan, const float *psi1, const float *beta,
                                    const float *rho, const float *c,
                                    double omega_fundamental, void *stream);

/* Run the series for all right-hand sides until each stops.
 * psi: device complex64 [n_rhs][N][N], written with the partial sum at stop.
 * info: tbs_solve_info[n_rhs], host or device memory; written asynchronously
 *       (synchronise the stream before reading host memory).
 * The stop test runs on the device in FP64 after every term; no per-term
 * host round trip.  Outcomes are data in info, not errors.
 * Errors: INVALID_ARG (NULL), STATE (no medium or no sources set), CUDA. */
tbs_status tbs_solve(tbs_plan_t plan, float *psi, tbs_solve_info *info, void *stream);

/* Batched solves: many plans (e.g. one per frequency of a broadband sweep,
 * each with its steering configurations as right-hand sides) captured as
 * parallel branches of ONE CUDA graph and launched together; each branch is
 * exactly the tbs_solve sequence of its plan, followed by copies of its psi
 * and info records.
 * plans: n_plans distinct plans (not freed before tbs_batch_destroy).
 * psi[i]: device complex64 [n_rhs_i][N_i][N_i]; info[i]: DEVICE
 *         tbs_solve_info[n_rhs_i] (the copies are graph nodes).
 * The graph is built once by tbs_batch_create; media and sources may change
 * between tbs_batch_solve calls (they are data in the plans' buffers).
 * Errors: INVALID_ARG (NULL, n_plans < 1, repeated plan, host info pointer),
 * STATE (a plan with per-kernel timing on, or without medium / sources at
 * solve time), CUDA. */
typedef struct tbs_batch_s *tbs_batch_t;
tbs_status tbs_batch_create(const tbs_plan_t *plans, int32_t n_plans, float *const *psi,
                            tbs_solve_info *const *info, tbs_batch_t *out);
tbs_status tbs_batch_solve(tbs_batch_t batch, void *stream);
tbs_status tbs_batch_destroy(tbs_batch_t batch);

/* Gradient of a real loss L(psi) with respect to c(x) and alpha(x) through
 * the truncated series of the last tbs_solve (its per-RHS term counts):
 *     ubar_{T-1} = g,  lambda_{j+1} = G^H ubar_{j+1},
 *     ubar_j = g + conj(V) lambda_{j+1},
 *     Q = sum_rhs sum_{j=0}^{T-2} conj(lambda_{j+1}) u_j,
 *     dL/dc = Re(Q dV/dc),  dL/dalpha = Re(Q dV/dalpha),
 * with G^H the convolution with conj(Gc) and V = p^2 - k0^2 as in
 * tbs_set_medium.  The adjoint of Eqs. 18-20 with respect to V.
 * grad_psi: device complex64 [n_rhs][N][N], g = dL/dRe(psi) + i dL/dIm(psi).
 * grad_c, grad_alpha: device float[N*N], overwritten (summed over RHS);
 *                     either may be NULL.
 * Requires TBS_FLAG_KEEP_TERMS, a medium set by tbs_set_medium and a prior
 * tbs_solve; otherwise STATE.  With TBS_FLAG_CHECKPOINT_TERMS the call
 * reads the term counts back to the host (it waits for the forward solve)
 * and recomputes each segment of terms before its reverse steps. */
tbs_status tbs_solve_adjoint(tbs_plan_t plan, const float *grad_psi, float *grad_c,
                             float *grad_alpha, void *stream);

/* Sum-term source of harmonic `order` = n in 2 .. 5 (Eqs. 28b-28e,
 * Section 2.3; difference terms are dropped, as in the paper):
 *     S_n = -xi (n omega)^2 [ sum_{a<b, a+b=n} psi_a psi_b + psi_{n/2}^2 / 2 ],
 *     xi = beta / (rho c^4),
 * written, times source_scale, as the dense source of `plan` (whose
 * frequency is n omega / 2 pi; on a periodic plan eps_factor k0^2 then
 * gives the paper's eps_n).  The sum is formed in FP64.
 * psi_lower: host array of order - 1 device pointers, psi_lower[k] holding
 *            psi_{k+1} / psi_scale[k], complex64 [n_rhs][N][N].
 * psi_scale: host double[order - 1], or NULL for all ones.
 * Scaling: harmonic n falls off roughly like |psi_1|^n times the
 * nonlinearity, and in the paper's run psi_5 is near 1e-36, at the bottom
 * of FP32; the series itself is linear, so a chain keeps each harmonic as
 * psi_n / 2^e_n with the exponent it chose (source_scale = 2^-e_n) and
 * passes the 2^e_a back here as psi_scale.
 * beta, rho, c: device float[N*N].  omega_fundamental: 2 pi f of psi_1.
 * Errors: INVALID_ARG (order outside 2 .. 5, NULL pointers, a scale that is
 * not finite and > 0).
 * (tbs_set_harmonic2_source is the order-2 case without scaling.) */
tbs_status tbs_set_harmonic_source(tbs_plan_t plan, int32_t order, const float *const *psi_lower,
                                   const double *psi_scale, const float *beta, const float *rho,
                                   const float *c, double omega_fundamental, double source_scale,
                                   void *stream);

/* One application of G (conj_kernel = 0) or G^H (conj_kernel = 1):
 * out = G f on the N x N grid for every right-hand side.
 * f, out: device complex64 [n_rhs][N][N] (may not alias).
 * Asynchronous: an expired wait inside its kernels is reported afterwards
 * by tbs_device_error. */
tbs_status tbs_apply_green(tbs_plan_t plan, const float *f, float *out, int32_t conj_kernel,
                           void *stream);

/* Allocation-free variant of tbs_apply_green (the paper has no counterpart:
 * this entry point exists for callers that may not call cudaMalloc -- code
 * running during CUDA graph capture, inside a memory pool or allocator that
 * must not re-enter it, or in real-time loops whose device memory is all
 * allocated at start-up by someone else).
 * out = G f (conj_kernel = 0) or G^H f (conj_kernel = 1) for ONE right-hand
 * side on an n x n grid, 2 <= n <= TBS_NOALLOC_MAX_N.
 * ghat: device complex64 [(M/2+1)^2], the spectrum quadrant that tbs_get_ghat
 *       returns for a plan with the same n, dx, freq_hz and c0 (M = the
 *       smallest power of two >= max(2n - 1, 16)); the caller keeps it in
 *       memory it owns.
 * f, out: device complex64 [n][n] (may not alias).
 * The scratch is a fixed library-owned __device__ array of 2,635,680 bytes
 * (held by every GPU that loads the library until exit), shared by all calls:
 * calls that overlap on the GPU race.  The first call on a device sets that
 * device up (and waits for the set-up on `stream`); make it before any stream
 * capture.  After cudaDeviceReset the set-up is lost: do not call this entry
 * point again in that process.  No cudaMalloc, cudaFree or allocating
 * library routine is called.
 * The kernels' waits for their copies are bounded; a wait that runs out (a
 * lost copy, never expected) is recorded in an error word inside the
 * scratch (cleared by each call) and leaves `out` undefined.  The call
 * returns before its kernels run, so its return code does not cover that.
 * Errors: UNSUPPORTED_SIZE (n outside [2, TBS_NOALLOC_MAX_N]), INVALID_ARG
 * (NULL or aliasing pointers), CUDA. */
#define TBS_NOALLOC_MAX_N 256
tbs_status tbs_apply_green_noalloc(int32_t n, const float *ghat, const float *f, float *out,
                                   int32_t conj_kernel, void *stream);

/* max over the grid of |U|, U = V + i eps the plan's potential without the
 * periodic grid's shift (U = p^2 - k0^2 of tbs_set_medium, Eqs. 13 and 25),
 * reduced in FP64 on the device; synchronous on `stream`.  This is the
 * bound the convergent Born series needs (eps >= max |U|, TBS_FLAG_CBS).
 * out_host: host double.  Errors: INVALID_ARG, STATE (no medium), CUDA. */
tbs_status tbs_potential_max_abs(tbs_plan_t plan, double *out_host, void *stream);

/* The plan's eps (0 without TBS_FLAG_PERIODIC): eps_factor k0^2, or the
 * value chosen from the last medium when TBS_FLAG_CBS was given
 * eps_factor = 0.  0 for a NULL plan. */
double tbs_plan_eps(tbs_plan_t plan);

/* The device error word of the plan's last tbs_solve, tbs_solve_adjoint or
 * tbs_apply_green (each clears it when it starts): *code = 0,
 * TBS_WAIT_TIMEOUT (a kernel's bounded wait for a copy ran out) or
 * TBS_COPY_CHECK_FAILED (a copy failed a kernel's alignment self-check);
 * either leaves that call's output invalid.  Synchronizes `stream`.
 * (A solve also reports it per RHS in tbs_solve_info.status.)
 * Errors: INVALID_ARG, CUDA. */
tbs_status tbs_device_error(tbs_plan_t plan, int32_t *code, void *stream);

/* Copy the stored spectrum quadrant Ghat[ky][kx], 0 <= kx, ky <= M/2, to host
 * complex64 [(M/2+1)^2] (full table: Ghat[ky][kx] = Ghat[M-ky][kx] = ...). */
tbs_status tbs_get_ghat(tbs_plan_t plan, float *out_host);

/* Per-kernel CUDA-event timing of the next solves (enable != 0) and the
 * accumulated totals: milliseconds in the column passes and in the
 * steady-state row passes (those running both the inverse and the forward
 * transform), and the number of launches of each.  Launches of a right-hand
 * side that has already stopped are timed too (they return at once), so time
 * with tol = 0 for per-launch figures.  Timing forces non-graph launches. */
tbs_status tbs_set_timing(tbs_plan_t plan, int32_t enable);
tbs_status tbs_get_timing(tbs_plan_t plan, double *row_ms, int32_t *row_launches,
                          double *col_ms, int32_t *col_launches);

/* Column-pass variants compiled for the plan's M, listed fastest first as
 * measured on GB300 (variant 0 is a plan's default): the lockstep kernel's
 * tile widths (the default width and, for M >= 512, narrower tiles with
 * more resident blocks per SM) and, for M >= 1024, the pipelined kernel
 * (one or two columns per thread, the latter also with the two columns
 * staggered); at M = 4096 the pipelined kernel with two columns per thread
 * comes first, at M = 1024 and 2048 the narrowed lockstep tiles.  At
 * M = 4096 the list also holds the two-column pipelined kernel with the FFT
 * split into four radix-8 stages instead of three radix-16 ones; periodic plans have the lockstep kernel with two and with
 * one column per thread and, for M >= 1024, the pipelined kernel with two
 * columns per thread (plain and staggered).  Variants with the same radix
 * split give bitwise the same result; the radix-8 split rounds differently
 * (agreement to FP32 rounding, the same parity with the exact operator).
 * tbs_col_variant_name describes variant v (v < 0: the active one) in a
 * static string, NULL outside the range or for a NULL plan.
 * tbs_set_col_variant selects one (takes effect at the next solve);
 * tbs_autotune times every variant on the plan's own buffers (`reps`
 * launches each after a warm-up, on `stream`, synchronously), activates the
 * fastest and returns it in *best and the mean milliseconds per launch in
 * times_ms[v] (either may be NULL).  Errors: INVALID_ARG, CUDA. */
int32_t tbs_col_variants(tbs_plan_t plan);
const char *tbs_col_variant_name(tbs_plan_t plan, int32_t variant);
tbs_status tbs_set_col_variant(tbs_plan_t plan, int32_t variant);
tbs_status tbs_autotune(tbs_plan_t plan, int32_t reps, double *times_ms, int32_t *best, void *stream);

/* Steady-state row-pass variants (the pass of every term after the first,
 * Eq. 19's inverse row transform, accumulation, norms, potential product and
 * forward row transform; on a periodic plan the paper's iteration of
 * Section 3.1): variant 0 is a persistent kernel (one or two blocks per SM,
 * each taking rows in a fixed stride and bulk-copying the next row's inputs
 * while it transforms the current one), variant 1 launches one block per
 * row.  The persistent variant exists for M >= 512 with an even N (padded
 * plans) or N = M (periodic plans); other plans have variant 0 only, one
 * block per row.  Both give bitwise the same result.  tbs_row_variants,
 * tbs_row_variant_name and tbs_set_row_variant work as their column-pass
 * counterparts.  tbs_autotune_rows times each variant (`reps` launches after
 * a warm-up, on `stream`, synchronously) at a steady-state term on the
 * plan's current medium and intermediates, activates the fastest and
 * returns it in *best and the mean milliseconds per launch in times_ms[v]
 * (either may be NULL).  The timed launches write the plan's scratch
 * intermediates and a temporary [n_rhs][N][N] field that the call allocates
 * and frees (so the plan's result and stored terms are untouched); it
 * synchronises the device.  Errors: INVALID_ARG, OOM, CUDA. */
int32_t tbs_row_variants(tbs_plan_t plan);
const char *tbs_row_variant_name(tbs_plan_t plan, int32_t variant);
tbs_status tbs_set_row_variant(tbs_plan_t plan, int32_t variant);
tbs_status tbs_autotune_rows(tbs_plan_t plan, int32_t reps, double *times_ms, int32_t *best, void *stream);

/* Test hooks.  TBS_DEBUG_WAIT_LIMIT_NS: limit of every in-kernel wait for a
 * copy (default 1e9 ns).  TBS_DEBUG_EXTRA_TX: fault injection -- the column
 * pass's copy barriers expect `value` bytes more than their copies deliver,
 * so the bounded wait runs out, the kernel leaves and the solve reports
 * TBS_WAIT_TIMEOUT (0 restores normal operation).  Takes effect at the next
 * solve.  Errors: INVALID_ARG. */
enum { TBS_DEBUG_WAIT_LIMIT_NS = 1, TBS_DEBUG_EXTRA_TX = 2 };
tbs_status tbs_debug_set(tbs_plan_t plan, int32_t key, int64_t value);

/* Broadband synthesis: the time signal of a set of single-frequency fields
 * (e.g. one field per frequency of a sweep, each on its own lambda/8 grid
 * over the same physical domain) at a lattice of receiver positions,
 *     s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t),
 * with the e^{-i omega t} time convention of the outgoing Green's function
 * (Section 2.2); Re s is the pressure.  The paper works at one frequency at
 * a time; this is the inverse Fourier sum over its frequency-domain fields.
 * psi_k(X) interpolates field k bilinearly between its cell centres
 * (x_i = i dx_k, y_j = j dx_k): fractional indices X/dx_k, Y/dx_k clamped to
 * [0, n_k - 1] (a receiver outside a field's grid sees the edge value).
 * freqs: host array of n_freq entries; each field is device complex64
 *        [n_rhs][n_k][n_k], n_k >= 2, dx_k > 0, freq_hz and weight finite.
 * Receivers: X = x0 + ix sx, Y = y0 + iy sy for 0 <= ix < nx, 0 <= iy < ny
 * [m].  Times: t_j = t0 + j dt, 0 <= j < n_t [s].
 * out: device complex64 [n_rhs][ny][nx][n_t] (caller-owned; overwritten).
 * Phases are reduced in FP64 (f_k t_j mod 1), samples and sums are FP32.
 * Asynchronous on `stream`; no device memory is allocated.
 * Errors: INVALID_ARG (NULL pointers, counts < 1, a bad frequency entry). */
typedef struct tbs_synth_freq {
    const float *field;  /* device complex64 [n_rhs][n][n]        */
    int32_t n;           /* grid side (>= 2)                      */
    double dx;           /* cell size [m]                         */
    double freq_hz;      /* frequency f_k [Hz]                    */
    double weight;       /* real weight w_k (e.g. the frequency step) */
} tbs_synth_freq;
tbs_status tbs_synthesize(const tbs_synth_freq *freqs, int32_t n_freq, int32_t n_rhs, double x0, double y0,
                          double sx, double sy, int32_t nx, int32_t ny, double t0, double dt, int32_t n_t,
                          float *out, void *stream);

/* Release every device buffer of the plan. */
tbs_status tbs_destroy(tbs_plan_t plan);

const char *tbs_status_string(tbs_status s);

/* Message of the last failed call on this thread ("" if none). */
const char *tbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TBS_H */
