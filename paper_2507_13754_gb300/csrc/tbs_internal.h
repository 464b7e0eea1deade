// tbs_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tbs {

// Row stride of the stored spectrum quadrant [(M/2+1) rows]: even, so every
// row starts 16-byte aligned and spans a multiple of 16 bytes (bulk copies).
__host__ __device__ constexpr int ghat_stride(int M) { return M / 2 + 2; }

// Per right-hand-side solver state, updated by the stop-test kernel.
struct RhsState {
    int done;        // 1 once the stop test has ended this RHS
    int terms;       // terms summed so far
    int status;      // TBS_* outcome
    int grow;        // consecutive terms with |u_n| > |u_{n-1}|
    double u0;       // |u_0|_2
    double prev;     // |u_{n-1}|_2
    double tmax;     // max |u_n|_2
    double residual; // last residual
    double psi_norm; // |psi_n|_2
    double pad_;
};

// Which right-hand sides a launch works on.
enum GateMode { GATE_ALL = 0, GATE_FWD = 1, GATE_ADJ = 2 };
struct Gate {
    const RhsState *st;  // per-RHS state
    int mode;
    int j;               // adjoint step: RHS active while j <= terms - 2
    const int *jdev;     // where the step is read from when j < 0 (graph loop)
};

// Row-pass variants.
enum RowKind {
    ROW_SRC = 0,       // y = src (spatial)              -> forward FFT -> X
    ROW_FWD = 1,       // W -> inverse FFT -> u; psi += u; norms; y = V u -> X
                       // (the last admissible term stops after the norms)
    ROW_ADJ = 3,       // W -> lambda; Q += conj(lambda) u_j; y = g + conj(V) lambda -> X
                       // (step j = 0 stops after Q)
    ROW_OUT = 5,       // W -> inverse FFT -> out (one application of G)
    ROW_VSRC = 6,      // y = V src (spatial) -> forward FFT -> X (recomputing a term)
    ROW_EPS = 7,       // periodic grid: W -> inverse FFT -> g; psi' = A g (A: absorbing
                       // layer, not at term 0); Eq. 30 sums of psi' - psi; y = V psi' + S -> X
    ROW_EPSK = 8       // ROW_EPS with the k-space potential: psi^0 = g stored at term 0,
                       // then psi' = A (g + psi^0); y = psi' -> X
};

struct StopArgs {
    const double2 *part;
    const double2 *l1;
    RhsState *st;
    double *norms;      // [rhs][max_terms]
    int *loop_ctl;      // graph loop: {arrivals, iterations}, or null outside one
    cudaGraphConditionalHandle loop;  // the WHILE node's condition (loop_ctl set)
    int n;
    int term;           // term index, or -1: each RHS's own count (RhsState::terms)
    int max_terms;
    double tol;
    int stop_mode;
    int div_grace;
    int div_window;
    double div_factor;
    int pdl;            // launch as a programmatic dependent of the previous kernel
};

struct RowArgs {
    const float2 *W;    // [rhs][N][M]
    const float2 *src;  // [rhs][N][N] spatial input (ROW_SRC), g (ROW_ADJ*)
    float2 *X;          // [rhs][N][M]
    float2 *psi;        // [rhs][N][N] partial sum (ROW_FWD*) / output (ROW_OUT)
    const float2 *V;    // [N][N]
    float2 *U;          // stored terms (ROW_FWD writes, ROW_ADJ reads), or null; term j
                        // is U + rhs * u_rhs + ((j - u_term0) / u_every) * u_slot
                        // (ROW_FWD stores only terms with (j - u_term0) % u_every == 0)
    size_t u_rhs, u_slot;
    int u_term0, u_every;
    float2 *Q;          // [rhs][N][N] adjoint accumulator
    double2 *part;      // [rhs][N] per-row (sum |u|^2, sum |psi|^2)
    double2 *l1;        // [rhs] (sum_row |u|, sum_row |psi_prev|)
    const float2 *tw;   // [M] twiddles
    Gate gate;
    int n;              // N
    int term;           // step j (adjoint); forward term index, or -1 for RhsState::terms
    int max_terms;
    int l1_row;         // row of the L1 test or -1
    int pdl;            // launch as a programmatic dependent of the previous kernel
    const float *abl;   // ROW_EPS/EPSK: per-axis absorbing-layer profile [N], or null
    float2 *psi0;       // ROW_EPSK: psi^0 = G S, stored at term 0 and added afterwards
    // ROW_EPS: per-row flags (null: every row dense): vflag[y] = 1 when row y
    // of V is one repeated value (read once), sflag[rhs][y] = 0 when row y of
    // that RHS's source is zero (not read)
    const unsigned char *vflag;
    const unsigned char *sflag;
    float cbs_inv_eps;  // ROW_EPS: 1 / eps with the convergent Born series preconditioner, else 0
    int *err;           // device error word (a bounded wait on a row copy ran out), or null
    unsigned long long wait_ns;  // limit of those waits
    int num_sms;        // SM count (persistent steady-state pass), or 0: one block per row
    int nrhs;           // set by the launcher
};

struct ColArgs {
    const float2 *X;    // [rhs][N][M]
    float2 *W;          // [rhs][N][M]
    const float2 *ghq;  // [(M/2+1)^2] spectrum quadrant
    const float2 *tw;   // [M]
    Gate gate;
    int n;
    int nrhs;
    int num_sms;        // persistent grid size (SMs x resident blocks per SM)
    int *err;           // device error word (a bounded wait ran out), or null
    unsigned long long wait_ns;  // limit of every wait on a copy
    unsigned extra_tx;  // fault injection: bytes a copy barrier expects in excess
    int xslice;         // set by the launcher: rows per slice of the 3D view of X
                        // (one tensor copy per tile), or 0: one 2D copy per BR rows
    int pdl;            // launch as a programmatic dependent of the previous kernel
    // periodic grid (N = M): the spectrum g~(p)/M^2 = 1/((|p|^2 - k0^2 - i eps) M^2)
    // is formed in the kernel from integer wavenumbers (ix, iy) in [-M/2, M/2):
    // g = gs (a + i eq) / (a^2 + eq^2), a = ix^2 + iy^2 - kq, with p = dp (ix, iy),
    // kq = k0^2/dp^2, eq = eps/dp^2, gs = 1/(dp^2 M^2)
    int periodic;
    float kq, eq, gs;
    // k-space absorbing-dispersive potential (periodic grid, after an RHS's
    // first term): the spectrum is multiplied by VV = a1 s^((nu+1)/2) -
    // i (a2 s^(nu/2) + eps), s = ix^2 + iy^2, a1 = eta dp^(nu+1), a2 = tau omega dp^nu
    int kspace;
    float vv_a1, vv_a2, vv_eps, vv_half_nu;
};



// Upper bound of the column-pass variants of any M (col_variants(M)); plans
// keep per-variant tensor maps and grids in arrays of this size.
constexpr int MAX_COL_VARIANTS = 8;

// Tensor maps of X (the column pass's tile loads) and W (its tile stores).
struct ColMaps {
    CUtensorMap x, w;
};

// launchers (tbs_kernels.cu); return cudaGetLastError() of the launch
cudaError_t launch_row(int kind, int M, int nrhs, const RowArgs &a, cudaStream_t s);
// column pass in tile-shape variant `variant` (0 = default; col_variants(M) exist)
cudaError_t launch_col(int M, int nrhs, bool conj_kernel, const ColArgs &a, const ColMaps *maps,
                       int variant, cudaStream_t s);
int col_variants(int M, bool periodic = false);
// a short description of a column-pass variant (nullptr outside the range)
const char *col_variant_name(int M, bool periodic, int variant);
// tensor maps of X and W ([nrhs * n][M] complex64 rows each) for the column
// pass's tile copies at this M and variant (of a periodic plan's variants
// when periodic is set; host, no allocation)
cudaError_t col_tensor_maps(ColMaps *maps, const float2 *X, const float2 *W, int n, int M, int nrhs, int variant,
                            bool periodic = false);
cudaError_t launch_stop(int nrhs, const StopArgs &a, cudaStream_t s);
// Adjoint graph loop control (one thread): with init, *j = max_r terms_r - 2,
// else *j -= 1; then the WHILE condition is set to (*j >= 0).
cudaError_t launch_adj_loop(int nrhs, const RhsState *st, int *j, cudaGraphConditionalHandle h, bool init,
                            cudaStream_t s);
cudaError_t launch_info(int nrhs, const RhsState *st, const int *err, void *info_dev, cudaStream_t s);
// V = p^2 - k0^2 - i eps_shift (eps_shift = 0 except on the periodic grid)
cudaError_t launch_medium(int count, const float *c, const float *alpha, double omega,
                          double c0, double tdel, double eps_shift, float2 *V, cudaStream_t s);
// *out = the bits of max |V + i eps_shift| over `count` points (FP64)
cudaError_t launch_potential_max(int count, const float2 *V, double eps_shift, unsigned long long *out,
                                 cudaStream_t s);
// V -= i eps_shift (a potential given directly, periodic grid)
cudaError_t launch_shift_potential(int count, double eps_shift, float2 *V, cudaStream_t s);
// the per-row flags of V and S that ROW_EPS reads (see RowArgs)
cudaError_t launch_row_flags(int n, int nrhs, const float2 *V, const float2 *S, unsigned char *vflag,
                             unsigned char *sflag, cudaStream_t s);
cudaError_t launch_deposit(int nrhs, int n, int n_cells, const int *cell, const int *seg,
                           const float2 *amp_sorted, int n_pts, double inv_dx2, float2 *S,
                           cudaStream_t s);
cudaError_t launch_harmonic2(int nrhs, int count, const float2 *psi1, const float *beta,
                             const float *rho, const float *c, double omega, float2 *S,
                             cudaStream_t s);
// the lower harmonics psi_1 .. psi_{order-1} ([nrhs][N][N] each)
struct HarmonicInputs {
    const float2 *psi[4];
    double scale[4];      // psi_a = scale[a-1] * psi[a-1]
    double source_scale;  // the source written is source_scale * S_n
};
cudaError_t launch_harmonic(int nrhs, int count, int order, const HarmonicInputs &in, const float *beta,
                            const float *rho, const float *c, double omega, float2 *S, cudaStream_t s);
cudaError_t launch_gradient(int nrhs, int count, const float2 *Q, const float *c,
                            const float *alpha, double omega, double tdel, float *grad_c,
                            float *grad_alpha, cudaStream_t s);
cudaError_t set_row_smem_attr(int M);
cudaError_t set_col_smem_attr(int M);

// plan build (tbs_plan.cu): twiddles and the spectrum quadrant of the
// cell-averaged Green's table.  Synchronous on s; returns the first error.
cudaError_t build_twiddles(int M, float2 *tw, cudaStream_t s);
cudaError_t build_ghat(int n, int M, double k0, double dx, float2 *ghq, cudaStream_t s);

// message returned by tbs_last_error() on this thread (tbs_api.cu)
void set_last_error(const char *msg);

// resident column-pass blocks per SM (after set_col_smem_attr), for the
// persistent grid (tbs_kernels.cu)
int col_resident_blocks_per_sm(int M, int variant, bool periodic = false);

}  // namespace tbs
