// tbs_kernels.cu -- the per-term kernels of the Born series (complex64 field,
// FP64 norms) and the small set-up kernels (medium, sources, harmonic source,
// gradient).
//
// One Born term u_{n+1} = G (V u_n) (arxiv 2507.13754, Eq. 19) is two passes
// over an N x M intermediate (row-major, rows y < N, M columns kx), with the
// zero padding never stored:
//
//   column pass C  X[y][kx] -> forward FFT along y (rows >= N are zero) ->
//                  x Ghat[ky][kx] -> inverse FFT along y -> keep y < N -> W
//   row pass R     W[y][kx] -> inverse FFT along x -> keep x < N = u_n ->
//                  psi += u_n, FP64 |u_n|^2 and |psi_n|^2 row sums ->
//                  V u_n, zero-extended -> forward FFT along x -> X
//
// so a term reads and writes the intermediate twice (4 N M 8 bytes), reads V
// and reads/writes psi.  Ghat carries the dx^2/M^2 scale, so both transforms
// are unnormalised.
#include "tbs_kernels.cuh"

namespace tbs {

// Stop decision for one RHS after its term `term` (a.term, or the RHS's own
// count), from the FP64 sums of |u_n|^2 and |psi_n|^2 (and the L1 row sums
// for Eq. 30).  One thread.
__device__ void stop_decide(const StopArgs &a, int rhs, double su, double sp) {
    RhsState *s = a.st + rhs;
    const double un = sqrt(su), pn = sqrt(sp);
    const int term = a.term >= 0 ? a.term : s->terms;
    a.norms[(size_t)rhs * a.max_terms + term] = un;
    if (term == 0) {
        s->u0 = un;
        s->tmax = un;
        s->grow = 0;
        s->residual = INFINITY;
        s->status = 1;  // TBS_MAX_TERMS until decided otherwise
    }
    if (un > s->tmax) s->tmax = un;
    s->terms = term + 1;
    s->psi_norm = pn;
    bool have_r = true;
    double r;
    if (a.stop_mode == 1) {
        if (term == 0) {
            have_r = false;
            r = INFINITY;
        } else {
            const double2 l = a.l1[rhs];
            r = l.x / l.y;
        }
    } else {
        r = pn > 0.0 ? un / pn : (un > 0.0 ? INFINITY : 0.0);
    }
    if (have_r) s->residual = r;
    if (term > 0) s->grow = (un > s->prev) ? s->grow + 1 : 0;
    int done = 0;
    if (!isfinite(un) || !isfinite(pn)) {
        s->status = 3;
        done = 1;
    } else if (have_r && r < a.tol) {
        s->status = 0;
        done = 1;
    } else if ((term >= a.div_grace && s->grow >= a.div_window) || un > a.div_factor * s->u0) {
        s->status = 2;
        done = 1;
    } else if (term + 1 >= a.max_terms) {
        s->status = 1;
        done = 1;
    }
    s->prev = un;
    s->done = done;
}

// Fixed-order FP64 reduction of the row partials of one RHS by a 256-thread
// block (per-thread strided sums, shuffle trees within and then across the
// warps), then the stop decision in thread 0.
__device__ void reduce_and_decide(const StopArgs &a, int rhs) {
    __shared__ double2 rw[8];
    double su = 0.0, sp = 0.0;
    const double2 *part = a.part + (size_t)rhs * a.n;
    for (int y = threadIdx.x; y < a.n; y += 256) {
        const double2 q = part[y];
        su += q.x;
        sp += q.y;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    if (lane == 0) rw[warp] = make_double2(su, sp);
    __syncthreads();
    if (warp == 0) {
        const double2 q = lane < 8 ? rw[lane] : make_double2(0.0, 0.0);
        su = q.x;
        sp = q.y;
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
        }
        if (lane == 0) stop_decide(a, rhs, su, sp);
    }
}

// One block per RHS.  Inside a graph loop the last block to finish also
// sets the WHILE condition: another iteration while any RHS is still active,
// and never more than max_terms iterations in all (so the loop ends even if a
// decision were lost).
__global__ void __launch_bounds__(256) stop_kernel(StopArgs a) {
    grid_dep_wait();
    const int rhs = blockIdx.x;
    if (!a.st[rhs].done) reduce_and_decide(a, rhs);
    if (a.loop_ctl && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.loop_ctl, 1) == (int)gridDim.x - 1) {
            __threadfence();
            const volatile RhsState *st = a.st;
            int more = 0;
            for (int r = 0; r < (int)gridDim.x; r++) more |= (st[r].done == 0);
            const int iters = a.loop_ctl[1] + 1;
            a.loop_ctl[1] = iters;
            a.loop_ctl[0] = 0;
            cudaGraphSetConditional(a.loop, (more && iters < a.max_terms) ? 1u : 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// stop test: FP64 reduction of the row partials, residual, divergence, flags
// (Eq. 30 for the L1 row mode; full-grid L2 otherwise)
// ---------------------------------------------------------------------------
struct InfoOut {  // layout of tbs_solve_info
    int32_t terms;
    int32_t status;
    double residual;
    double term_norm_max;
    double psi_norm;
};

__global__ void adj_loop_kernel(int nrhs, const RhsState *st, int *jdev, cudaGraphConditionalHandle h, int init) {
    int j;
    if (init) {
        int tmax = 0;
        for (int r = 0; r < nrhs; r++) tmax = max(tmax, st[r].terms);
        j = tmax - 2;
    } else {
        j = *jdev - 1;
    }
    *jdev = j;
    cudaGraphSetConditional(h, j >= 0 ? 1u : 0u);
}

__global__ void info_kernel(int nrhs, const RhsState *st, const int *err, InfoOut *out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    out[r].terms = st[r].terms;
    // error word: 1 -> TBS_WAIT_TIMEOUT (4), 2 -> TBS_COPY_CHECK_FAILED (5)
    out[r].status = (err && *err) ? 3 + *err : st[r].status;
    out[r].residual = st[r].residual;
    out[r].term_norm_max = st[r].tmax;
    out[r].psi_norm = st[r].psi_norm;
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------

// V = p^2 - k0^2, p = omega/c + alpha (tdel + i), tdel = tan(pi y/2) delta
// V = p^2 - k0^2 (Eqs. 3, 4, 7, 13, 25) with p = omega/c + alpha (tdel + i),
// k0 = omega/c0.  The two nearly equal squares are never formed: with
// d = Re p - k0 = omega (c0 - c) / (c c0) + alpha tdel (c0 - c is exact in FP32
// for c within a factor two of c0), Re V = d (2 k0 + d) - alpha^2 and
// Im V = 2 Re p alpha - eps_shift, so FP32 keeps V to a few ulp of itself
// (an FP64 evaluation was FP64-issue-bound on this GPU: ~0.1 ms at 2048^2).
__global__ void medium_kernel(int count, const float *__restrict__ c, const float *__restrict__ alpha,
                              float omega, float k0, float c0, float tdel, float eps_shift,
                              float2 *__restrict__ V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float ci = c[i];
    const float al = alpha ? alpha[i] : 0.f;
    const float d = fmaf(al, tdel, omega * (c0 - ci) / (ci * c0));
    const float pr = k0 + d;
    V[i] = make_float2(fmaf(d, fmaf(2.f, k0, d), -al * al), fmaf(2.f * pr, al, -eps_shift));
}

// Per-row flags for the periodic row pass: block (y, 0) sets vflag[y] = 1
// when every element of V's row y equals its first (compared bit for bit);
// block (y, 1 + r) sets sflag[r][y] = 1 when RHS r's source row y has a
// nonzero element.
__global__ void __launch_bounds__(256) row_flags_kernel(int n, const float2 *__restrict__ V,
                                                        const float2 *__restrict__ S,
                                                        unsigned char *__restrict__ vflag,
                                                        unsigned char *__restrict__ sflag) {
    const int y = blockIdx.x;
    if (blockIdx.y == 0) {
        const float2 *row = V + (size_t)y * n;
        const float2 v0 = row[0];
        int same = 1;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const float2 v = row[x];
            same &= (__float_as_uint(v.x) == __float_as_uint(v0.x)) & (__float_as_uint(v.y) == __float_as_uint(v0.y));
        }
        same = __syncthreads_and(same);
        if (threadIdx.x == 0) vflag[y] = (unsigned char)same;
    } else {
        const int r = blockIdx.y - 1;
        const float2 *row = S + ((size_t)r * n + y) * n;
        int any = 0;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const float2 v = row[x];
            any |= (v.x != 0.f) | (v.y != 0.f);
        }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) sflag[(size_t)r * n + y] = (unsigned char)(any != 0);
    }
}

__global__ void shift_potential_kernel(int count, double eps_shift, float2 *__restrict__ V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) V[i].y = (float)((double)V[i].y - eps_shift);
}

// max over the grid of |U|, U = V + i eps_shift (the potential without the
// periodic grid's shift), in FP64: block maxima, then one atomicMax on the
// bit pattern (non-negative doubles order like their unsigned bits)
__global__ void potential_max_kernel(int count, const float2 *__restrict__ V, double eps_shift,
                                     unsigned long long *out) {
    __shared__ double wmax[8];
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double re = V[i].x, im = (double)V[i].y + eps_shift;
        m = fmax(m, sqrt(re * re + im * im));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmax(m, wmax[w]);
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
    }
}

// S[rhs][cell_k] = (sum of the amplitudes of the elements in cell k) / dx^2
__global__ void deposit_kernel(int nrhs, int nn, int n_cells, const int *__restrict__ cell,
                               const int *__restrict__ seg, const float2 *__restrict__ amp,
                               int n_pts, double inv_dx2, float2 *__restrict__ S) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (k >= n_cells) return;
    double re = 0.0, im = 0.0;
    for (int p = seg[k]; p < seg[k + 1]; p++) {
        const float2 v = amp[(size_t)rhs * n_pts + p];
        re += v.x;
        im += v.y;
    }
    S[(size_t)rhs * nn + cell[k]] = make_float2((float)(re * inv_dx2), (float)(im * inv_dx2));
}

// S2 = -(1/2) beta/(rho c^4) (2 omega)^2 psi1^2   (Eqs. 11, 28b)
__global__ void harmonic2_kernel(int nrhs, int count, const float2 *__restrict__ psi1,
                                 const float *__restrict__ beta, const float *__restrict__ rho,
                                 const float *__restrict__ c, double omega, float2 *__restrict__ S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double cc = (double)c[i] * (double)c[i];
    const double xi = (double)beta[i] / ((double)rho[i] * cc * cc);
    const double w2 = 2.0 * omega;
    const double f = -0.5 * xi * w2 * w2;
    for (int r = 0; r < nrhs; r++) {
        const float2 p = psi1[(size_t)r * count + i];
        const double re = (double)p.x * p.x - (double)p.y * p.y;
        const double im = 2.0 * (double)p.x * p.y;
        S[(size_t)r * count + i] = make_float2((float)(f * re), (float)(f * im));
    }
}

// Sum-term source of harmonic `order` (2 .. 5) from psi_1 .. psi_{order-1}
// (Eqs. 28b-28e; inputs stored divided by in.scale, output times source_scale):
//   S_n = -xi (n omega)^2 [ sum_{a<b, a+b=n} psi_a psi_b + psi_{n/2}^2 / 2 ]
__global__ void harmonic_kernel(int nrhs, int count, int order, HarmonicInputs in,
                                const float *__restrict__ beta, const float *__restrict__ rho,
                                const float *__restrict__ c, double omega, float2 *__restrict__ S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double cc = (double)c[i] * (double)c[i];
    const double xi = (double)beta[i] / ((double)rho[i] * cc * cc);
    const double wn = order * omega;
    const double f = -xi * wn * wn * in.source_scale;
    for (int r = 0; r < nrhs; r++) {
        double re = 0.0, im = 0.0;
        for (int a = 1; 2 * a <= order; a++) {
            const float2 pa = in.psi[a - 1][(size_t)r * count + i];
            const float2 pb = in.psi[order - a - 1][(size_t)r * count + i];
            const double w = ((2 * a == order) ? 0.5 : 1.0) * in.scale[a - 1] * in.scale[order - a - 1];
            re += w * ((double)pa.x * pb.x - (double)pa.y * pb.y);
            im += w * ((double)pa.x * pb.y + (double)pa.y * pb.x);
        }
        S[(size_t)r * count + i] = make_float2((float)(f * re), (float)(f * im));
    }
}

// grad = Re(sum_rhs Q * dV/dtheta), dV/dc = 2 p (-omega/c^2), dV/dalpha = 2 p (tdel + i)
__global__ void gradient_kernel(int nrhs, int count, const float2 *__restrict__ Q,
                                const float *__restrict__ c, const float *__restrict__ alpha,
                                double omega, double tdel, float *__restrict__ gc,
                                float *__restrict__ ga) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double qr = 0.0, qi = 0.0;
    for (int r = 0; r < nrhs; r++) {
        const float2 q = Q[(size_t)r * count + i];
        qr += q.x;
        qi += q.y;
    }
    const double ci = c[i];
    const double al = alpha ? (double)alpha[i] : 0.0;
    const double pr = omega / ci + al * tdel, pim = al;
    if (gc) {
        const double s = -omega / (ci * ci);
        // Re(Q * 2 p s)
        gc[i] = (float)(2.0 * s * (qr * pr - qi * pim));
    }
    if (ga) {
        // dV/dalpha = 2 p (tdel + i) = 2 (pr tdel - pim, pr + pim tdel)
        const double dr = 2.0 * (pr * tdel - pim), di = 2.0 * (pr + pim * tdel);
        ga[i] = (float)(qr * dr - qi * di);
    }
}

// ---------------------------------------------------------------------------
// dispatch over M (the per-size functions live in the tbs_inst_*.cu files)
// ---------------------------------------------------------------------------
#define TBS_EXTERN_M(MM) TBS_PER_M(extern, MM)
TBS_FOR_EACH_M(TBS_EXTERN_M)
#undef TBS_EXTERN_M

cudaError_t launch_row(int kind, int M, int nrhs, const RowArgs &a, cudaStream_t s) {
#define TBS_CASE(MM) \
    case MM: return launch_row_m<MM>(kind, nrhs, a, s);
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return cudaErrorInvalidValue;
}

int col_variants(int M, bool periodic) { return periodic ? col_periodic_variant_count(M) : col_variant_count(M); }

const char *col_variant_name(int M, bool periodic, int variant) {
    if (variant < 0 || variant >= col_variants(M, periodic)) return nullptr;
    if (periodic) {
        if (col_variants(M, true) == 1) return "periodic, lockstep, 1 column/thread";
        static const char *names[4] = {"periodic, lockstep, 2 columns/thread", "periodic, lockstep, 1 column/thread",
                                       "periodic, pipelined, 2 columns/thread",
                                       "periodic, pipelined, 2 columns/thread, staggered"};
        return names[variant];
    }
    switch (col_variant_kind(M, variant)) {
    case COL_S0: return "tile S0 (lockstep, default width)";
    case COL_S1: return "tile S1 (lockstep, width/2)";
    case COL_S2: return "tile S2 (lockstep, width/4)";
    case COL_P1: return "pipelined, 1 column/thread";
    case COL_P2: return "pipelined, 2 columns/thread";
    case COL_P2S: return "pipelined, 2 columns/thread, staggered";
    case COL_P2R8: return "pipelined, 2 columns/thread, radix 8x8x8x8";
    }
    return nullptr;
}

cudaError_t col_tensor_maps(ColMaps *maps, const float2 *X, const float2 *W, int n, int M, int nrhs, int variant,
                            bool periodic) {
#define TBS_CASE(MM) \
    case MM: return col_tensor_maps_m<MM>(maps, X, W, n, nrhs, variant, periodic);
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_col(int M, int nrhs, bool cj, const ColArgs &a, const ColMaps *maps, int variant,
                       cudaStream_t s) {
#define TBS_CASE(MM) \
    case MM: return launch_col_m<MM>(nrhs, cj, a, maps, variant, s);
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return cudaErrorInvalidValue;
}

int col_resident_blocks_per_sm(int M, int variant, bool periodic) {
#define TBS_CASE(MM) \
    case MM: return col_resident_blocks_m<MM>(variant, periodic);
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return 1;
}

cudaError_t set_col_smem_attr(int M) {
#define TBS_CASE(MM) \
    case MM: return set_col_smem_attr_m<MM>();
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t set_row_smem_attr(int M) {
#define TBS_CASE(MM) \
    case MM: return set_row_smem_attr_m<MM>();
    switch (M) { TBS_FOR_EACH_M(TBS_CASE) }
#undef TBS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_stop(int nrhs, const StopArgs &a, cudaStream_t s) {
    return launch_k(stop_kernel, dim3(nrhs), dim3(256), 0, s, a.pdl != 0, a);
}

cudaError_t launch_adj_loop(int nrhs, const RhsState *st, int *j, cudaGraphConditionalHandle h, bool init,
                            cudaStream_t s) {
    adj_loop_kernel<<<1, 1, 0, s>>>(nrhs, st, j, h, init ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_info(int nrhs, const RhsState *st, const int *err, void *info_dev, cudaStream_t s) {
    info_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(nrhs, st, err, (InfoOut *)info_dev);
    return cudaGetLastError();
}

cudaError_t launch_medium(int count, const float *c, const float *alpha, double omega, double c0,
                          double tdel, double eps_shift, float2 *V, cudaStream_t s) {
    medium_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, c, alpha, (float)omega, (float)(omega / c0), (float)c0,
                                                      (float)tdel, (float)eps_shift, V);
    return cudaGetLastError();
}

cudaError_t launch_row_flags(int n, int nrhs, const float2 *V, const float2 *S, unsigned char *vflag,
                             unsigned char *sflag, cudaStream_t s) {
    row_flags_kernel<<<dim3(n, 1 + nrhs), 256, 0, s>>>(n, V, S, vflag, sflag);
    return cudaGetLastError();
}

cudaError_t launch_potential_max(int count, const float2 *V, double eps_shift, unsigned long long *out,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(*out), s);
    if (e != cudaSuccess) return e;
    int blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    potential_max_kernel<<<blocks, 256, 0, s>>>(count, V, eps_shift, out);
    return cudaGetLastError();
}

cudaError_t launch_shift_potential(int count, double eps_shift, float2 *V, cudaStream_t s) {
    shift_potential_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, eps_shift, V);
    return cudaGetLastError();
}

cudaError_t launch_deposit(int nrhs, int n, int n_cells, const int *cell, const int *seg,
                           const float2 *amp_sorted, int n_pts, double inv_dx2, float2 *S,
                           cudaStream_t s) {
    if (n_cells == 0) return cudaSuccess;
    dim3 grid((n_cells + 127) / 128, nrhs);
    deposit_kernel<<<grid, 128, 0, s>>>(nrhs, n * n, n_cells, cell, seg, amp_sorted, n_pts, inv_dx2, S);
    return cudaGetLastError();
}

cudaError_t launch_harmonic2(int nrhs, int count, const float2 *psi1, const float *beta,
                             const float *rho, const float *c, double omega, float2 *S,
                             cudaStream_t s) {
    harmonic2_kernel<<<(count + 255) / 256, 256, 0, s>>>(nrhs, count, psi1, beta, rho, c, omega, S);
    return cudaGetLastError();
}

cudaError_t launch_harmonic(int nrhs, int count, int order, const HarmonicInputs &in, const float *beta,
                            const float *rho, const float *c, double omega, float2 *S, cudaStream_t s) {
    harmonic_kernel<<<(count + 255) / 256, 256, 0, s>>>(nrhs, count, order, in, beta, rho, c, omega, S);
    return cudaGetLastError();
}

cudaError_t launch_gradient(int nrhs, int count, const float2 *Q, const float *c,
                            const float *alpha, double omega, double tdel, float *grad_c,
                            float *grad_alpha, cudaStream_t s) {
    gradient_kernel<<<(count + 255) / 256, 256, 0, s>>>(nrhs, count, Q, c, alpha, omega, tdel,
                                                        grad_c, grad_alpha);
    return cudaGetLastError();
}

}  // namespace tbs
