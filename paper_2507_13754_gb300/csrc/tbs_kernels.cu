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
#include "tbs_fft.cuh"
#include "tbs_internal.h"

#include <math.h>

namespace tbs {

// ---------------------------------------------------------------------------
// configurations
// ---------------------------------------------------------------------------
template <int M>
struct RowCfg {
    static constexpr int E = 16;
    static constexpr int T = M / E;
    static constexpr int RPB = T >= 256 ? 1 : 256 / T;  // rows per block
    static constexpr int THREADS = T * RPB;               // 256
    static constexpr int LINE = padded_len(M);
    static constexpr size_t SMEM = (size_t)RPB * LINE * sizeof(float2);
};

template <int M>
struct ColCfg {
    static constexpr int TC = M >= 4096 ? 4 : M >= 2048 ? 8 : 16;  // columns per block
    static constexpr int L = 2;                                    // columns per thread
    static constexpr int E = 16;
    static constexpr int T = M / E;
    static constexpr int THREADS = T * (TC / L);
    static constexpr size_t SMEM = (size_t)padded_len(M) * TC * sizeof(float2);
};

int col_tile(int M) {
    return M >= 4096 ? 4 : M >= 2048 ? 8 : 16;
}

__device__ __forceinline__ bool gate_active(const Gate &g, int rhs) {
    if (g.mode == GATE_FWD) return g.st[rhs].done == 0;
    if (g.mode == GATE_ADJ) return g.j <= g.st[rhs].terms - 2;
    return true;
}

__device__ __forceinline__ double abs2d(float2 a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// Sum over the T threads of one row (rows are T-aligned lane groups of a
// 256-thread block).  Fixed shuffle-butterfly order, then a fixed-order sum of
// the per-warp results: deterministic.  Result valid in the row's thread 0.
template <int T>
__device__ __forceinline__ double row_sum(double v, double *red, int lr) {
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int o = W / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if constexpr (T > 32) {
        constexpr int WPR = T / 32;  // warps per row
        const int lane = threadIdx.x & 31;
        const int warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double s = 0.0;
        if ((threadIdx.x % T) == 0) {
#pragma unroll
            for (int w = 0; w < WPR; w++) s += red[lr * WPR + w];
        }
        return s;
    } else {
        return v;
    }
}

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------
template <int M, int KIND>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
row_kernel(RowArgs a) {
    using C = RowCfg<M>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ double red[4][8];
    const int rhs = blockIdx.y;
    if (!gate_active(a.gate, rhs)) return;
    const int lr = threadIdx.x / T;
    const int t = threadIdx.x % T;
    const int n = a.n;
    const int y = blockIdx.x * C::RPB + lr;
    const bool valid = y < n;
    const size_t nn = (size_t)n * n;
    const size_t row_sp = (size_t)rhs * nn + (size_t)y * n;  // spatial row offset
    const Lines<1> sm{smem + lr * C::LINE, 1};
    float2 va[1][E];
    float2 (&v)[E] = va[0];

    if constexpr (KIND == ROW_SRC) {
        const float2 *s = a.src + row_sp;
#pragma unroll
        for (int m = 0; m < E; m++) {
            const int x = t + T * m;
            v[m] = (m < E / 2 && valid && x < n) ? s[x] : make_float2(0.f, 0.f);
        }
    } else {
        const float2 *w = a.W + ((size_t)rhs * n + (valid ? y : 0)) * M;
#pragma unroll
        for (int m = 0; m < E; m++) v[m] = valid ? w[t + T * m] : make_float2(0.f, 0.f);
        fft_lines<M, E, +1, 1>(va, sm, t, a.tw);

        if constexpr (KIND == ROW_FWD || KIND == ROW_FWD_LAST) {
            double su = 0.0, sp = 0.0, lu = 0.0, lp = 0.0;
            const bool first = (a.term == 0);
            float2 *U = a.U ? a.U + ((size_t)rhs * a.max_terms + a.term) * nn + (size_t)y * n : nullptr;
#pragma unroll
            for (int m = 0; m < E; m++) {
                const int x = t + T * m;
                if (m < E / 2 && valid && x < n) {
                    const float2 u = v[m];
                    const float2 pold = first ? make_float2(0.f, 0.f) : a.psi[row_sp + x];
                    const float2 p = cadd(pold, u);
                    a.psi[row_sp + x] = p;
                    if (U) U[x] = u;
                    su += abs2d(u);
                    sp += abs2d(p);
                    lu += sqrt(abs2d(u));
                    lp += sqrt(abs2d(pold));
                    v[m] = cmul(a.V[(size_t)y * n + x], u);
                } else {
                    v[m] = make_float2(0.f, 0.f);
                }
            }
            su = row_sum<T>(su, red[0], lr);
            sp = row_sum<T>(sp, red[1], lr);
            const int r0 = blockIdx.x * C::RPB;
            const bool has_l1 = a.l1_row >= r0 && a.l1_row < r0 + C::RPB;  // block-uniform
            if (has_l1) {
                lu = row_sum<T>(lu, red[2], lr);
                lp = row_sum<T>(lp, red[3], lr);
            }
            if (t == 0 && valid) {
                a.part[(size_t)rhs * n + y] = make_double2(su, sp);
                if (y == a.l1_row) a.l1[rhs] = make_double2(lu, lp);
            }
        } else if constexpr (KIND == ROW_ADJ || KIND == ROW_ADJ_LAST) {
            const float2 *Uj = a.U + ((size_t)rhs * a.max_terms + a.term) * nn + (size_t)y * n;
#pragma unroll
            for (int m = 0; m < E; m++) {
                const int x = t + T * m;
                if (m < E / 2 && valid && x < n) {
                    const float2 lam = v[m];
                    float2 q = a.Q[row_sp + x];
                    q = cadd(q, cmulc(Uj[x], lam));  // conj(lambda) u_j
                    a.Q[row_sp + x] = q;
                    // ubar_j = g + conj(V) lambda
                    v[m] = cadd(a.src[row_sp + x], cmulc(lam, a.V[(size_t)y * n + x]));
                } else {
                    v[m] = make_float2(0.f, 0.f);
                }
            }
        } else if constexpr (KIND == ROW_OUT) {
#pragma unroll
            for (int m = 0; m < E / 2; m++) {
                const int x = t + T * m;
                if (valid && x < n) a.psi[row_sp + x] = v[m];
            }
        }
    }

    if constexpr (KIND == ROW_SRC || KIND == ROW_FWD || KIND == ROW_ADJ) {
        fft_lines<M, E, -1, 1>(va, sm, t, a.tw);
        if (valid) {
            float2 *xo = a.X + ((size_t)rhs * n + y) * M;
#pragma unroll
            for (int m = 0; m < E; m++) xo[t + T * m] = v[m];
        }
    }
}

// ---------------------------------------------------------------------------
// column pass
// ---------------------------------------------------------------------------
template <int M, bool CONJ>
__global__ void __launch_bounds__(ColCfg<M>::THREADS)
col_kernel(ColArgs a) {
    using C = ColCfg<M>;
    constexpr int E = C::E, T = C::T, TC = C::TC, L = C::L, G = TC / L;
    extern __shared__ __align__(16) float2 smem[];
    const int rhs = blockIdx.y;
    if (!gate_active(a.gate, rhs)) return;
    const int cg = threadIdx.x % G;  // column pair within the tile
    const int t = threadIdx.x / G;
    const int kx = blockIdx.x * TC + L * cg;  // first of this thread's two columns
    const int n = a.n;
    const float2 *X = a.X + (size_t)rhs * n * M;
    const Lines<L> sm{smem + L * cg, TC};
    float2 v[L][E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int ky = t + T * m;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < E / 2 && ky < n) f = *reinterpret_cast<const float4 *>(X + (size_t)ky * M + kx);
        v[0][m] = make_float2(f.x, f.y);
        v[1][m] = make_float2(f.z, f.w);
    }
    fft_lines<M, E, -1, L>(v, sm, t, a.tw);
    constexpr int QS = M / 2 + 1;
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int kxl = kx + l;
        const int kxq = kxl <= M / 2 ? kxl : M - kxl;
#pragma unroll
        for (int m = 0; m < E; m++) {
            const int ky = t + T * m;
            const int kyq = ky <= M / 2 ? ky : M - ky;
            const float2 g = __ldg(a.ghq + (size_t)kyq * QS + kxq);
            v[l][m] = CONJ ? cmulc(v[l][m], g) : cmul(v[l][m], g);
        }
    }
    fft_lines<M, E, +1, L>(v, sm, t, a.tw);
    float2 *W = a.W + (size_t)rhs * n * M;
#pragma unroll
    for (int m = 0; m < E / 2; m++) {
        const int y = t + T * m;
        if (y < n)
            *reinterpret_cast<float4 *>(W + (size_t)y * M + kx) =
                make_float4(v[0][m].x, v[0][m].y, v[1][m].x, v[1][m].y);
    }
}

// ---------------------------------------------------------------------------
// stop test: FP64 reduction of the row partials, residual, divergence, flags
// (Eq. 30 for the L1 row mode; full-grid L2 otherwise)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) stop_kernel(StopArgs a) {
    const int rhs = blockIdx.x;
    RhsState *s = a.st + rhs;
    if (s->done) return;
    __shared__ double ru[256], rp[256];
    double su = 0.0, sp = 0.0;
    const double2 *part = a.part + (size_t)rhs * a.n;
    for (int y = threadIdx.x; y < a.n; y += 256) {
        su += part[y].x;
        sp += part[y].y;
    }
    ru[threadIdx.x] = su;
    rp[threadIdx.x] = sp;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if (threadIdx.x < o) {
            ru[threadIdx.x] += ru[threadIdx.x + o];
            rp[threadIdx.x] += rp[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double un = sqrt(ru[0]), pn = sqrt(rp[0]);
    const int term = a.term;
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

struct InfoOut {  // layout of tbs_solve_info
    int32_t terms;
    int32_t status;
    double residual;
    double term_norm_max;
    double psi_norm;
};

__global__ void info_kernel(int nrhs, const RhsState *st, InfoOut *out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    out[r].terms = st[r].terms;
    out[r].status = st[r].status;
    out[r].residual = st[r].residual;
    out[r].term_norm_max = st[r].tmax;
    out[r].psi_norm = st[r].psi_norm;
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------

// V = p^2 - k0^2, p = omega/c + alpha (tdel + i), tdel = tan(pi y/2) delta
__global__ void medium_kernel(int count, const float *__restrict__ c, const float *__restrict__ alpha,
                              double omega, double k0, double tdel, float2 *__restrict__ V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double al = alpha ? (double)alpha[i] : 0.0;
    const double pr = omega / (double)c[i] + al * tdel;
    const double pi_ = al;
    V[i] = make_float2((float)(pr * pr - pi_ * pi_ - k0 * k0), (float)(2.0 * pr * pi_));
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
// launchers
// ---------------------------------------------------------------------------
template <int M, int KIND>
static cudaError_t row_launch(int nrhs, const RowArgs &a, cudaStream_t s) {
    using C = RowCfg<M>;
    dim3 grid((a.n + C::RPB - 1) / C::RPB, nrhs);
    row_kernel<M, KIND><<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int M>
static cudaError_t row_dispatch_kind(int kind, int nrhs, const RowArgs &a, cudaStream_t s) {
    switch (kind) {
    case ROW_SRC: return row_launch<M, ROW_SRC>(nrhs, a, s);
    case ROW_FWD: return row_launch<M, ROW_FWD>(nrhs, a, s);
    case ROW_FWD_LAST: return row_launch<M, ROW_FWD_LAST>(nrhs, a, s);
    case ROW_ADJ: return row_launch<M, ROW_ADJ>(nrhs, a, s);
    case ROW_ADJ_LAST: return row_launch<M, ROW_ADJ_LAST>(nrhs, a, s);
    case ROW_OUT: return row_launch<M, ROW_OUT>(nrhs, a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_row(int kind, int M, int nrhs, const RowArgs &a, cudaStream_t s) {
    switch (M) {
    case 16: return row_dispatch_kind<16>(kind, nrhs, a, s);
    case 32: return row_dispatch_kind<32>(kind, nrhs, a, s);
    case 64: return row_dispatch_kind<64>(kind, nrhs, a, s);
    case 128: return row_dispatch_kind<128>(kind, nrhs, a, s);
    case 256: return row_dispatch_kind<256>(kind, nrhs, a, s);
    case 512: return row_dispatch_kind<512>(kind, nrhs, a, s);
    case 1024: return row_dispatch_kind<1024>(kind, nrhs, a, s);
    case 2048: return row_dispatch_kind<2048>(kind, nrhs, a, s);
    case 4096: return row_dispatch_kind<4096>(kind, nrhs, a, s);
    }
    return cudaErrorInvalidValue;
}

template <int M, bool CONJ>
static cudaError_t col_launch(int nrhs, const ColArgs &a, cudaStream_t s) {
    using C = ColCfg<M>;
    dim3 grid(M / C::TC, nrhs);
    col_kernel<M, CONJ><<<grid, C::THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_col(int M, int nrhs, bool cj, const ColArgs &a, cudaStream_t s) {
#define TBS_COL_CASE(MM) \
    case MM: return cj ? col_launch<MM, true>(nrhs, a, s) : col_launch<MM, false>(nrhs, a, s);
    switch (M) {
        TBS_COL_CASE(16)
        TBS_COL_CASE(32)
        TBS_COL_CASE(64)
        TBS_COL_CASE(128)
        TBS_COL_CASE(256)
        TBS_COL_CASE(512)
        TBS_COL_CASE(1024)
        TBS_COL_CASE(2048)
        TBS_COL_CASE(4096)
    }
#undef TBS_COL_CASE
    return cudaErrorInvalidValue;
}

template <int M>
static cudaError_t col_attr() {
    using C = ColCfg<M>;
    cudaError_t e = cudaFuncSetAttribute(col_kernel<M, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(col_kernel<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM);
}

cudaError_t set_col_smem_attr(int M) {
    switch (M) {
    case 16: return col_attr<16>();
    case 32: return col_attr<32>();
    case 64: return col_attr<64>();
    case 128: return col_attr<128>();
    case 256: return col_attr<256>();
    case 512: return col_attr<512>();
    case 1024: return col_attr<1024>();
    case 2048: return col_attr<2048>();
    case 4096: return col_attr<4096>();
    }
    return cudaErrorInvalidValue;
}

template <int M>
static cudaError_t row_attr() {
    using C = RowCfg<M>;
    const int b = (int)C::SMEM;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_FWD_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_ADJ_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    return cudaFuncSetAttribute(row_kernel<M, ROW_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

cudaError_t set_row_smem_attr(int M) {
    switch (M) {
    case 16: return row_attr<16>();
    case 32: return row_attr<32>();
    case 64: return row_attr<64>();
    case 128: return row_attr<128>();
    case 256: return row_attr<256>();
    case 512: return row_attr<512>();
    case 1024: return row_attr<1024>();
    case 2048: return row_attr<2048>();
    case 4096: return row_attr<4096>();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stop(int nrhs, const StopArgs &a, cudaStream_t s) {
    stop_kernel<<<nrhs, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_info(int nrhs, const RhsState *st, void *info_dev, cudaStream_t s) {
    info_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(nrhs, st, (InfoOut *)info_dev);
    return cudaGetLastError();
}

cudaError_t launch_medium(int count, const float *c, const float *alpha, double omega, double k0,
                          double tdel, float2 *V, cudaStream_t s) {
    medium_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, c, alpha, omega, k0, tdel, V);
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

cudaError_t launch_gradient(int nrhs, int count, const float2 *Q, const float *c,
                            const float *alpha, double omega, double tdel, float *grad_c,
                            float *grad_alpha, cudaStream_t s) {
    gradient_kernel<<<(count + 255) / 256, 256, 0, s>>>(nrhs, count, Q, c, alpha, omega, tdel,
                                                        grad_c, grad_alpha);
    return cudaGetLastError();
}

}  // namespace tbs
