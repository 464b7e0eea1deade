// tbs_kernels.cuh -- the per-term kernels of the Born series as templates
// over the padded size M (row pass, column pass and their launchers).
// Included by tbs_kernels.cu (dispatch) and the tbs_inst_*.cu files, which
// instantiate the sizes.
#pragma once
#include "tbs_fft.cuh"
#include "tbs_internal.h"
#include "tbs_tma.cuh"

#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <type_traits>
#include <utility>

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
    static constexpr int LINE = (padded_len(M) + 1) & ~1;  // FFT exchange line, 16-byte multiple
    static constexpr int HALF = M / 2;                    // >= N: psi / V row buffers
    // per row: the exchange line (the W row lands there unpadded first), then
    // the prefetched psi and V rows
    static constexpr int ROWSTRIDE = LINE + 2 * HALF;
    static constexpr size_t SMEM = (size_t)RPB * ROWSTRIDE * sizeof(float2);
    // every row's buffers start 16-byte aligned (16-byte cp.async targets)
    static_assert(LINE % 2 == 0 && ROWSTRIDE % 2 == 0, "row buffers must be 16-byte aligned");
};

// Column-pass shape: TC columns per tile, L columns per thread, E elements per
// column per thread; MINB resident blocks per SM targeted by the register
// budget.  PER_: 1 for the periodic grid (all M rows are grid points, the
// spectrum is formed in the kernel, no Ghat columns are copied), 2 for the
// periodic grid with the k-space potential (a kernel of its own, so that the
// plain periodic pass keeps its code size).
template <int M, int TC_, int L_, int MINB_ = 1, int PER_ = 0>
struct ColShape {
    static constexpr bool PIPE = false;  // col_kernel (ColPShape: col_pipe_kernel)
    static constexpr int MINB = MINB_;
    static constexpr int TC = TC_;
    static constexpr int L = L_;
    static constexpr bool PER = PER_ != 0;
    static constexpr bool KS = PER_ == 2;
    static constexpr int E = 16;
    static constexpr int T = M / E;
    static constexpr int THREADS = T * (TC / L);
    // BLOCKED: column group cg is threads [cg T, (cg + 1) T) and syncs its
    // transforms with its own named barrier (two groups, whole warps each);
    // otherwise the groups interleave thread by thread (cg = thread % G, for
    // conflict-free reads of the [row][TC] landing rows when TC > 2) and
    // sync the whole block.
    static constexpr bool BLOCKED = (TC / L == 2) && T >= 32;
    static constexpr int HALF = M / 2;  // >= N rows of input
    // exchange lines: one padded line per column.  Lanes of a warp that
    // differ in their column group access lines L apart; a line stride of
    // 8/L float2 past a multiple of 16 puts those lines 16 banks apart.
    static constexpr int LSTRIDE = ((padded_len(M) + 15) / 16) * 16 + 8 / L_;
    // two stages (this tile, next tile), each holding the input rows
    // [HALF][TC] (later the output rows) and the Ghat columns [TC][QSP]
    static constexpr size_t LAND = (size_t)(PER ? M : HALF) * TC;
    static constexpr int QSP = ghat_stride(M);  // stored quadrant row stride
    static constexpr size_t GBUF = PER ? 0 : (size_t)QSP * TC;
    // stages start 128-byte aligned (tensor-copy destinations)
    static constexpr size_t STAGE = (LAND + GBUF + 15) & ~(size_t)15;
    static_assert(LAND % 16 == 0, "landing buffer keeps boxes 128-byte aligned");
    static constexpr int BR = HALF < 256 ? HALF : 256;  // rows per tensor-copy box
    // + 128 bytes: the kernel rounds its dynamic shared base up to 128 bytes
    static constexpr size_t SMEM = (2 * STAGE + (size_t)LSTRIDE * TC) * sizeof(float2) + 128;
    static_assert(LAND % 2 == 0 && (TC % 2 == 0 || TC == 1) && TC % L == 0, "16-byte aligned rows");
};

template <int M>
using ColCfg = ColShape<M, (M >= 4096 ? 2 : M >= 2048 ? 4 : 8), 1>;
template <int M>
using ColCfgP = ColShape<M, ColCfg<M>::TC, 1, 1, 1>;
template <int M>
using ColCfgPK = ColShape<M, ColCfg<M>::TC, 1, 1, 2>;
// periodic grid, two columns per thread (M >= 32: a tile of >= 2 columns)
template <int M>
using ColCfgP2 = ColShape<M, ColCfg<M>::TC, 2, 1, 1>;
template <int M>
using ColCfgPK2 = ColShape<M, ColCfg<M>::TC, 2, 1, 2>;
// periodic plans: lockstep with two columns per thread (M >= 32) and one
// plus, for M >= 1024, the pipelined kernel with two columns per thread
// (unstaggered, staggered)
__host__ __device__ constexpr int col_periodic_variant_count(int M) { return M >= 1024 ? 4 : M >= 32 ? 2 : 1; }

// Autotuned alternatives: variant V narrows the tile to TC >> V columns (one
// column per thread), so blocks get smaller and more of them are resident
// per SM.  Tensor-copy boxes need >= 16-byte rows, hence TC >= 2; variants
// are compiled for M >= 512.
template <int M, int V>
struct ColVariant {
    static constexpr int TC = ColCfg<M>::TC >> V;
    static constexpr int THREADS = (M / 16) * (TC > 0 ? TC : 1);
    static constexpr int MINB = THREADS >= 512 ? 1 : 65536 / (THREADS * 128);
    using type = ColShape<M, (TC >= 2 ? TC : 2), 1, MINB>;
};

// tile shapes of col_kernel: variants v with (default TC >> v) >= 2
__host__ __device__ constexpr int col_shape_count(int M) {
    return M < 512 ? 1 : (M >= 4096 ? 1 : M >= 2048 ? 2 : 3);
}
// the pipelined kernel exists for M >= 1024
__host__ __device__ constexpr bool col_has_pipe(int M) { return M >= 1024; }
// For M >= 1024 there is also the pipelined kernel with one or two columns
// per thread (P1, P2; P2S: the two columns staggered).
// At M = 4096 also the unstaggered pair with the radix split 8 x 8 x 8 x 8 (P2R8).
__host__ __device__ constexpr int col_variant_count(int M) {
    return col_shape_count(M) + (col_has_pipe(M) ? 3 : 0) + (M >= 4096 ? 1 : 0);
}
// The variants of each M, fastest first as measured on GB300 at N = M/2
// (variant 0 is a plan's default; tbs_autotune re-times them all):
// S0 = col_kernel's default tile, S1/S2 = its tile narrowed once/twice.
enum ColKind { COL_S0 = 0, COL_S1 = 1, COL_S2 = 2, COL_P1 = 3, COL_P2 = 4, COL_P2S = 5, COL_P2R8 = 6 };
__host__ __device__ constexpr int col_variant_kind(int M, int v) {
    if (M >= 4096) {
        constexpr int k[5] = {COL_P2, COL_P2S, COL_P1, COL_S0, COL_P2R8};
        return k[v];
    }
    if (M == 2048) {
        constexpr int k[5] = {COL_S1, COL_P2S, COL_P2, COL_P1, COL_S0};
        return k[v];
    }
    if (M == 1024) {
        constexpr int k[6] = {COL_S2, COL_S1, COL_P2S, COL_P2, COL_P1, COL_S0};
        return k[v];
    }
    return v;  // S0, S1, S2 in order
}
static_assert(col_variant_count(1024) <= MAX_COL_VARIANTS && col_variant_count(512) <= MAX_COL_VARIANTS &&
                  col_periodic_variant_count(4096) <= MAX_COL_VARIANTS,
              "per-variant plan arrays hold every variant");


// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor drains; grid_dep_wait()
// returns once the predecessor has completed and its writes are visible (at
// once for an ordinary launch).  Everything before it touches only data no
// kernel of the term loop writes (twiddles, parameters, shared memory).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// lets the dependent grid be scheduled once every block has passed this point
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// cudaLaunchKernelEx with programmatic stream serialization when pdl is set
template <typename... P, typename... A>
static cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                            A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

__device__ __forceinline__ bool gate_active(const Gate &g, int rhs) {
    if (g.mode == GATE_FWD) return g.st[rhs].done == 0;
    if (g.mode == GATE_ADJ) return (g.j >= 0 ? g.j : *g.jdev) <= g.st[rhs].terms - 2;
    return true;
}

// Double-float (hi + lo) sums: Knuth's TwoSum keeps each fp32 addition exact,
// so a warp reduction in fp32 pairs carries ~2 x 24 significant bits -- as
// good as FP64 for these norms -- while running on the FP32 pipes (GB300's
// FP64 rate is a small fraction of its FP32 rate).
struct DFloat {
    float hi, lo;
};

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    const float e = (a.hi - (s - v)) + (b.hi - v);
    const float lo = a.lo + b.lo + e;
    const float hi = s + lo;
    return DFloat{hi, lo - (hi - s)};
}

// Sums of K values over the T threads of one row (rows are T-aligned lane
// groups of a 256-thread block).  Fixed shuffle-butterfly order in
// double-float within each warp, then across the row's warps by its first
// warp (also double-float, fixed order): deterministic, and one FP64
// conversion per result.  Results valid in the row's thread 0.  red[k] is
// used once per launch (no barrier guards its reuse).
template <int T, int K>
__device__ __forceinline__ void row_sums(const float (&x)[K], double (&out)[K], float2 (*red)[8], int lr) {
    constexpr int W = T < 32 ? T : 32;
    DFloat v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = DFloat{x[k], 0.f};
#pragma unroll
    for (int o = W / 2; o >= 1; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            const DFloat u{__shfl_xor_sync(0xffffffffu, v[k].hi, o), __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
            v[k] = df_add(v[k], u);
        }
    }
    if constexpr (T > 32) {
        constexpr int WPR = T / 32;  // warps per row
        const int lane = threadIdx.x & 31;
        const int warp = threadIdx.x >> 5;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) red[k][warp] = make_float2(v[k].hi, v[k].lo);
        }
        __syncthreads();
        if (warp == lr * WPR) {  // the row's first warp; its lane 0 is the row's thread 0
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float2 r = lane < WPR ? red[k][lr * WPR + lane] : make_float2(0.f, 0.f);
                v[k] = DFloat{r.x, r.y};
            }
#pragma unroll
            for (int o = WPR / 2; o >= 1; o >>= 1) {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const DFloat u{__shfl_xor_sync(0xffffffffu, v[k].hi, o), __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
                    v[k] = df_add(v[k], u);
                }
            }
#pragma unroll
            for (int k = 0; k < K; k++) out[k] = (double)v[k].hi + (double)v[k].lo;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) out[k] = (double)v[k].hi + (double)v[k].lo;
    }
}

// Optional phase timers for experiments (compiled out unless defined).
#ifndef TBS_ROW_PHASE
#define TBS_ROW_PHASE_DECL
#define TBS_ROW_PHASE(k)
#define TBS_ROW_PHASE_END
#endif

// ---------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------
template <int M, int KIND>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 2)
row_kernel(RowArgs a) {
    using C = RowCfg<M>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float2 red[4][8];
    const int rhs = blockIdx.y;
    const int lr = threadIdx.x / T;
    const int t = threadIdx.x % T;
    const int n = a.n;
    const int y = blockIdx.x * C::RPB + lr;
    const bool valid = y < n;
    const size_t nn = (size_t)n * n;
    const size_t row_sp = (size_t)rhs * nn + (size_t)y * n;  // spatial row offset
    float2 *line = smem + lr * C::ROWSTRIDE;
    float2 *psi_s = line + C::LINE;
    float2 *v_s = psi_s + C::HALF;
    const Lines<1> sm{line, 0};
    float2 va[1][E];
    float2 (&v)[E] = va[0];
    constexpr bool PREFETCH = (KIND == ROW_FWD);
    // The W, psi and V rows of the steady-state pass are prefetched into
    // shared memory: for even N (every row 16-byte aligned) by three bulk
    // copies per row, issued by the row's thread 0 and completing on two
    // barriers (bar[lr][0]: W, bar[lr][1]: psi and V) -- they bypass L1 and
    // every thread waits on the barrier itself; for odd N by cp.async from
    // every thread (W then needs a block barrier).
    __shared__ __align__(8) uint64_t rbar[PREFETCH ? C::RPB : 1][2];
    const bool bulk = PREFETCH && (n & 1) == 0;
    if (bulk && t == 0) {
        mbar_init(&rbar[lr][0], 1);
        mbar_init(&rbar[lr][1], 1);
        mbar_init_fence();
    }
    ThreadTwiddles<M, E> twr;  // shared by the inverse and the forward transform
    twr.load(a.tw, t);
    if (bulk) __syncthreads();  // the barriers are initialised before anyone waits
    grid_dep_wait();
    if constexpr (PREFETCH) {
        // Start the row copies first so that their latency overlaps the flag
        // load below; a stopped RHS waits for them before leaving.  The psi
        // row is fetched even for the first term (whose psi_0 is zero and the
        // fetched values unused), so that no copy waits on the term index.
        const float2 *w = a.W + ((size_t)rhs * n + (valid ? y : 0)) * M;
        if (bulk) {
            if (t == 0 && valid) {
                mbar_arrive_expect_tx(&rbar[lr][0], (unsigned)(M * sizeof(float2)));
                bulk_load(line, w, (unsigned)(M * sizeof(float2)), &rbar[lr][0]);
                mbar_arrive_expect_tx(&rbar[lr][1], (unsigned)(2 * n * sizeof(float2)));
                bulk_load(psi_s, a.psi + row_sp, (unsigned)(n * sizeof(float2)), &rbar[lr][1]);
                bulk_load(v_s, a.V + (size_t)y * n, (unsigned)(n * sizeof(float2)), &rbar[lr][1]);
            }
        } else {
            if (valid) {
#pragma unroll
                for (int m = 0; m < E / 2; m++) cp_async16(line + 2 * (t + T * m), w + 2 * (t + T * m));
            }
            cp_async_commit();
            if (valid) {
                for (int x = t; x < n; x += T) {
                    cp_async8(psi_s + x, a.psi + row_sp + x);
                    cp_async8(v_s + x, a.V + (size_t)y * n + x);
                }
            }
            cp_async_commit();
        }
    }
    grid_dep_launch();  // the stop test may be scheduled once every row block runs
    TBS_ROW_PHASE_DECL
    if (!gate_active(a.gate, rhs)) {
        if (bulk) {
            if (t == 0 && valid) {  // the copies must land before the block leaves
                mbar_wait_bounded(&rbar[lr][0], 0, a.wait_ns, a.err);
                mbar_wait_bounded(&rbar[lr][1], 0, a.wait_ns, a.err);
            }
        } else {
            cp_async_wait<0>();
        }
        return;
    }
    // forward term index (given, or this RHS's count of terms summed so far)
    // or adjoint step j (given, or the graph loop's counter)
    const int term = a.term >= 0                          ? a.term
                     : (KIND == ROW_FWD || KIND == ROW_EPS || KIND == ROW_EPSK) ? a.gate.st[rhs].terms
                     : KIND == ROW_ADJ                      ? *a.gate.jdev
                                                            : 0;
    TBS_ROW_PHASE(0)

    // a periodic grid (N = M) has no zero padding: every element is a grid point
    const bool full = n > M / 2;
    if constexpr (KIND == ROW_SRC || KIND == ROW_VSRC) {
        const float2 *s = a.src + row_sp;
#pragma unroll
        for (int m = 0; m < E; m++) {
            const int x = t + T * m;
            const bool in = (m < E / 2 || full) && valid && x < n;
            v[m] = in ? s[x] : make_float2(0.f, 0.f);
            // ROW_VSRC: the input of the next term, V u_j (as the steady pass forms it)
            if constexpr (KIND == ROW_VSRC)
                if (in) v[m] = cmul(a.V[(size_t)y * n + x], v[m]);
        }
    } else {
        const float2 *w = a.W + ((size_t)rhs * n + (valid ? y : 0)) * M;
        if constexpr (PREFETCH) {
            // the W row went to the (unpadded) exchange line, the psi and V
            // rows to their buffers: wait for W only
            if (bulk) {
                if (valid) mbar_wait_bounded(&rbar[lr][0], 0, a.wait_ns, a.err);
            } else {
                cp_async_wait<1>();
                __syncthreads();
            }
            TBS_ROW_PHASE(1)
#pragma unroll
            for (int m = 0; m < E; m++) v[m] = valid ? line[t + T * m] : make_float2(0.f, 0.f);
        } else {
#pragma unroll
            for (int m = 0; m < E; m++) v[m] = valid ? w[t + T * m] : make_float2(0.f, 0.f);
        }
        fft_lines<M, E, +1, 1>(va, sm, t, a.tw, &twr);

        if constexpr (KIND == ROW_FWD) {
            // Squares are summed in fp32 over the <= E/2 elements of a thread,
            // then across the row in double-float pairs and across warps and
            // rows in FP64 (GB300's FP64 rate is a small fraction of its FP32
            // rate, so no FP64 per element).
            float su_f = 0.f, sp_f = 0.f, lu_f = 0.f, lp_f = 0.f;
            const bool first = (term == 0);
            const int r0 = blockIdx.x * C::RPB;
            const bool has_l1 = a.l1_row >= r0 && a.l1_row < r0 + C::RPB;  // block-uniform
            const bool l1_here = has_l1 && y == a.l1_row;
            const int tu = term - a.u_term0;
            float2 *U = (a.U && valid && tu >= 0 && tu % a.u_every == 0)
                            ? a.U + rhs * a.u_rhs + (size_t)(tu / a.u_every) * a.u_slot + (size_t)y * n
                            : nullptr;
            TBS_ROW_PHASE(2)
            // psi / V rows: with bulk copies every thread waits on their
            // barrier; with cp.async a thread reads exactly the elements it copied
            if (bulk) {
                if (valid) mbar_wait_bounded(&rbar[lr][1], 0, a.wait_ns, a.err);
            } else {
                cp_async_wait<0>();
            }
            TBS_ROW_PHASE(3)
#pragma unroll
            for (int m = 0; m < E; m++) {
                const int x = t + T * m;
                if (m < E / 2 && valid && x < n) {
                    const float2 u = v[m];
                    const float2 pold = first ? make_float2(0.f, 0.f) : psi_s[x];
                    const float2 p = cadd(pold, u);
                    a.psi[row_sp + x] = p;
                    if (U) U[x] = u;
                    su_f = fmaf(u.x, u.x, fmaf(u.y, u.y, su_f));
                    sp_f = fmaf(p.x, p.x, fmaf(p.y, p.y, sp_f));
                    if (l1_here) {
                        lu_f += hypotf(u.x, u.y);
                        lp_f += hypotf(pold.x, pold.y);
                    }
                    v[m] = cmul(v_s[x], u);
                } else {
                    v[m] = make_float2(0.f, 0.f);
                }
            }
            double su, sp, lu = 0.0, lp = 0.0;
            if (has_l1) {
                double o[4];
                row_sums<T, 4>({su_f, sp_f, lu_f, lp_f}, o, red, lr);
                su = o[0], sp = o[1], lu = o[2], lp = o[3];
            } else {
                double o[2];
                row_sums<T, 2>({su_f, sp_f}, o, red, lr);
                su = o[0], sp = o[1];
            }
            if (t == 0 && valid) {
                a.part[(size_t)rhs * n + y] = make_double2(su, sp);
                if (y == a.l1_row) a.l1[rhs] = make_double2(lu, lp);
            }
            TBS_ROW_PHASE(4)

        } else if constexpr (KIND == ROW_ADJ) {
            const float2 *Uj = a.U + rhs * a.u_rhs + (size_t)((term - a.u_term0) / a.u_every) * a.u_slot +
                               (size_t)y * n;
            // loads of a batch before its stores (Q is read-modify-written)
            constexpr int CH = 4;
#pragma unroll
            for (int m0 = 0; m0 < E / 2; m0 += CH) {
                float2 qo[CH], uu[CH], gg[CH], vv[CH];
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    const int x = t + T * (m0 + k);
                    const bool in = valid && x < n;
                    qo[k] = in ? a.Q[row_sp + x] : make_float2(0.f, 0.f);
                    uu[k] = in ? __ldg(Uj + x) : make_float2(0.f, 0.f);
                    gg[k] = in ? __ldg(a.src + row_sp + x) : make_float2(0.f, 0.f);
                    vv[k] = in ? __ldg(a.V + (size_t)y * n + x) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    const int m = m0 + k;
                    const int x = t + T * m;
                    if (valid && x < n) {
                        const float2 lam = v[m];
                        a.Q[row_sp + x] = cadd(qo[k], cmulc(uu[k], lam));  // += conj(lambda) u_j
                        v[m] = cadd(gg[k], cmulc(lam, vv[k]));              // ubar_j = g + conj(V) lambda
                    } else {
                        v[m] = make_float2(0.f, 0.f);
                    }
                }
            }
#pragma unroll
            for (int m = E / 2; m < E; m++) v[m] = make_float2(0.f, 0.f);
        } else if constexpr (KIND == ROW_EPS || KIND == ROW_EPSK) {
            constexpr bool KS = KIND == ROW_EPSK;  // k-space potential
            // The paper's iteration on the periodic grid (Section 3.1,
            // Algorithm 1): g = G (V psi + S) arrives here transformed back;
            // psi' = A g with the absorbing layer A(x, y) = abl[x] abl[y]
            // (none for psi^0 = G S), the Eq. 30 sums of |psi' - psi| and
            // |psi| on the l1 row and the squares of psi' - psi and psi', then
            // the next input V psi' + S.
            float su_f = 0.f, sp_f = 0.f, lu_f = 0.f, lp_f = 0.f;
            const bool first = (term == 0);
            const int r0 = blockIdx.x * C::RPB;
            const bool has_l1 = a.l1_row >= r0 && a.l1_row < r0 + C::RPB;  // block-uniform
            const bool l1_here = has_l1 && y == a.l1_row;
            const float ay = (!first && a.abl && valid) ? a.abl[y] : 1.f;
            // rows of V that repeat one value are read once, zero source rows
            // not at all (row-uniform branches)
            bool vuni = false, sany = true;
            float2 v0 = make_float2(0.f, 0.f);
            if constexpr (!KS) {
                vuni = a.vflag && valid && a.vflag[y];
                sany = !a.sflag || (valid && a.sflag[(size_t)rhs * n + y]);
                if (vuni) v0 = __ldg(a.V + (size_t)y * n);
            }
            // A batch's loads (psi read-modify-written; V, S and the layer
            // read-only) are all issued before its stores: one memory round
            // trip per batch instead of one per element.
            constexpr int CH = 4;
#pragma unroll
            for (int m0 = 0; m0 < E; m0 += CH) {
                float2 po[CH], vv[CH], ss[CH];
                float ax[CH];
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    const int x = t + T * (m0 + k);
                    const bool in = valid && x < n;
                    po[k] = (in && !first) ? a.psi[row_sp + x] : make_float2(0.f, 0.f);
                    if constexpr (KS) {  // vv <- psi^0 (after term 0)
                        vv[k] = (in && !first) ? a.psi0[row_sp + x] : make_float2(0.f, 0.f);
                        ss[k] = make_float2(0.f, 0.f);
                    } else {
                        vv[k] = in ? (vuni ? v0 : __ldg(a.V + (size_t)y * n + x)) : make_float2(0.f, 0.f);
                        ss[k] = (in && sany) ? __ldg(a.src + row_sp + x) : make_float2(0.f, 0.f);
                    }
                    ax[k] = (in && !first && a.abl) ? __ldg(a.abl + x) : 1.f;
                }
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    const int m = m0 + k;
                    const int x = t + T * m;
                    if (valid && x < n) {
                        const float sc = (!first && a.abl) ? ay * ax[k] : 1.f;
                        // k-space potential: psi' = A (g + psi^0) after term 0;
                        // preconditioned: psi' = A (psi + gamma (g - psi)), gamma = i V / eps
                        float2 gv = (KS && !first) ? cadd(v[m], vv[k]) : v[m];
                        if (!KS && a.cbs_inv_eps != 0.f && !first) {
                            const float2 gam = make_float2(-vv[k].y * a.cbs_inv_eps, vv[k].x * a.cbs_inv_eps);
                            gv = cadd(po[k], cmul(gam, make_float2(gv.x - po[k].x, gv.y - po[k].y)));
                        }
                        const float2 pn = make_float2(sc * gv.x, sc * gv.y);
                        if (KS && first) a.psi0[row_sp + x] = pn;
                        const float2 pold = po[k];
                        const float2 d = make_float2(pn.x - pold.x, pn.y - pold.y);
                        a.psi[row_sp + x] = pn;
                        su_f = fmaf(d.x, d.x, fmaf(d.y, d.y, su_f));
                        sp_f = fmaf(pn.x, pn.x, fmaf(pn.y, pn.y, sp_f));
                        if (l1_here) {
                            lu_f += hypotf(d.x, d.y);
                            lp_f += hypotf(pold.x, pold.y);
                        }
                        // next input: V psi' + S, or psi' itself with the k-space potential
                        v[m] = KS ? pn : cadd(cmul(vv[k], pn), ss[k]);
                    } else {
                        v[m] = make_float2(0.f, 0.f);
                    }
                }
            }
            double su, sp, lu = 0.0, lp = 0.0;
            if (has_l1) {
                double o[4];
                row_sums<T, 4>({su_f, sp_f, lu_f, lp_f}, o, red, lr);
                su = o[0], sp = o[1], lu = o[2], lp = o[3];
            } else {
                double o[2];
                row_sums<T, 2>({su_f, sp_f}, o, red, lr);
                su = o[0], sp = o[1];
            }
            if (t == 0 && valid) {
                a.part[(size_t)rhs * n + y] = make_double2(su, sp);
                if (y == a.l1_row) a.l1[rhs] = make_double2(lu, lp);
            }
        } else if constexpr (KIND == ROW_OUT) {
#pragma unroll
            for (int m = 0; m < E; m++) {
                const int x = t + T * m;
                if ((m < E / 2 || full) && valid && x < n) a.psi[row_sp + x] = v[m];
            }
        }
    }

    if constexpr (KIND == ROW_SRC || KIND == ROW_VSRC || KIND == ROW_FWD || KIND == ROW_ADJ || KIND == ROW_EPS ||
                  KIND == ROW_EPSK) {
        // the forward transform's first stores may skip their write-after-
        // read barrier where no thread has read the line since a block
        // barrier: the source pass (line unused so far) and the steady pass
        // with multi-warp rows (the row-norm barrier follows the inverse
        // transform's last reads)
        constexpr bool STEADY_FWD = KIND == ROW_FWD || KIND == ROW_EPS || KIND == ROW_EPSK;
        constexpr bool FRESH = KIND == ROW_SRC || KIND == ROW_VSRC || (STEADY_FWD && T > 32);
        // the padded passes' inputs are zero past column N <= M/2 (the source
        // passes may serve the periodic grid, whose rows are full)
        constexpr bool ZIN = KIND == ROW_FWD || KIND == ROW_ADJ;
        // the last admissible term, and adjoint step 0, feed no further
        // column pass (block-uniform)
        if (STEADY_FWD && term + 1 >= a.max_terms) return;
        if (KIND == ROW_ADJ && term == 0) return;
        fft_lines<M, E, -1, 1, ThreadTwiddles<M, E>, BlockSync, FRESH, ZIN>(va, sm, t, a.tw, &twr);
        TBS_ROW_PHASE(5)
        if (valid) {
            float2 *xo = a.X + ((size_t)rhs * n + y) * M;
#pragma unroll
            for (int m = 0; m < E; m++) xo[t + T * m] = v[m];
        }
        TBS_ROW_PHASE(6)
        TBS_ROW_PHASE_END
    }
}

// ---------------------------------------------------------------------------
// persistent steady-state row pass
// ---------------------------------------------------------------------------
// Named-barrier vote over a warp-aligned group: true when any thread's v is.
__device__ __forceinline__ bool group_sync_or(int id, int count, bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Sums of K values over the T threads of one row slot (T >= 32, warp-aligned
// groups of a block): an FP32 shuffle tree within each warp (the per-thread
// values are themselves FP32 sums of at most 8 squares, so the 5 tree levels
// add at most 5 roundings to their 7: a relative error below 1e-6, far below
// what the stop test resolves), then the slot's first warp combines the
// per-warp sums in double-float pairs and converts once to FP64 (fixed
// order: deterministic).  Results valid in the slot's thread 0.  Every call
// passes one barrier over the slot (`sync`), after which all of the slot's
// threads have made their calls.  red[k][w] holds slot warp w's sum of value k.
template <int T, int K, class SYNC>
__device__ __forceinline__ void slot_sums(const float (&x)[K], double (&out)[K], float2 (*red)[8], int t,
                                          const SYNC &sync) {
    static_assert(T >= 32 && T % 32 == 0 && T / 32 <= 8, "row slots of 1..8 warps");
    float xs[K];
#pragma unroll
    for (int k = 0; k < K; k++) xs[k] = x[k];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; k++) xs[k] += __shfl_xor_sync(0xffffffffu, xs[k], o);
    }
    DFloat v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = DFloat{xs[k], 0.f};
    constexpr int WPR = T / 32;
    const int lane = t & 31, w = t >> 5;
    if (WPR > 1 && lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) red[k][w] = make_float2(v[k].hi, v[k].lo);
    }
    sync();
    if constexpr (WPR > 1) {
        if (w == 0) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float2 r = lane < WPR ? red[k][lane] : make_float2(0.f, 0.f);
                v[k] = DFloat{r.x, r.y};
            }
#pragma unroll
            for (int o = WPR / 2; o >= 1; o >>= 1) {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const DFloat u{__shfl_xor_sync(0xffffffffu, v[k].hi, o),
                                   __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
                    v[k] = df_add(v[k], u);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) out[k] = (double)v[k].hi + (double)v[k].lo;
}

// Steady-state forward row pass (ROW_FWD) as a persistent kernel for M >= 512
// and even N: each block holds RPB row slots of T = M/16 threads, and each
// slot walks the rows i = slot, slot + (number of slots), ... of all active
// right-hand sides (row y of RHS r is i = r N + y).  A slot keeps four
// buffers: the padded exchange line, a landing row for the next W row, and
// the psi and V rows of the current row.  The next row's W is bulk-copied as
// soon as the current one is in registers, and its psi and V rows once the
// current epilogue has read them, so every copy has about a row's work to
// land.  The arithmetic per row is exactly that of row_kernel<M, ROW_FWD>.
template <int M>
struct RowPCfg {
    static constexpr int E = 16, T = M / E;
    static constexpr int RPB = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = T * RPB;
    static constexpr int LINE = RowCfg<M>::LINE;
    static constexpr int HALF = M / 2;
    static constexpr int SLOT = LINE + M + 2 * HALF;  // float2 elements per slot
    static constexpr size_t SMEM = (size_t)RPB * SLOT * sizeof(float2);
    static_assert(T >= 32 && RPB <= 8, "one to eight warp-aligned row slots per block");
    static_assert(LINE % 2 == 0 && M % 2 == 0 && HALF % 2 == 0, "16-byte aligned slot buffers");
};

template <int M>
__global__ void __launch_bounds__(RowPCfg<M>::THREADS, 2)
row_fwd_persistent_kernel(RowArgs a) {
    using C = RowPCfg<M>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float2 red_all[C::RPB][4][8];
    __shared__ __align__(8) uint64_t bars[C::RPB][2];  // [slot][0: W, 1: psi and V]
    const int lr = threadIdx.x / T;
    const int t = threadIdx.x % T;
    const int n = a.n;
    float2 *line = smem + (size_t)lr * C::SLOT;
    float2 *wl = line + C::LINE;
    float2 *psi_s = wl + M;
    float2 *v_s = psi_s + C::HALF;
    const GroupSync sync{1 + lr, T};
    const Lines<1> sm{line, 0};
    uint64_t *bar_w = &bars[lr][0], *bar_pv = &bars[lr][1];
    if (t == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_pv, 1);
        mbar_init_fence();
    }
    ThreadTwiddles<M, E> twr;
    twr.load(a.tw, t);
    sync();  // the slot's barriers are initialised before anyone waits
    grid_dep_wait();
    const int total = a.nrhs * n;
    const int nslots = gridDim.x * C::RPB;
    // each RHS's flag and term index cannot change during this launch: read
    // them once per RHS (rows are RHS-major, so the cache almost always hits)
    int cached_rhs = -1, cached_term = 0;
    bool cached_active = false;
    auto next_active = [&](int i) {
        while (i < total) {
            const int r = i / n;
            if (r != cached_rhs) {
                cached_rhs = r;
                cached_active = gate_active(a.gate, r);
                cached_term = a.term >= 0 ? a.term : a.gate.st[r].terms;
            }
            if (cached_active) break;
            i += nslots;
        }
        return i;
    };
    const unsigned wbytes = (unsigned)(M * sizeof(float2)), rbytes = (unsigned)(n * sizeof(float2));
    auto issue_w = [&](int i) {  // slot thread 0
        const int r = i / n, y = i - r * n;
        mbar_arrive_expect_tx(bar_w, wbytes);
        bulk_load(wl, a.W + ((size_t)r * n + y) * M, wbytes, bar_w);
    };
    auto issue_pv = [&](int i) {  // slot thread 0
        const int r = i / n, y = i - r * n;
        mbar_arrive_expect_tx(bar_pv, 2 * rbytes);
        bulk_load(psi_s, a.psi + (size_t)r * n * n + (size_t)y * n, rbytes, bar_pv);
        bulk_load(v_s, a.V + (size_t)y * n, rbytes, bar_pv);
    };
    int i = next_active(blockIdx.x * C::RPB + lr);
    if (t == 0 && i < total) {
        issue_w(i);
        issue_pv(i);
    }
    grid_dep_launch();  // the stop test may be scheduled once every row block runs
    unsigned ph_w = 0, ph_pv = 0;
    float2 va[1][E];
    float2 (&v)[E] = va[0];
    float2 (*red)[8] = red_all[lr];
    while (i < total) {
        const int rhs = i / n, y = i - rhs * n;
        const int term = cached_term;  // of row i's RHS (next_active left the cache on it)
        const int inext = next_active(i + nslots);
        // the W row: registers, then the landing row is free for the next one
        const bool okw = mbar_wait_bounded(bar_w, ph_w, a.wait_ns, a.err);
        ph_w ^= 1u;
        if (group_sync_or(1 + lr, T, !okw)) {
            // a copy never completed: give the outstanding ones a bounded
            // chance to land, then leave this slot (error word set)
            if (t == 0) {
                mbar_wait_bounded(bar_w, ph_w ^ 1u, a.wait_ns, nullptr);
                mbar_wait_bounded(bar_pv, ph_pv, a.wait_ns, nullptr);
            }
            return;
        }
#pragma unroll
        for (int m = 0; m < E; m++) v[m] = wl[t + T * m];
        sync();  // every thread's reads of the landing row are done
        if (t == 0 && inext < total) {
            fence_proxy_async_smem();
            issue_w(inext);
        }
        // the previous row's forward transform read the exchange line before
        // the barrier above: the inverse transform's first stores need no other
        fft_lines<M, E, +1, 1, ThreadTwiddles<M, E>, GroupSync, true>(va, sm, t, a.tw, &twr, sync);

        float su_f = 0.f, sp_f = 0.f, lu_f = 0.f, lp_f = 0.f;
        const bool first = (term == 0);
        const bool l1_here = y == a.l1_row;  // slot-uniform
        const int tu = term - a.u_term0;
        float2 *U = (a.U && tu >= 0 && tu % a.u_every == 0)
                        ? a.U + rhs * a.u_rhs + (size_t)(tu / a.u_every) * a.u_slot + (size_t)y * n
                        : nullptr;
        const size_t row_sp = (size_t)rhs * n * n + (size_t)y * n;
        const bool okp = mbar_wait_bounded(bar_pv, ph_pv, a.wait_ns, a.err);
        ph_pv ^= 1u;
        if (group_sync_or(1 + lr, T, !okp)) {  // as above; the next W row may be in flight
            if (t == 0) {
                if (inext < total) mbar_wait_bounded(bar_w, ph_w, a.wait_ns, nullptr);
                mbar_wait_bounded(bar_pv, ph_pv ^ 1u, a.wait_ns, nullptr);
            }
            return;
        }
        // u -> psi += u, the norms' partial sums, V u; the N = M/2 grids (every
        // slot of the half row a grid point) skip the per-element bound
        auto epilogue = [&](auto full_c) {
            constexpr bool FULL = decltype(full_c)::value;
#pragma unroll
            for (int m = 0; m < E / 2; m++) {
                const int x = t + T * m;
                if (FULL || x < n) {
                    const float2 u = v[m];
                    const float2 pold = first ? make_float2(0.f, 0.f) : psi_s[x];
                    const float2 p = cadd(pold, u);
                    a.psi[row_sp + x] = p;
                    if (U) U[x] = u;
                    su_f = fmaf(u.x, u.x, fmaf(u.y, u.y, su_f));
                    sp_f = fmaf(p.x, p.x, fmaf(p.y, p.y, sp_f));
                    if (l1_here) {
                        lu_f += hypotf(u.x, u.y);
                        lp_f += hypotf(pold.x, pold.y);
                    }
                    v[m] = cmul(v_s[x], u);
                } else {
                    v[m] = make_float2(0.f, 0.f);
                }
            }
        };
        if (n == M / 2)
            epilogue(std::true_type{});
        else
            epilogue(std::false_type{});
#pragma unroll
        for (int m = E / 2; m < E; m++) v[m] = make_float2(0.f, 0.f);
        // the sums pass one slot barrier, after every thread's reads of the
        // psi and V rows: their buffers are free for the next row's copies
        double su, sp, lu = 0.0, lp = 0.0;
        if (l1_here) {
            double o[4];
            slot_sums<T, 4>({su_f, sp_f, lu_f, lp_f}, o, red, t, sync);
            su = o[0], sp = o[1], lu = o[2], lp = o[3];
        } else {
            double o[2];
            slot_sums<T, 2>({su_f, sp_f}, o, red, t, sync);
            su = o[0], sp = o[1];
        }
        if (t == 0) {
            if (inext < total) {
                fence_proxy_async_smem();
                issue_pv(inext);
            }
            a.part[(size_t)rhs * n + y] = make_double2(su, sp);
            if (l1_here) a.l1[rhs] = make_double2(lu, lp);
        }
        if (term + 1 < a.max_terms) {  // the last admissible term feeds no further column pass
            // the barrier in the sums follows the inverse transform's last
            // reads of the exchange line
            fft_lines<M, E, -1, 1, ThreadTwiddles<M, E>, GroupSync, true, true>(va, sm, t, a.tw, &twr, sync);
            float2 *xo = a.X + ((size_t)rhs * n + y) * M;
#pragma unroll
            for (int m = 0; m < E; m++) xo[t + T * m] = v[m];
        }
        i = inext;
    }
}

// Steady-state periodic row pass (ROW_EPS, or ROW_EPSK with the k-space
// potential) as a persistent kernel, M >= 512: the paper's iteration on the
// field itself (Section 3.1, Algorithm 1) with the arithmetic of
// row_kernel<M, ROW_EPS/EPSK>.  Each row slot keeps the exchange line, a
// landing row for the next W row and the current psi row (whole rows: the
// periodic grid has no padding); both are bulk-copied a row ahead.  V, S and
// psi^0 are read from global memory in batches, with the per-row flags (V
// rows of one value read once, zero source rows not at all).
template <int M>
struct RowECfg {
    static constexpr int E = 16, T = M / E;
    static constexpr int RPB = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = T * RPB;
    static constexpr int LINE = RowCfg<M>::LINE;
    static constexpr int SLOT = LINE + 2 * M;  // exchange line, W landing, psi row
    static constexpr size_t SMEM = (size_t)RPB * SLOT * sizeof(float2);
    static_assert(T >= 32 && RPB <= 8, "one to eight warp-aligned row slots per block");
};

template <int M, bool KS>
__global__ void __launch_bounds__(RowECfg<M>::THREADS, 2)
row_eps_persistent_kernel(RowArgs a) {
    using C = RowECfg<M>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float2 red_all[C::RPB][4][8];
    __shared__ __align__(8) uint64_t bars[C::RPB][2];  // [slot][0: W, 1: psi]
    const int lr = threadIdx.x / T;
    const int t = threadIdx.x % T;
    const int n = a.n;  // = M
    float2 *line = smem + (size_t)lr * C::SLOT;
    float2 *wl = line + C::LINE;
    float2 *psi_s = wl + M;
    const GroupSync sync{1 + lr, T};
    const Lines<1> sm{line, 0};
    uint64_t *bar_w = &bars[lr][0], *bar_p = &bars[lr][1];
    if (t == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_p, 1);
        mbar_init_fence();
    }
    ThreadTwiddles<M, E> twr;
    twr.load(a.tw, t);
    // bit m: the layer profile at this thread's column t + T m is not 1 (the
    // interior of the grid needs no profile load in the epilogue)
    unsigned amask = 0u;
    if (a.abl) {
#pragma unroll
        for (int m = 0; m < E; m++) amask |= (__ldg(a.abl + t + T * m) != 1.f ? 1u : 0u) << m;
    }
    sync();
    grid_dep_wait();
    const int total = a.nrhs * n;
    const int nslots = gridDim.x * C::RPB;
    int cached_rhs = -1, cached_term = 0;
    bool cached_active = false;
    auto next_active = [&](int i) {
        while (i < total) {
            const int r = i / n;
            if (r != cached_rhs) {
                cached_rhs = r;
                cached_active = gate_active(a.gate, r);
                cached_term = a.term >= 0 ? a.term : a.gate.st[r].terms;
            }
            if (cached_active) break;
            i += nslots;
        }
        return i;
    };
    const unsigned rbytes = (unsigned)(M * sizeof(float2));
    auto issue_w = [&](int i) {
        const int r = i / n, y = i - r * n;
        mbar_arrive_expect_tx(bar_w, rbytes);
        bulk_load(wl, a.W + ((size_t)r * n + y) * M, rbytes, bar_w);
    };
    auto issue_p = [&](int i) {
        const int r = i / n, y = i - r * n;
        mbar_arrive_expect_tx(bar_p, rbytes);
        bulk_load(psi_s, a.psi + (size_t)r * n * n + (size_t)y * n, rbytes, bar_p);
        // the epilogue reads psi^0 element by element: have L2 fetch the row now
        if constexpr (KS) bulk_prefetch_l2(a.psi0 + (size_t)r * n * n + (size_t)y * n, rbytes);
    };
    int i = next_active(blockIdx.x * C::RPB + lr);
    if (t == 0 && i < total) {
        issue_w(i);
        issue_p(i);
    }
    grid_dep_launch();
    unsigned ph_w = 0, ph_p = 0;
    float2 va[1][E];
    float2 (&v)[E] = va[0];
    float2 (*red)[8] = red_all[lr];
    while (i < total) {
        const int rhs = i / n, y = i - rhs * n;
        const int term = cached_term;
        const int inext = next_active(i + nslots);
        const bool okw = mbar_wait_bounded(bar_w, ph_w, a.wait_ns, a.err);
        ph_w ^= 1u;
        if (group_sync_or(1 + lr, T, !okw)) {
            if (t == 0) {
                mbar_wait_bounded(bar_w, ph_w ^ 1u, a.wait_ns, nullptr);
                mbar_wait_bounded(bar_p, ph_p, a.wait_ns, nullptr);
            }
            return;
        }
#pragma unroll
        for (int m = 0; m < E; m++) v[m] = wl[t + T * m];
        sync();
        if (t == 0 && inext < total) {
            fence_proxy_async_smem();
            issue_w(inext);
        }
        fft_lines<M, E, +1, 1, ThreadTwiddles<M, E>, GroupSync, true>(va, sm, t, a.tw, &twr, sync);

        // psi' = A g (no layer for psi^0 = G S), the Eq. 30 sums of
        // |psi' - psi| and |psi| on the l1 row and the squares of psi' - psi
        // and psi', then the next input V psi' + S (or psi' itself, k-space)
        float su_f = 0.f, sp_f = 0.f, lu_f = 0.f, lp_f = 0.f;
        const bool first = (term == 0);
        const bool l1_here = y == a.l1_row;
        const float ay = (!first && a.abl) ? a.abl[y] : 1.f;
        bool vuni = false, sany = true;
        float2 v0 = make_float2(0.f, 0.f);
        if constexpr (!KS) {
            vuni = a.vflag && a.vflag[y];
            sany = !a.sflag || a.sflag[(size_t)rhs * n + y];
            if (vuni) v0 = __ldg(a.V + (size_t)y * n);
        }
        const size_t row_sp = (size_t)rhs * n * n + (size_t)y * n;
        const bool okp = mbar_wait_bounded(bar_p, ph_p, a.wait_ns, a.err);
        ph_p ^= 1u;
        if (group_sync_or(1 + lr, T, !okp)) {
            if (t == 0) {
                if (inext < total) mbar_wait_bounded(bar_w, ph_w, a.wait_ns, nullptr);
                mbar_wait_bounded(bar_p, ph_p ^ 1u, a.wait_ns, nullptr);
            }
            return;
        }
        // a batch's loads are issued before its stores; the k-space pass reads
        // only psi^0 per element, so it takes larger batches (fewer round trips)
        constexpr int CH = KS ? 8 : 4;
#pragma unroll
        for (int m0 = 0; m0 < E; m0 += CH) {
            float2 vv[CH], ss[CH];
            float ax[CH];
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int x = t + T * (m0 + k);
                if constexpr (KS) {  // vv <- psi^0 (after term 0)
                    vv[k] = !first ? a.psi0[row_sp + x] : make_float2(0.f, 0.f);
                    ss[k] = make_float2(0.f, 0.f);
                } else {
                    vv[k] = vuni ? v0 : __ldg(a.V + (size_t)y * n + x);
                    ss[k] = sany ? __ldg(a.src + row_sp + x) : make_float2(0.f, 0.f);
                }
                ax[k] = (!first && ((amask >> (m0 + k)) & 1u)) ? __ldg(a.abl + x) : 1.f;
            }
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int m = m0 + k;
                const int x = t + T * m;
                const float2 pold = first ? make_float2(0.f, 0.f) : psi_s[x];
                const float sc = (!first && a.abl) ? ay * ax[k] : 1.f;
                float2 gv = (KS && !first) ? cadd(v[m], vv[k]) : v[m];
                if (!KS && a.cbs_inv_eps != 0.f && !first) {
                    const float2 gam = make_float2(-vv[k].y * a.cbs_inv_eps, vv[k].x * a.cbs_inv_eps);
                    gv = cadd(pold, cmul(gam, make_float2(gv.x - pold.x, gv.y - pold.y)));
                }
                const float2 pn = make_float2(sc * gv.x, sc * gv.y);
                if (KS && first) a.psi0[row_sp + x] = pn;
                const float2 d = make_float2(pn.x - pold.x, pn.y - pold.y);
                a.psi[row_sp + x] = pn;
                su_f = fmaf(d.x, d.x, fmaf(d.y, d.y, su_f));
                sp_f = fmaf(pn.x, pn.x, fmaf(pn.y, pn.y, sp_f));
                if (l1_here) {
                    lu_f += hypotf(d.x, d.y);
                    lp_f += hypotf(pold.x, pold.y);
                }
                v[m] = KS ? pn : cadd(cmul(vv[k], pn), ss[k]);
            }
        }
        double su, sp, lu = 0.0, lp = 0.0;
        if (l1_here) {
            double o[4];
            slot_sums<T, 4>({su_f, sp_f, lu_f, lp_f}, o, red, t, sync);
            su = o[0], sp = o[1], lu = o[2], lp = o[3];
        } else {
            double o[2];
            slot_sums<T, 2>({su_f, sp_f}, o, red, t, sync);
            su = o[0], sp = o[1];
        }
        if (t == 0) {
            if (inext < total) {
                fence_proxy_async_smem();
                issue_p(inext);
            }
            a.part[(size_t)rhs * n + y] = make_double2(su, sp);
            if (l1_here) a.l1[rhs] = make_double2(lu, lp);
        }
        if (term + 1 < a.max_terms) {
            fft_lines<M, E, -1, 1, ThreadTwiddles<M, E>, GroupSync, true>(va, sm, t, a.tw, &twr, sync);
            float2 *xo = a.X + ((size_t)rhs * n + y) * M;
#pragma unroll
            for (int m = 0; m < E; m++) xo[t + T * m] = v[m];
        }
        i = inext;
    }
}

// ---------------------------------------------------------------------------
// column pass
// ---------------------------------------------------------------------------
// 2^x by the hardware's approximate base-2 exponential (PTX ex2.approx.ftz:
// +0 for x = -inf; the callers' arguments are >= 0 or -inf).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The periodic grid's spectrum at integer wavenumbers (ix, iy) (Section 2.2
// with finite eps): g~(p)/M^2 = gs (a + i eq) / (a^2 + eq^2), a = ix^2 + iy^2
// - kq, and with the k-space potential (Section 3.1 case II) times
// VV(p) = eta |p|^(nu+1) - i (tau omega |p|^nu + eps).
template <bool KS>
__device__ __forceinline__ float2 periodic_spectrum(const ColArgs &a, float ix, float iy) {
    const float sq = fmaf(ix, ix, iy * iy);
    const float q = sq - a.kq;
    // the fast division (2 ulp; the denominator is >= eq^2 > 0 and far below
    // 2^126 for M <= 4096)
    const float r = __fdividef(a.gs, fmaf(q, q, a.eq * a.eq));
    float2 g = make_float2(q * r, a.eq * r);
    if constexpr (KS) {
        // s^(nu/2) and s^((nu+1)/2) from one base-2 logarithm and two base-2
        // exponentials, each the hardware approximation (PTX lg2.approx /
        // ex2.approx, a few ulp each: a relative error of a few 1e-6 at most
        // in the powers, against the 2e-5 field tolerance); s = 0 gives
        // log2 = -inf and powers 0 (VV(0) = -i eps)
        const float lg = __log2f(sq);
        const float sn = ex2_approx(a.vv_half_nu * lg);
        const float sn1 = ex2_approx((a.vv_half_nu + 0.5f) * lg);
        g = cmul(g, make_float2(a.vv_a1 * sn1, -(a.vv_a2 * sn + a.vv_eps)));
    }
    return g;
}

// Loads this thread's L columns (rows t + T m, m < E/2, below N) of a tile.
template <class C, int M>
__device__ __forceinline__ void col_load(float2 (&v)[C::L][C::E], const float2 *src, int stride,
                                         int n, int t, int c0) {
    constexpr int E = C::E, T = C::T, L = C::L;
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int ky = t + T * m;
        const bool in = (C::PER || m < E / 2) && ky < n;
        if constexpr (L == 2) {
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) f = *reinterpret_cast<const float4 *>(src + (size_t)ky * stride + c0);
            v[0][m] = make_float2(f.x, f.y);
            v[1][m] = make_float2(f.z, f.w);
        } else {
#pragma unroll
            for (int l = 0; l < L; l++) v[l][m] = in ? src[(size_t)ky * stride + c0 + l] : make_float2(0.f, 0.f);
        }
    }
}

// Forward FFT along y, x Ghat (the tile's columns in shared memory,
// [kyq][QSP] per column), inverse FFT; rows y < N of the result go to `out`
// ([row][TC] like the input tile).  between(): called after the Ghat product.
template <class C, int M, bool CONJ, class MID, class SYNC>
__device__ __forceinline__ void col_transform(float2 (&v)[C::L][C::E], float2 *exch, const ColArgs &a, int t,
                                              int lane_group, int x0, bool kspace, const ThreadTwiddles<M, C::E> &twr,
                                              const float2 *gbuf, float2 *out, MID between, const SYNC &sync) {
    constexpr int E = C::E, T = C::T, L = C::L;
    const int n = a.n;
    // two columns per thread: the two lines interleaved (16-byte accesses)
    const Lines<L, L == 2> sm{exch + L * lane_group * C::LSTRIDE, C::LSTRIDE};
    // the tile loop's block barrier follows the previous tile's last reads
    // of the exchange line: the forward transform's first stores need no other
    fft_lines<M, E, -1, L, ThreadTwiddles<M, E>, SYNC, true, !C::PER>(v, sm, t, a.tw, &twr, sync);
    // the spectral product (with the k-space potential: its own kernel, and
    // a second unrolled loop for the RHS's first term, which applies G only)
    auto multiply = [&](auto ks) {
        constexpr bool KS = decltype(ks)::value;
#pragma unroll
        for (int l = 0; l < L; l++) {
            const int kx = x0 + L * lane_group + l;
            const float ix = (float)(kx < M / 2 ? kx : kx - M);
#pragma unroll
            for (int m = 0; m < E; m++) {
                const int ky = t + T * m;
                float2 g;
                if constexpr (C::PER) {
                    g = periodic_spectrum<KS>(a, ix, (float)(ky < M / 2 ? ky : ky - M));
                } else {
                    const int kyq = ky <= M / 2 ? ky : M - ky;
                    g = gbuf[(L * lane_group + l) * C::QSP + kyq];
                }
                v[l][m] = CONJ ? cmulc(v[l][m], g) : cmul(v[l][m], g);
            }
        }
    };
    if constexpr (C::KS) {
        if (kspace)
            multiply(std::true_type{});
        else
            multiply(std::false_type{});
    } else {
        multiply(std::false_type{});
    }
    between();
    fft_lines<M, E, +1, L>(v, sm, t, a.tw, &twr, sync);
#pragma unroll
    for (int m = 0; m < (C::PER ? E : E / 2); m++) {
        const int y = t + T * m;
        if (y < n) {
            if constexpr (L == 2) {  // both columns with one 16-byte store
                *reinterpret_cast<float4 *>(out + (size_t)y * C::TC + 2 * lane_group) =
                    make_float4(v[0][m].x, v[0][m].y, v[1][m].x, v[1][m].y);
            } else {
#pragma unroll
                for (int l = 0; l < L; l++) out[(size_t)y * C::TC + L * lane_group + l] = v[l][m];
            }
        }
    }
}

// Optional phase timers for experiments (compiled out unless defined).
#ifndef TBS_COL_PHASE
#define TBS_COL_PHASE_DECL
#define TBS_COL_PHASE(k)
#define TBS_COL_PHASE_END
#endif

// Persistent column pass: one block per SM (or per resident slot) walks the
// tiles of TC columns.  Shared memory holds two stages, each [input rows
// (HALF x TC)][Ghat columns (TC x QSP)], and the exchange lines.  A tile's
// input arrives by tensor copies into its stage; its output rows are written
// back into the same landing rows (free once loaded into registers) and leave
// by a tensor store, issued after the next tile's block barrier.  The next
// tile's copies are issued after the forward transform, once that store has
// read the rows they overwrite.
template <int M, bool CONJ, class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
col_kernel(ColArgs a, const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw) {
    constexpr int TC = C::TC, L = C::L, G = TC / L;
    constexpr int TILES = M / TC;
    extern __shared__ __align__(16) float2 smem_raw[];
    // tensor-copy destinations must be 128-byte aligned in the shared window
    float2 *smem = reinterpret_cast<float2 *>(reinterpret_cast<char *>(smem_raw) +
                                              ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    const int n = a.n;
    const int cg = C::BLOCKED ? threadIdx.x / C::T : threadIdx.x % G;  // column group within the tile
    const int t = C::BLOCKED ? threadIdx.x % C::T : threadIdx.x / G;
    float2 v[L][C::E];
    ThreadTwiddles<M, C::E> twr;  // this thread's twiddles, for every tile
    twr.load(a.tw, t);
    float2 *exch = smem + 2 * C::STAGE;
    const int total = TILES * a.nrhs;
    // The RHS flags cannot change during this launch: read each RHS's flag
    // once (tiles are ordered by RHS, so the cache almost always hits).
    int cached_rhs = -1;
    bool cached_active = false;
    auto next_active = [&](int i) {
        while (i < total) {
            const int r = i / TILES;
            if (r != cached_rhs) {
                cached_rhs = r;
                cached_active = gate_active(a.gate, r);
            }
            if (cached_active) break;
            i += gridDim.x;
        }
        return i;
    };
    TBS_COL_PHASE_DECL
    // One copy barrier per stage.  A tile's input rows arrive by one 3D
    // tensor copy (or one per BR rows) and its Ghat columns by one bulk copy
    // each.  Thread 0 arms a stage's barrier before the block barrier that
    // precedes its copies, so every copy finds it armed.
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    grid_dep_wait();  // X, the RHS flags
    unsigned par0 = 0u, par1 = 0u;  // phase parity of each stage's barrier (registers, not an array)
    constexpr int NW = (C::THREADS + 31) / 32;  // warps (blocks of 8 or 16 threads: one)
    static_assert(NW >= 1, "the copy-issue loop advances by NW");
    constexpr unsigned GROW = C::QSP * sizeof(float2);  // one stored quadrant row
    const int nx = a.xslice ? 1 : (n + C::BR - 1) / C::BR;  // row copies per tile
    const unsigned xbytes = (unsigned)((a.xslice ? n : nx * C::BR) * TC * sizeof(float2));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // self-check of the copies' alignment rules (stage base, first column,
    // Ghat rows): a violation is reported through the error word and no copy
    // is issued (the wait then runs out)
    auto copies_aligned = [&](int i, int buf) {
        const float2 *st = smem + buf * C::STAGE;
        const int x0 = (i % TILES) * TC;
        return (smem_u32(st) & 127u) == 0 && ((x0 * (int)sizeof(float2)) & 15) == 0 &&
               (C::PER || ((smem_u32(st + C::LAND) & 15u) == 0 && (GROW & 15u) == 0 &&
                           (reinterpret_cast<uintptr_t>(a.ghq) & 15u) == 0));
    };
    auto arm = [&](int i, int buf) {  // thread 0
        if (copies_aligned(i, buf)) {
            mbar_arrive_expect_tx(&bar[buf], xbytes + (C::PER ? 0u : TC * GROW) + a.extra_tx);
        } else {
            if (a.err) atomicExch(a.err, 2);
            mbar_arrive_expect_tx(&bar[buf], 16u);  // never completes: the bounded wait ends it
        }
    };
    // Tile rows in the box geometry of the tensor maps: one box of n rows at
    // slice z = rhs * (n / xslice), or boxes of BR rows at (q * BR, rhs).
    // Thread 0 issues the row copies (they overwrite the rows its last
    // tensor store reads, so it first waits for that read); Ghat column c is
    // issued by lane 0 of warp (1 + c) % NW.
    auto issue = [&](int i, int buf) {
        if (lane != 0 || !copies_aligned(i, buf)) return;
        float2 *st = smem + buf * C::STAGE;
        const int x0 = (i % TILES) * TC;
        const int r = i / TILES;
        if (warp == 0) {
            bulk_wait_read_all();
            fence_proxy_async_smem();  // and the block's reads before its last barrier
            for (int q = 0; q < nx; q++) {
                if (a.xslice)
                    tma_load_3d(st, &tmx, x0, 0, r * (n / a.xslice), &bar[buf]);
                else
                    tma_load_3d(st + (size_t)q * C::BR * TC, &tmx, x0, q * C::BR, r, &bar[buf]);
            }
        }
        bool fenced = warp == 0;
        for (int c = 0; c < (C::PER ? 0 : TC); c++) {
            if ((1 + c) % NW != warp) continue;
            if (!fenced) fence_proxy_async_smem();  // the block's reads of these Ghat rows came first
            fenced = true;
            // Ghat column kxq is quadrant row kxq (the spectrum is symmetric
            // under transposition): one contiguous copy
            const int kx = x0 + c;
            const int kxq = kx <= M / 2 ? kx : M - kx;
            bulk_load(st + C::LAND + c * C::QSP, a.ghq + (size_t)kxq * C::QSP, GROW, &bar[buf]);
        }
    };
    auto store = [&](int i, int buf) {  // thread 0: output rows of tile i from stage buf
        const float2 *st = smem + buf * C::STAGE;
        const int x0 = (i % TILES) * TC;
        const int r = i / TILES;
        for (int q = 0; q < nx; q++) {
            if (a.xslice)
                tma_store_3d(&tmw, x0, 0, r * (n / a.xslice), st);
            else
                tma_store_3d(&tmw, x0, q * C::BR, r, st + (size_t)q * C::BR * TC);
        }
        bulk_commit();
    };
    int i = next_active(blockIdx.x);
    if (i < total) {
        if (threadIdx.x == 0) arm(i, 0);
        __syncthreads();
        issue(i, 0);
    }
    int prev = -1;  // tile whose output rows wait in the other stage
    for (int buf = 0; i < total; buf ^= 1) {
        const int inext = next_active(i + gridDim.x);
        TBS_COL_PHASE(0)
        const unsigned par = buf ? par1 : par0;
        const bool ok = mbar_wait_bounded(&bar[buf], par, a.wait_ns, a.err);
        // stage buf^1 was last waited on (by every thread) before the
        // previous block barrier: its barrier may be re-armed now
        if (threadIdx.x == 0 && ok && inext < total) arm(inext, buf ^ 1);
        fence_proxy_async_smem();  // this thread's output rows of tile prev, for the tensor store
        // tile i has landed in stage buf; tile prev's output rows are complete
        if (__syncthreads_or(!ok)) {
            // a copy never completed: give its bytes one more bounded chance
            // to land, let the stores finish, then leave (error word set)
            mbar_wait_bounded(&bar[buf], par, a.wait_ns, nullptr);
            if (threadIdx.x == 0) bulk_wait_all();
            return;
        }
        if (buf) par1 ^= 1u;
        else par0 ^= 1u;
        if (threadIdx.x == 0 && prev >= 0) store(prev, buf ^ 1);
        TBS_COL_PHASE(1)
        float2 *st = smem + buf * C::STAGE;
        col_load<C, M>(v, st, TC, n, t, L * cg);
        auto between = [&] {
            TBS_COL_PHASE(2)
            if (inext < total) issue(inext, buf ^ 1);
            TBS_COL_PHASE(3)
        };
        // k-space potential: from the RHS's second term on (its first applies G only)
        const bool kspace = C::KS && a.gate.st && a.gate.st[i / TILES].terms > 0;
        if constexpr (C::BLOCKED)
            col_transform<C, M, CONJ>(v, exch, a, t, cg, (i % TILES) * TC, kspace, twr, st + C::LAND, st, between,
                                      GroupSync{1 + cg, C::T});
        else
            col_transform<C, M, CONJ>(v, exch, a, t, cg, (i % TILES) * TC, kspace, twr, st + C::LAND, st, between,
                                      BlockSync{});
        TBS_COL_PHASE(5)
        prev = i;
        i = inext;
        if (i >= total) {
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) store(prev, buf);
        }
    }
    TBS_COL_PHASE_END
    if (threadIdx.x == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// pipelined column pass (M >= 1024; padded grid, or the periodic grid)
// ---------------------------------------------------------------------------
// The tile shape and thread layout of col_kernel (TC = 8192 / M columns per
// tile, one column per T = M/16 threads, 512 threads), with the staging
// split by lifetime so that every copy is issued a whole tile or more ahead:
//   D[0], D[1]  input rows of tiles k and k+1 (a tile's rows are in registers
//               right after its copy lands, so tile k+2 is copied into D[k&1]
//               at once)
//   GB          the Ghat columns of the current tile (the next tile's are
//               copied as soon as the spectral product has read them)
//   O           output rows, written after the inverse transform and sent by
//               one tensor store (the next tile writes O once that store has
//               read it)
//   exchange lines, one per column of the tile.
// Periodic grid (PER_ = 1, or 2 with the k-space potential): all M rows are
// grid points, so D[0], D[1] hold twice the rows; the spectrum is formed in
// the kernel (no GB), and O lies over the exchange lines (the tile's output
// rows are written there after the inverse transform's last exchange, and
// the next tile's first exchange waits until the tensor store has read them).
// RS_: the FFT's radix split (0: 16 x 16 x 16 at M = 4096, 1: 8 x 8 x 8 x 8).
template <int M, int L_ = 1, bool STAG_ = false, int PER_ = 0, int RS_ = 0>
struct ColPShape : ColShape<M, 8192 / M, L_, 1, PER_> {
    using B_ = ColShape<M, 8192 / M, L_, 1, PER_>;
    static constexpr bool PIPE = true;
    static constexpr int PERK = PER_;
    static constexpr int RS = RS_;
    static_assert(RS_ == 0 || !STAG_, "the staggered pair uses the default radix split");
    // two columns per thread transformed staggered (fft_pair), each in its
    // own exchange buffer with its own block-wide named barrier
    static constexpr bool STAG = STAG_;
    static_assert(!STAG_ || L_ == 2, "staggering pairs two columns");
    static constexpr size_t OFF_G = (PER_ ? 2 : 3) * B_::LAND;
    static constexpr size_t OFF_X = OFF_G + (PER_ ? 0 : (((size_t)B_::QSP * B_::TC + 15) & ~(size_t)15));
    static constexpr size_t OFF_O = PER_ ? OFF_X : 2 * B_::LAND;
    static constexpr size_t SMEM = (OFF_X + (size_t)B_::LSTRIDE * B_::TC) * sizeof(float2) + 128;
    static_assert(B_::LAND % 16 == 0 && OFF_X % 16 == 0, "stages, O and the lines stay 128-byte aligned");
    static_assert(!PER_ || B_::LAND <= (size_t)B_::LSTRIDE * B_::TC, "O fits over the exchange lines");
    static_assert(SMEM <= 232448, "one block's shared memory");
    static_assert(B_::THREADS == 512 / L_, "512 / L threads per block");
};

// L = 2: each thread transforms two columns of the tile (256 threads, up to
// 255 registers each, one block barrier per exchange for both columns, or
// with STAG the two columns staggered on two barriers)
template <int M, bool CONJ, int L_ = 1, bool STAG_ = false, int PER_ = 0, int RS_ = 0>
__global__ void __launch_bounds__(512 / L_, 1)
col_pipe_kernel(ColArgs a, const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw) {
    using C = ColPShape<M, L_, STAG_, PER_, RS_>;
    static_assert(!PER_ || !CONJ, "the periodic grid has the forward spectrum only");
    constexpr int TC = C::TC, L = C::L, G = TC / L, E = C::E, T = C::T;
    constexpr int TILES = M / TC;
    extern __shared__ __align__(16) float2 smem_raw[];
    float2 *smem = reinterpret_cast<float2 *>(reinterpret_cast<char *>(smem_raw) +
                                              ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    float2 *D0 = smem, *D1 = smem + C::LAND, *O = smem + C::OFF_O, *GB = smem + C::OFF_G;
    float2 *exch = smem + C::OFF_X;
    const int n = a.n;
    const int cg = C::BLOCKED ? threadIdx.x / T : threadIdx.x % G;
    const int t = C::BLOCKED ? threadIdx.x % T : threadIdx.x / G;
    using TWR = ThreadTwiddles<M, E, C::RS>;
    TWR twr;
    twr.load(a.tw, t);
    __shared__ __align__(8) uint64_t bars[3];  // D[0], D[1], GB
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_init_fence();
    }
    __syncthreads();
    grid_dep_wait();  // X, the RHS flags
    const int total = TILES * a.nrhs;
    int cached_rhs = -1;
    bool cached_active = false;
    auto next_active = [&](int i) {
        while (i < total) {
            const int r = i / TILES;
            if (r != cached_rhs) {
                cached_rhs = r;
                cached_active = gate_active(a.gate, r);
            }
            if (cached_active) break;
            i += gridDim.x;
        }
        return i;
    };
    constexpr unsigned GROW = C::QSP * sizeof(float2);
    const int nx = a.xslice ? 1 : (n + C::BR - 1) / C::BR;
    const unsigned xbytes = (unsigned)((a.xslice ? n : nx * C::BR) * TC * sizeof(float2));
    // thread 0 issues every copy; each first checks the copy rules (a
    // violation sets the error word and arms a barrier that never completes)
    auto load_rows = [&](int i, float2 *st, uint64_t *bar) {
        const int x0 = (i % TILES) * TC, r = i / TILES;
        if ((smem_u32(st) & 127u) != 0 || ((x0 * (int)sizeof(float2)) & 15) != 0) {
            if (a.err) atomicExch(a.err, 2);
            mbar_arrive_expect_tx(bar, 16u);
            return;
        }
        mbar_arrive_expect_tx(bar, xbytes + a.extra_tx);
        for (int q = 0; q < nx; q++) {
            if (a.xslice)
                tma_load_3d(st, &tmx, x0, 0, r * (n / a.xslice), bar);
            else
                tma_load_3d(st + (size_t)q * C::BR * TC, &tmx, x0, q * C::BR, r, bar);
        }
    };
    auto load_ghat = [&](int i) {
        if constexpr (C::PER) return;  // the spectrum is formed in the kernel
        const int x0 = (i % TILES) * TC;
        if ((smem_u32(GB) & 15u) != 0 || (GROW & 15u) != 0 || (reinterpret_cast<uintptr_t>(a.ghq) & 15u) != 0) {
            if (a.err) atomicExch(a.err, 2);
            mbar_arrive_expect_tx(&bars[2], 16u);
            return;
        }
        mbar_arrive_expect_tx(&bars[2], TC * GROW);
        for (int c = 0; c < TC; c++) {
            const int kx = x0 + c;
            const int kxq = kx <= M / 2 ? kx : M - kx;  // column kx of Ghat = quadrant row kxq
            bulk_load(GB + c * C::QSP, a.ghq + (size_t)kxq * C::QSP, GROW, &bars[2]);
        }
    };
    auto store_rows = [&](int i) {
        const int x0 = (i % TILES) * TC, r = i / TILES;
        for (int q = 0; q < nx; q++) {
            if (a.xslice)
                tma_store_3d(&tmw, x0, 0, r * (n / a.xslice), O);
            else
                tma_store_3d(&tmw, x0, q * C::BR, r, O + (size_t)q * C::BR * TC);
        }
        bulk_commit();
    };
    int cur = next_active(blockIdx.x);
    int nx1 = cur < total ? next_active(cur + gridDim.x) : total;
    bool fl0 = false, fl1 = false, flg = false;  // copies in flight into D[0], D[1], GB
    if (threadIdx.x == 0 && cur < total) {
        load_rows(cur, D0, &bars[0]);
        load_ghat(cur);
        if (nx1 < total) load_rows(nx1, D1, &bars[1]);
    }
    fl0 = cur < total;
    flg = !C::PER && cur < total;
    fl1 = nx1 < total;
    unsigned ph0 = 0u, ph1 = 0u, phg = 0u;
    // leave after a copy that never completed: let the others land (bounded),
    // let the stores finish; the error word is set
    auto bail = [&]() {
        if (threadIdx.x == 0) {
            if (fl0) mbar_wait_bounded(&bars[0], ph0, a.wait_ns, nullptr);
            if (fl1) mbar_wait_bounded(&bars[1], ph1, a.wait_ns, nullptr);
            if (flg) mbar_wait_bounded(&bars[2], phg, a.wait_ns, nullptr);
            bulk_wait_all();
        }
    };
    // two columns per thread: one interleaved exchange buffer, 16-byte accesses
    // (staggered: one buffer per column, block-wide named barriers 1 and 2)
    constexpr bool ILV = (L == 2 && !C::STAG);
    const Lines<L, ILV> sm{exch + L * cg * C::LSTRIDE, C::LSTRIDE};
    float2 *lineA = exch + L * cg * C::LSTRIDE, *lineB = lineA + C::LSTRIDE;
    const GroupSync syncA{1, C::THREADS}, syncB{2, C::THREADS};
    (void)lineB;
    for (int k = 0; cur < total; k++) {
        const int s = k & 1;
        float2 *st = s ? D1 : D0;
        const int nx2 = nx1 < total ? next_active(nx1 + gridDim.x) : total;
        const bool ok = mbar_wait_bounded(&bars[s], s ? ph1 : ph0, a.wait_ns, a.err);
        float2 v[L][E];
        col_load<C, M>(v, st, TC, n, t, L * cg);
        // periodic: O lies over the exchange lines, so the previous tile's
        // store must have read it before this tile's first exchange
        if constexpr (C::PER)
            if (threadIdx.x == 0) bulk_wait_read_all();
        // one barrier: every copy into D[s] checked, every read of it done
        if (__syncthreads_or(!ok)) {
            bail();
            return;
        }
        if (s) ph1 ^= 1u, fl1 = false;
        else ph0 ^= 1u, fl0 = false;
        if (threadIdx.x == 0 && nx2 < total) {
            fence_proxy_async_smem();
            load_rows(nx2, st, &bars[s]);
        }
        if (nx2 < total) {
            if (s) fl1 = true;
            else fl0 = true;
        }
        const int x0 = (cur % TILES) * TC;
        // the barrier above follows the previous tile's last exchange reads
        // (periodic: its output writes, and the store's read of them)
        constexpr bool ZIN = !C::PER;  // padded: rows >= N are zero
        if constexpr (C::STAG)
            fft_pair<M, E, -1, true, ZIN>(v[0], v[1], lineA, lineB, t, twr, syncA, syncB);
        else if constexpr (C::BLOCKED)
            fft_lines<M, E, -1, L, TWR, GroupSync, true, ZIN, ILV, C::RS>(v, sm, t, a.tw, &twr,
                                                                          GroupSync{1 + cg, T});
        else
            fft_lines<M, E, -1, L, TWR, BlockSync, true, ZIN, ILV, C::RS>(v, sm, t, a.tw, &twr);
        (void)x0;
        bool okg = true;
        if constexpr (C::PER) {
            // the spectrum from the integer wavenumbers; with the k-space
            // potential from the RHS's second term on (its first applies G only)
            auto multiply = [&](auto ks) {
                constexpr bool KS = decltype(ks)::value;
#pragma unroll
                for (int l = 0; l < L; l++) {
                    const int kx = x0 + L * cg + l;
                    const float ix = (float)(kx < M / 2 ? kx : kx - M);
#pragma unroll
                    for (int m = 0; m < E; m++) {
                        const int ky = t + T * m;
                        v[l][m] = cmul(v[l][m], periodic_spectrum<KS>(a, ix, (float)(ky < M / 2 ? ky : ky - M)));
                    }
                }
            };
            if constexpr (C::PERK == 2) {
                if (a.gate.st && a.gate.st[cur / TILES].terms > 0)
                    multiply(std::true_type{});
                else
                    multiply(std::false_type{});
            } else {
                multiply(std::false_type{});
            }
            // the forward transform's last exchange reads done
            __syncthreads();
        } else {
            okg = mbar_wait_bounded(&bars[2], phg, a.wait_ns, a.err);
#pragma unroll
            for (int l = 0; l < L; l++) {
                const float2 *gcol = GB + (L * cg + l) * C::QSP;
#pragma unroll
                for (int m = 0; m < E; m++) {
                    const int ky = t + T * m;
                    const float2 g = gcol[ky <= M / 2 ? ky : M - ky];
                    v[l][m] = CONJ ? cmulc(v[l][m], g) : cmul(v[l][m], g);
                }
            }
            if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tile's store has read O
            // one barrier: Ghat checked and read, O free, the forward transform's
            // last exchange reads done
            if (__syncthreads_or(!okg)) {
                bail();
                return;
            }
            phg ^= 1u;
            flg = false;
            if (threadIdx.x == 0 && nx1 < total) {
                fence_proxy_async_smem();
                load_ghat(nx1);
            }
            flg = nx1 < total;
        }
        if constexpr (C::STAG)
            fft_pair<M, E, +1, true, false>(v[0], v[1], lineA, lineB, t, twr, syncA, syncB);
        else if constexpr (C::BLOCKED)
            fft_lines<M, E, +1, L, TWR, GroupSync, true, false, ILV, C::RS>(v, sm, t, a.tw, &twr,
                                                                            GroupSync{1 + cg, T});
        else
            fft_lines<M, E, +1, L, TWR, BlockSync, true, false, ILV, C::RS>(v, sm, t, a.tw, &twr);
        // periodic: O is the exchange lines, free once every thread is past
        // the inverse transform's last exchange reads
        if constexpr (C::PER) __syncthreads();
#pragma unroll
        for (int m = 0; m < (C::PER ? E : E / 2); m++) {
            const int y = t + T * m;
            if (y < n) {
                if constexpr (L == 2) {  // both columns with one 16-byte store
                    *reinterpret_cast<float4 *>(O + (size_t)y * TC + 2 * cg) =
                        make_float4(v[0][m].x, v[0][m].y, v[1][m].x, v[1][m].y);
                } else {
#pragma unroll
                    for (int l = 0; l < L; l++) O[(size_t)y * TC + L * cg + l] = v[l][m];
                }
            }
        }
        fence_proxy_async_smem();  // this thread's output rows, for the tensor store
        __syncthreads();
        if (threadIdx.x == 0) store_rows(cur);
        cur = nx1;
        nx1 = nx2;
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int M>
static int row_persistent_blocks_per_sm() {
    static int nb = 0;  // per process: the kernel's resources do not change
    if (nb == 0) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, row_fwd_persistent_kernel<M>, RowPCfg<M>::THREADS,
                                                          RowPCfg<M>::SMEM) != cudaSuccess || q < 1)
            q = 1;
        nb = q;
    }
    return nb;
}

template <int M, bool KS>
static int row_eps_persistent_blocks_per_sm() {
    static int nb = 0;  // per process: the kernel's resources do not change
    if (nb == 0) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, row_eps_persistent_kernel<M, KS>, RowECfg<M>::THREADS,
                                                          RowECfg<M>::SMEM) != cudaSuccess || q < 1)
            q = 1;
        nb = q;
    }
    return nb;
}

template <int M, int KIND>
static cudaError_t row_launch(int nrhs, const RowArgs &a, cudaStream_t s) {
    using C = RowCfg<M>;
    RowArgs b = a;
    if (b.wait_ns == 0) b.wait_ns = 1000000000ull;  // 1 s
    if constexpr ((KIND == ROW_EPS || KIND == ROW_EPSK) && M >= 512) {
        if (a.n == M && a.num_sms > 0) {
            using P = RowECfg<M>;
            b.nrhs = nrhs;
            const int slots = nrhs * a.n;
            int grid = a.num_sms * row_eps_persistent_blocks_per_sm<M, KIND == ROW_EPSK>();
            if (grid * P::RPB > slots) grid = (slots + P::RPB - 1) / P::RPB;
            return launch_k(row_eps_persistent_kernel<M, KIND == ROW_EPSK>, dim3(grid), dim3(P::THREADS), P::SMEM, s,
                            a.pdl != 0, b);
        }
    }
    if constexpr (KIND == ROW_FWD && M >= 512) {
        if ((a.n & 1) == 0 && a.num_sms > 0) {
            using P = RowPCfg<M>;
            b.nrhs = nrhs;
            const int slots = nrhs * a.n;
            int grid = a.num_sms * row_persistent_blocks_per_sm<M>();
            if (grid * P::RPB > slots) grid = (slots + P::RPB - 1) / P::RPB;
            return launch_k(row_fwd_persistent_kernel<M>, dim3(grid), dim3(P::THREADS), P::SMEM, s, a.pdl != 0, b);
        }
    }
    dim3 grid((a.n + C::RPB - 1) / C::RPB, nrhs);
    return launch_k(row_kernel<M, KIND>, grid, dim3(C::THREADS), C::SMEM, s, a.pdl != 0, b);
}

template <int M>
static cudaError_t row_dispatch_kind(int kind, int nrhs, const RowArgs &a, cudaStream_t s) {
    switch (kind) {
    case ROW_SRC: return row_launch<M, ROW_SRC>(nrhs, a, s);
    case ROW_FWD: return row_launch<M, ROW_FWD>(nrhs, a, s);
    case ROW_ADJ: return row_launch<M, ROW_ADJ>(nrhs, a, s);
    case ROW_OUT: return row_launch<M, ROW_OUT>(nrhs, a, s);
    case ROW_VSRC: return row_launch<M, ROW_VSRC>(nrhs, a, s);
    case ROW_EPS: return row_launch<M, ROW_EPS>(nrhs, a, s);
    case ROW_EPSK: return row_launch<M, ROW_EPSK>(nrhs, a, s);
    }
    return cudaErrorInvalidValue;
}

// Rows per slice when X's N rows of one RHS are viewed as [N / d][d] (3D
// tensor map): the largest d <= br dividing n with n / d <= 256 (the box
// limit per dimension), or 0 when there is none (2D copies of br rows).
static int x_slice_rows(int n, int br) {
    for (int d = n < br ? n : br; d >= 1; d--)
        if (n % d == 0) return n / d <= 256 ? d : 0;
    return 0;
}

template <int M, bool CONJ, class C = ColCfg<M>>
static cudaError_t col_launch(int nrhs, const ColArgs &a, const ColMaps *maps, cudaStream_t s) {
    if (!maps) return cudaErrorInvalidValue;
    ColArgs b = a;
    b.nrhs = nrhs;
    b.xslice = x_slice_rows(a.n, C::BR);
    if (b.wait_ns == 0) b.wait_ns = 1000000000ull;  // 1 s
    const int tiles = (M / C::TC) * nrhs;
    if constexpr (C::PIPE) {
        const int grid = tiles < a.num_sms ? tiles : a.num_sms;
        return launch_k(col_pipe_kernel<M, CONJ, C::L, C::STAG, C::PERK, C::RS>, dim3(grid), dim3(C::THREADS), C::SMEM,
                        s, a.pdl != 0, b, maps->x, maps->w);
    } else {
        const int grid = tiles < a.num_sms ? tiles : a.num_sms;
        return launch_k(col_kernel<M, CONJ, C>, dim3(grid), dim3(C::THREADS), C::SMEM, s, a.pdl != 0, b, maps->x,
                        maps->w);
    }
}

// dispatch helper: F<shape>() for the shape of (M, variant)
template <int M, class F>
static cudaError_t with_col_variant(int variant, F f) {
    if (variant < 0 || variant >= col_variant_count(M)) return cudaErrorInvalidValue;
    const int kind = col_variant_kind(M, variant);
    if constexpr (col_has_pipe(M)) {
        if (kind == COL_P1) return f(ColPShape<M, 1>{});
        if (kind == COL_P2) return f(ColPShape<M, 2>{});
        if (kind == COL_P2S) return f(ColPShape<M, 2, true>{});
        if constexpr (M >= 4096)
            if (kind == COL_P2R8) return f(ColPShape<M, 2, false, 0, 1>{});
    }
    if (kind == COL_S0) return f(ColCfg<M>{});
    if constexpr (col_shape_count(M) > 1)
        if (kind == COL_S1) return f(typename ColVariant<M, 1>::type{});
    if constexpr (col_shape_count(M) > 2)
        if (kind == COL_S2) return f(typename ColVariant<M, 2>::type{});
    return cudaErrorInvalidValue;
}

// Tensor map of an [nrhs * n][M] complex64 buffer (X or W) in the column
// pass's tile geometry.  Elements are moved as opaque 8-byte words; rows are
// M elements apart.  With a slice size d (x_slice_rows) the map is the 3D
// view [nrhs * n / d][d][M] with a box of one RHS's n rows and TC columns;
// otherwise [nrhs][n][M] with boxes of BR rows, whose rows past n are
// zero-filled on loads and dropped on stores (the launcher passes the same
// x_slice_rows to the kernel).
template <class C>
static cudaError_t tile_tensor_map(CUtensorMap *map, const float2 *base, int n, int M, int nrhs) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int d = x_slice_rows(n, C::BR);
    const cuuint64_t row = (cuuint64_t)M * sizeof(float2);
    const cuuint32_t estr[3] = {1, 1, 1};
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3];
    if (d) {
        dims[0] = M, dims[1] = d, dims[2] = (cuuint64_t)nrhs * (n / d);
        strides[0] = row, strides[1] = row * d;
        box[0] = C::TC, box[1] = d, box[2] = n / d;
    } else {
        dims[0] = M, dims[1] = n, dims[2] = nrhs;
        strides[0] = row, strides[1] = row * n;
        box[0] = C::TC, box[1] = C::BR, box[2] = 1;
    }
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void *)base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// per-size entry points: defined here, instantiated for each M in one of the
// tbs_inst_*.cu files (so that the sizes compile in parallel) and called
// through the switches of tbs_kernels.cu
// ---------------------------------------------------------------------------
template <int M>
cudaError_t launch_row_m(int kind, int nrhs, const RowArgs &a, cudaStream_t s) {
    return row_dispatch_kind<M>(kind, nrhs, a, s);
}

// periodic plans: F<shape>() for (variant, k-space)
template <int M, class F>
static cudaError_t with_col_variant_per(int variant, bool ks, F f) {
    // fastest first as measured on GB300 at M = 4096: two columns per thread,
    // then one (the only shape below M = 32)
    if constexpr (col_periodic_variant_count(M) > 1) {
        if (variant == 0) return ks ? f(ColCfgPK2<M>{}) : f(ColCfgP2<M>{});
        if (variant == 1) return ks ? f(ColCfgPK<M>{}) : f(ColCfgP<M>{});
    } else {
        if (variant == 0) return ks ? f(ColCfgPK<M>{}) : f(ColCfgP<M>{});
    }
    if constexpr (col_periodic_variant_count(M) > 2) {
        if (variant == 2) return ks ? f(ColPShape<M, 2, false, 2>{}) : f(ColPShape<M, 2, false, 1>{});
        if (variant == 3) return ks ? f(ColPShape<M, 2, true, 2>{}) : f(ColPShape<M, 2, true, 1>{});
    }
    return cudaErrorInvalidValue;
}

template <int M>
cudaError_t col_tensor_maps_m(ColMaps *maps, const float2 *X, const float2 *W, int n, int nrhs, int variant,
                              bool periodic) {
    if (periodic)
        return with_col_variant_per<M>(variant, false, [&](auto c) {
            cudaError_t e = tile_tensor_map<decltype(c)>(&maps->x, X, n, M, nrhs);
            return e == cudaSuccess ? tile_tensor_map<decltype(c)>(&maps->w, W, n, M, nrhs) : e;
        });
    return with_col_variant<M>(variant, [&](auto c) {
        cudaError_t e = tile_tensor_map<decltype(c)>(&maps->x, X, n, M, nrhs);
        return e == cudaSuccess ? tile_tensor_map<decltype(c)>(&maps->w, W, n, M, nrhs) : e;
    });
}

template <int M>
cudaError_t launch_col_m(int nrhs, bool cj, const ColArgs &a, const ColMaps *maps, int variant, cudaStream_t s) {
    if (a.periodic) {  // forward spectrum only
        if (cj) return cudaErrorInvalidValue;
        return with_col_variant_per<M>(variant, a.kspace != 0,
                                       [&](auto c) { return col_launch<M, false, decltype(c)>(nrhs, a, maps, s); });
    }
    return with_col_variant<M>(variant, [&](auto c) {
        using CC = decltype(c);
        return cj ? col_launch<M, true, CC>(nrhs, a, maps, s) : col_launch<M, false, CC>(nrhs, a, maps, s);
    });
}

template <int M, class C = ColCfg<M>>
static int col_blocks_per_sm() {
    int nb = 0;
    cudaError_t e;
    if constexpr (C::PIPE)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, col_pipe_kernel<M, false, C::L, C::STAG, C::PERK, C::RS>,
                                                          C::THREADS, C::SMEM);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, col_kernel<M, false, C>, C::THREADS, C::SMEM);
    if (e != cudaSuccess) nb = 1;
    return nb > 0 ? nb : 1;
}

template <int M>
int col_resident_blocks_m(int variant, bool periodic) {
    int nb = 1;
    if (periodic) {
        with_col_variant_per<M>(variant, false, [&](auto c) {
            nb = col_blocks_per_sm<M, decltype(c)>();
            return cudaSuccess;
        });
        return nb;
    }
    with_col_variant<M>(variant, [&](auto c) {
        nb = col_blocks_per_sm<M, decltype(c)>();
        return cudaSuccess;
    });
    return nb;
}

template <int M, class C = ColCfg<M>>
static cudaError_t col_attr() {
    if constexpr (C::PIPE) {
        cudaError_t e = cudaFuncSetAttribute(col_pipe_kernel<M, false, C::L, C::STAG, C::PERK, C::RS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess || C::PERK) return e;  // the periodic grid has no adjoint pass
        return cudaFuncSetAttribute(col_pipe_kernel<M, true, C::L, C::STAG, 0, C::RS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    } else {
        cudaError_t e = cudaFuncSetAttribute(col_kernel<M, false, C>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(col_kernel<M, true, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)C::SMEM);
    }
}

template <int M>
cudaError_t set_col_smem_attr_m() {
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < col_variant_count(M) && e == cudaSuccess; v++)
        e = with_col_variant<M>(v, [&](auto c) { return col_attr<M, decltype(c)>(); });
    for (int v = 0; v < col_periodic_variant_count(M) && e == cudaSuccess; v++)
        for (int ks = 0; ks < 2 && e == cudaSuccess; ks++)
            e = with_col_variant_per<M>(v, ks != 0, [&](auto c) {
                using CC = decltype(c);
                if constexpr (CC::PIPE)
                    return col_attr<M, CC>();
                else
                    return cudaFuncSetAttribute(col_kernel<M, false, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)CC::SMEM);
            });
    return e;
}

template <int M>
static cudaError_t row_attr() {
    using C = RowCfg<M>;
    const int b = (int)C::SMEM;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_VSRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_EPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(row_kernel<M, ROW_EPSK>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    return cudaFuncSetAttribute(row_kernel<M, ROW_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

template <int M>
cudaError_t set_row_smem_attr_m() {
    cudaError_t e = row_attr<M>();
    if constexpr (M >= 512) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(row_fwd_persistent_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)RowPCfg<M>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(row_eps_persistent_kernel<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)RowECfg<M>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(row_eps_persistent_kernel<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)RowECfg<M>::SMEM);
    }
    return e;
}

#define TBS_FOR_EACH_M(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

// explicit instantiation (PRE empty) or its extern declaration (PRE extern)
#define TBS_PER_M(PRE, MM)                                                                              \
    PRE template cudaError_t launch_row_m<MM>(int, int, const RowArgs &, cudaStream_t);                 \
    PRE template cudaError_t col_tensor_maps_m<MM>(ColMaps *, const float2 *, const float2 *, int, int, \
                                                   int, bool);                                          \
    PRE template cudaError_t launch_col_m<MM>(int, bool, const ColArgs &, const ColMaps *, int,         \
                                              cudaStream_t);                                            \
    PRE template int col_resident_blocks_m<MM>(int, bool);                                              \
    PRE template cudaError_t set_col_smem_attr_m<MM>();                                                 \
    PRE template cudaError_t set_row_smem_attr_m<MM>();
}  // namespace tbs
