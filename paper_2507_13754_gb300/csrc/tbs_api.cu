// tbs_api.cu -- the C ABI declared in include/tbs.h.
//
// A plan owns every device buffer of one (N, k0, n_rhs) problem family:
// the spectrum quadrant Ghat, twiddles, V, the medium, the dense sources, the
// two N x M intermediates X and W, the partial sum psi, FP64 row partials and
// the per-RHS stop state.  A solve is
//
//     row pass on S  ->  { column pass, row pass, stop test } while active
//
// and the host never waits between terms.  tbs_solve captures it once into a
// CUDA graph (on a plan-owned stream) and replays it: the loop is a WHILE
// conditional node whose condition the stop test sets, so the graph runs the
// terms the slowest RHS needs (in bodies of four; launches past an RHS's stop
// return at once).  Without a graph (timing,
// TBS_FLAG_NO_GRAPH) the loop is unrolled max_terms times on the stream and
// launches after every RHS has stopped return at once.  Each launch checks
// its RHS's device flag, so an RHS that stopped early does no further work.
#include "tbs.h"
#include "tbs_internal.h"

#include <math.h>
#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

using namespace tbs;

namespace {

thread_local char g_err[512] = "";

tbs_status fail(tbs_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define TBS_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? TBS_ERR_OOM : TBS_ERR_CUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int padded_size_for(int n) {
    int m = 16;
    while (m < 2 * n - 1) m *= 2;
    return m;
}

int fft_size_for(const tbs_plan_desc *d) {
    return (d->flags & TBS_FLAG_PERIODIC) ? d->n : padded_size_for(d->n);
}

struct TimingRec {
    cudaEvent_t a, b;
    int col;  // 1: column pass, 0: row pass
};

}  // namespace

void tbs::set_last_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

struct tbs_plan_s {
    tbs_plan_desc d;
    int n = 0, M = 0, nrhs = 0, num_sms = 1;  // num_sms: SM count of the device
    double omega = 0, k0 = 0;
    // device buffers
    void *base = nullptr;            // every fixed-size buffer below is carved from it
    bool owns_base = false;          // false: caller's workspace (tbs_plan_with_workspace)
    float2 *tw = nullptr, *ghq = nullptr, *V = nullptr, *S = nullptr, *X = nullptr, *W = nullptr;
    float2 *psi = nullptr, *U = nullptr, *Q = nullptr, *G = nullptr;
    // TBS_FLAG_CHECKPOINT_TERMS: U holds every ck-th term ([ncp][rhs][N][N]),
    // Useg one recomputed segment ([ck][rhs][N][N]), Xs the recomputation's
    // row-pass output (the adjoint's own X is busy)
    int ck = 0, ncp = 0;
    bool periodic = false;           // TBS_FLAG_PERIODIC: M = N, spectrum in the kernel
    double eps = 0.0;                // epsilon of the periodic grid's Green's function
    bool cbs_auto = false;           // TBS_FLAG_CBS with eps_factor 0: eps chosen per medium
    float *abl = nullptr;            // per-axis absorbing-layer profile [N] (periodic)
    float2 *psi0 = nullptr;          // psi^0 per RHS (periodic, k-space potential)
    unsigned char *vflag = nullptr;  // periodic: per-row flags of V [N] and S [rhs][N]
    unsigned char *sflag = nullptr;
    float2 *Useg = nullptr, *Xs = nullptr;
    ColMaps cmaps_rc[MAX_COL_VARIANTS];             // Xs -> W tensor maps, per variant
    float *c = nullptr, *alpha = nullptr;
    double2 *part = nullptr, *l1 = nullptr;
    RhsState *state = nullptr;
    double *norms = nullptr;
    int *err = nullptr;              // device words: [0] error of bounded waits, [1..2] graph-loop control
    ColMaps cmaps[MAX_COL_VARIANTS];                // X and W tensor maps of the column pass, per variant
    int col_variant = 0;             // active column-pass tile shape
    int row_variant = 0;             // steady-state row pass: 0 persistent, 1 one block per row
    int col_grid[MAX_COL_VARIANTS] = {1, 1, 1, 1, 1, 1, 1, 1};     // persistent grid per variant
    unsigned long long wait_ns = 1000000000ull;
    unsigned extra_tx = 0;           // fault injection (tests)
    void *info_dev = nullptr;
    int *src_cell = nullptr, *src_seg = nullptr;
    float2 *src_amp = nullptr;
    int src_cap = 0;
    std::vector<int> h_cell, h_seg;      // host staging of the source upload
    std::vector<float2> h_amp;
    // medium bookkeeping
    bool have_medium = false, medium_from_c = false, have_alpha = false, have_sources = false;
    bool solved = false;
    double ypow = 1.0, fref = 0.0, tdel = 0.0;
    // graph
    cudaStream_t cap = nullptr;
    cudaStream_t body = nullptr;     // captures the body of the graph's term loop
    cudaGraphExec_t exec = nullptr;      // forward solve
    cudaGraphExec_t exec_adj = nullptr;  // adjoint sweep
    // timing
    bool timing = false;
    std::vector<TimingRec> tev;
    size_t tev_used = 0;
    double row_ms = 0, col_ms = 0;
    int row_n = 0, col_n = 0;
};

namespace {

RowArgs row_args(tbs_plan_s *p) {
    RowArgs a;
    memset(&a, 0, sizeof(a));
    a.W = p->W;
    a.src = p->S;
    a.X = p->X;
    a.psi = p->psi;
    a.V = p->V;
    a.U = (p->d.flags & TBS_FLAG_KEEP_TERMS) ? p->U : nullptr;
    const size_t nn = (size_t)p->n * p->n;
    if (p->ck) {  // checkpoints [ncp][rhs][N][N]: the forward stores every ck-th term
        a.u_rhs = nn;
        a.u_slot = (size_t)p->nrhs * nn;
        a.u_every = p->ck;
    } else {      // [rhs][max_terms][N][N]
        a.u_rhs = (size_t)p->d.max_terms * nn;
        a.u_slot = nn;
        a.u_every = 1;
    }
    a.u_term0 = 0;
    a.Q = p->Q;
    a.part = p->part;
    a.l1 = p->l1;
    a.tw = p->tw;
    a.gate.st = p->state;
    a.gate.mode = GATE_ALL;
    a.n = p->n;
    a.max_terms = p->d.max_terms;
    a.l1_row = p->d.stop_mode == TBS_STOP_L1_ROW ? p->d.l1_row : -1;
    a.abl = p->abl;
    a.psi0 = p->psi0;
    a.vflag = p->vflag;
    a.sflag = p->sflag;
    a.cbs_inv_eps = (p->d.flags & TBS_FLAG_CBS) ? (float)(1.0 / p->eps) : 0.f;
    a.err = p->err;
    a.wait_ns = p->wait_ns;
    a.num_sms = p->row_variant == 0 ? p->num_sms : 0;
    return a;
}

ColArgs col_args(tbs_plan_s *p) {
    ColArgs a;
    a.X = p->X;
    a.W = p->W;
    a.ghq = p->ghq;
    a.tw = p->tw;
    a.gate.st = p->state;
    a.gate.mode = GATE_ALL;
    a.gate.j = 0;
    a.gate.jdev = nullptr;
    a.pdl = 0;
    a.periodic = p->periodic;
    a.kq = a.eq = a.gs = 0.f;
    if (p->periodic) {
        const double dp = 2.0 * M_PI / (p->M * p->d.dx);
        a.kq = (float)(p->k0 * p->k0 / (dp * dp));
        a.eq = (float)(p->eps / (dp * dp));
        a.gs = (float)(1.0 / (dp * dp * (double)p->M * (double)p->M));
    }
    a.kspace = p->psi0 != nullptr;
    a.vv_a1 = a.vv_a2 = a.vv_eps = a.vv_half_nu = 0.f;
    if (a.kspace) {  // tau = -2 alpha0 c0^(nu-1), eta = 2 alpha0 c0^nu tan(pi nu / 2)
        const double dp = 2.0 * M_PI / (p->M * p->d.dx), nu = p->d.kspace_nu, a0 = p->d.kspace_alpha0;
        const double tau = -2.0 * a0 * pow(p->d.c0, nu - 1.0), eta = 2.0 * a0 * pow(p->d.c0, nu) * tan(M_PI * nu / 2.0);
        a.vv_a1 = p->d.kspace_absorption_only ? 0.f : (float)(eta * pow(dp, nu + 1.0));
        a.vv_a2 = (float)(tau * p->omega * pow(dp, nu));
        a.vv_eps = (float)p->eps;
        a.vv_half_nu = (float)(0.5 * nu);
    }
    a.n = p->n;
    a.nrhs = p->nrhs;
    a.num_sms = p->col_grid[p->col_variant];
    a.err = p->err;
    a.wait_ns = p->wait_ns;
    a.extra_tx = p->extra_tx;
    return a;
}

TimingRec *timing_slot(tbs_plan_s *p, int col) {
    if (p->tev_used == p->tev.size()) {
        TimingRec r;
        if (cudaEventCreate(&r.a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&r.b) != cudaSuccess) return nullptr;
        p->tev.push_back(r);
    }
    TimingRec *r = &p->tev[p->tev_used++];
    r->col = col;
    return r;
}

cudaError_t timed_row(tbs_plan_s *p, int kind, const RowArgs &a, cudaStream_t s) {
    // only the steady-state row passes (both transforms) are timed
    const bool steady = kind == ROW_FWD || kind == ROW_ADJ || kind == ROW_EPS || kind == ROW_EPSK;
    TimingRec *r = (p->timing && steady) ? timing_slot(p, 0) : nullptr;
    if (r) cudaEventRecord(r->a, s);
    cudaError_t e = launch_row(kind, p->M, p->nrhs, a, s);
    if (r) cudaEventRecord(r->b, s);
    return e;
}

cudaError_t timed_col(tbs_plan_s *p, bool cj, const ColArgs &a, cudaStream_t s) {
    TimingRec *r = p->timing ? timing_slot(p, 1) : nullptr;
    if (r) cudaEventRecord(r->a, s);
    cudaError_t e = launch_col(p->M, p->nrhs, cj, a, &p->cmaps[p->col_variant], p->col_variant, s);
    if (r) cudaEventRecord(r->b, s);
    return e;
}

// A condition for a WHILE node in the graph being captured on s; each
// launch of the graph resets it to 1.
tbs_status loop_condition(cudaStream_t s, cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    TBS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return fail(TBS_ERR_STATE, "graph loop outside a stream capture");
    TBS_CK(cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault));
    return TBS_OK;
}

// Appends a WHILE node on condition h to the graph being captured on s (after
// everything captured so far) and captures its body: body(p->body) enqueues
// one iteration on the plan's second stream, and one of its kernels sets h.
template <class Body>
tbs_status capture_while(tbs_plan_s *p, cudaStream_t s, cudaGraphConditionalHandle h, Body body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *dp = nullptr;
    size_t nd = 0;
    TBS_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &dp, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(TBS_ERR_STATE, "graph loop outside a stream capture");
    std::vector<cudaGraphNode_t> deps(dp, dp + nd);
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};  // aggregate: the rest zero
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    TBS_CK(cudaGraphAddNode(&node, g, deps.data(), nullptr, deps.size(), &np));
    cudaGraph_t bg = np.conditional.phGraph_out[0];
    TBS_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    TBS_CK(cudaStreamBeginCaptureToGraph(p->body, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = body(p->body);
    cudaGraph_t out = nullptr;  // bg again, owned by the node
    const cudaError_t e2 = cudaStreamEndCapture(p->body, &out);
    TBS_CK(e);
    TBS_CK(e2);
    return TBS_OK;
}

// Captures s into a graph with enqueue(s) and instantiates it into *exec.
template <class Enqueue>
tbs_status capture_graph(cudaStream_t s, cudaGraphExec_t *exec, Enqueue enqueue) {
    cudaGraph_t g = nullptr;
    TBS_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const tbs_status st = enqueue(s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != TBS_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    TBS_CK(e);
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    TBS_CK(e);
    return TBS_OK;
}

void drop_graphs(tbs_plan_s *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->exec_adj) cudaGraphExecDestroy(p->exec_adj);
    p->exec = p->exec_adj = nullptr;
}

tbs_status enqueue_solve(tbs_plan_s *p, cudaStream_t s, bool graph_loop) {
    TBS_CK(cudaMemsetAsync(p->state, 0, sizeof(RhsState) * p->nrhs, s));
    TBS_CK(cudaMemsetAsync(p->err, 0, 4 * sizeof(int), s));
    RowArgs ra = row_args(p);
    ColArgs ca = col_args(p);
    TBS_CK(timed_row(p, ROW_SRC, ra, s));
    StopArgs sa;
    sa.part = p->part;
    sa.l1 = p->l1;
    sa.st = p->state;
    sa.norms = p->norms;
    sa.n = p->n;
    sa.max_terms = p->d.max_terms;
    sa.tol = p->d.tol;
    sa.stop_mode = p->d.stop_mode;
    sa.div_grace = p->d.div_grace;
    sa.div_window = p->d.div_window;
    sa.div_factor = p->d.div_factor;
    sa.loop_ctl = nullptr;
    sa.loop = 0;
    // in the term loop the row pass and the stop test are programmatic
    // dependents of the kernel before them (their prologues overlap its tail)
    sa.pdl = 1;
    ra.pdl = 1;
    ra.gate.mode = GATE_FWD;
    ca.gate.mode = GATE_FWD;
    // the steady row pass: the term recurrence, or the paper's iteration on
    // psi on the periodic grid
    const int rk = !p->periodic ? ROW_FWD : p->psi0 ? ROW_EPSK : ROW_EPS;
    // which rows of V are one repeated value and which source rows are zero
    // (the medium and sources may change between solves of a plan)
    if (rk == ROW_EPS) TBS_CK(launch_row_flags(p->n, p->nrhs, p->V, p->S, p->vflag, p->sflag, s));
    if (graph_loop) {
        // The body runs TERMS_PER_ITERATION terms; each kernel reads its
        // RHS's term index from the RHS state and returns at once for an RHS
        // that has stopped.  The last stop test of the body sets the
        // condition (a WHILE iteration costs a few microseconds more than
        // the launches it holds, so the loop is unrolled).
        constexpr int TERMS_PER_ITERATION = 4;
        cudaGraphConditionalHandle h;
        tbs_status st = loop_condition(s, &h);
        if (st != TBS_OK) return st;
        ra.term = -1;
        sa.term = -1;
        st = capture_while(p, s, h, [&](cudaStream_t b) {
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < TERMS_PER_ITERATION && e == cudaSuccess; k++) {
                ColArgs ck = ca;
                ck.pdl = k > 0;  // follows the previous term's stop test
                StopArgs sk = sa;
                sk.loop = h;
                sk.loop_ctl = k == TERMS_PER_ITERATION - 1 ? p->err + 1 : nullptr;
                e = launch_col(p->M, p->nrhs, false, ck, &p->cmaps[p->col_variant], p->col_variant, b);
                if (e == cudaSuccess) e = launch_row(rk, p->M, p->nrhs, ra, b);
                if (e == cudaSuccess) e = launch_stop(p->nrhs, sk, b);
            }
            return e;
        });
        if (st != TBS_OK) return st;
    } else {
        for (int t = 0; t < p->d.max_terms; t++) {
            TBS_CK(timed_col(p, false, ca, s));
            ra.term = t;
            // the last admissible term runs the inverse transform only: not
            // a steady-state row pass, so it is not timed
            if (t == p->d.max_terms - 1)
                TBS_CK(launch_row(rk, p->M, p->nrhs, ra, s));
            else
                TBS_CK(timed_row(p, rk, ra, s));
            sa.term = t;
            TBS_CK(launch_stop(p->nrhs, sa, s));
        }
    }
    TBS_CK(launch_info(p->nrhs, p->state, p->err, p->info_dev, s));
    return TBS_OK;
}

// Reverse sweep of the truncated series (the plan's stored terms u_j):
// ubar_{T-1} = g; for j = T-2 .. 0: lambda = G^H ubar_{j+1}, Q += conj(lambda)
// u_j, ubar_j = g + conj(V) lambda, with T the RHS's own term count.  In a
// graph the steps are a WHILE node whose counter starts at max_r T_r - 2.
tbs_status enqueue_adjoint(tbs_plan_s *p, cudaStream_t s, bool graph_loop) {
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemsetAsync(p->Q, 0, sizeof(float2) * p->nrhs * nn, s));
    RowArgs ra = row_args(p);
    ra.src = p->G;
    ColArgs ca = col_args(p);
    TBS_CK(timed_row(p, ROW_SRC, ra, s));  // X = FFT_x(ubar_{T-1} = g)
    ra.pdl = 1;  // the reverse steps' row passes follow their column passes programmatically
    ra.gate.mode = GATE_ADJ;
    ca.gate.mode = GATE_ADJ;
    if (graph_loop) {
        int *jdev = p->err + 3;
        cudaGraphConditionalHandle h;
        tbs_status st = loop_condition(s, &h);
        if (st != TBS_OK) return st;
        TBS_CK(launch_adj_loop(p->nrhs, p->state, jdev, h, true, s));
        ra.term = -1;
        ra.gate.j = ca.gate.j = -1;
        ra.gate.jdev = ca.gate.jdev = jdev;
        return capture_while(p, s, h, [&](cudaStream_t b) {
            cudaError_t e = launch_col(p->M, p->nrhs, true, ca, &p->cmaps[p->col_variant], p->col_variant, b);
            if (e == cudaSuccess) e = launch_row(ROW_ADJ, p->M, p->nrhs, ra, b);
            if (e == cudaSuccess) e = launch_adj_loop(p->nrhs, p->state, jdev, h, false, b);
            return e;
        });
    }
    for (int j = p->d.max_terms - 2; j >= 0; j--) {
        ca.gate.j = j;
        ra.gate.j = j;
        ra.term = j;
        TBS_CK(timed_col(p, true, ca, s));
        // step 0 runs the inverse transform only: not timed
        if (j == 0)
            TBS_CK(launch_row(ROW_ADJ, p->M, p->nrhs, ra, s));
        else
            TBS_CK(timed_row(p, ROW_ADJ, ra, s));
    }
    return TBS_OK;
}

// The reverse sweep with checkpointed terms (TBS_FLAG_CHECKPOINT_TERMS):
// for each segment of ck steps, from the last down, the segment's terms are
// recomputed from its checkpoint (u_{j+1} = G (V u_j): row pass on V u_j into
// Xs, column pass, inverse row pass into Useg) and then consumed by the
// reverse steps.  The recomputation runs the forward pass's arithmetic on the
// same values, so the terms are bitwise those of the forward solve.  tmax:
// the largest term count over the RHS.
tbs_status enqueue_adjoint_ckpt(tbs_plan_s *p, cudaStream_t s, int tmax) {
    const size_t nn = (size_t)p->n * p->n, slot = (size_t)p->nrhs * nn;
    TBS_CK(cudaMemsetAsync(p->Q, 0, sizeof(float2) * slot, s));
    RowArgs ra = row_args(p);
    ra.src = p->G;
    ColArgs ca = col_args(p);
    TBS_CK(timed_row(p, ROW_SRC, ra, s));  // X = FFT_x(ubar_{T-1} = g)
    ra.gate.mode = GATE_ADJ;
    ca.gate.mode = GATE_ADJ;
    ra.U = p->Useg;
    ra.u_rhs = nn;
    ra.u_slot = slot;
    ra.u_every = 1;
    RowArgs rv = row_args(p), ro = row_args(p);
    ro.U = rv.U = nullptr;
    rv.X = p->Xs;
    ColArgs cr = col_args(p);
    const int K = p->ck, jtop = tmax - 2;
    for (int c = jtop >= 0 ? jtop / K : -1; c >= 0; c--) {
        const int j0 = c * K, j1 = std::min(j0 + K - 1, jtop);
        TBS_CK(cudaMemcpyAsync(p->Useg, p->U + (size_t)c * slot, sizeof(float2) * slot, cudaMemcpyDeviceToDevice, s));
        for (int k = 1; k <= j1 - j0; k++) {
            rv.src = p->Useg + (size_t)(k - 1) * slot;
            TBS_CK(launch_row(ROW_VSRC, p->M, p->nrhs, rv, s));
            TBS_CK(launch_col(p->M, p->nrhs, false, cr, &p->cmaps_rc[p->col_variant], p->col_variant, s));
            ro.psi = p->Useg + (size_t)k * slot;
            TBS_CK(launch_row(ROW_OUT, p->M, p->nrhs, ro, s));
        }
        ra.u_term0 = j0;
        for (int j = j1; j >= j0; j--) {
            ca.gate.j = ra.gate.j = ra.term = j;
            TBS_CK(timed_col(p, true, ca, s));
            TBS_CK(launch_row(ROW_ADJ, p->M, p->nrhs, ra, s));
        }
    }
    return TBS_OK;
}

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_plan(tbs_plan_s *p) {
    drop_graphs(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->body) cudaStreamDestroy(p->body);
    for (auto &r : p->tev) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (p->owns_base && p->base) cudaFree(p->base);
    void *bufs[] = {p->src_cell, p->src_seg, p->src_amp};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
}

}  // namespace

extern "C" {

void tbs_plan_desc_init(tbs_plan_desc *d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->n_rhs = 1;
    d->max_terms = 64;
    d->tol = 1e-6;
    d->stop_mode = TBS_STOP_L2;
    d->l1_row = -1;
    d->div_grace = 8;
    d->div_window = 4;
    d->div_factor = 1e6;
    d->eps_factor = 0.8;
}

// Fixed-size device buffers of a plan, carved from one block at 256-byte
// aligned offsets (the order of the enum); U, Q, G only with KEEP_TERMS.
enum PlanBuf { B_TW, B_GHQ, B_V, B_C, B_ALPHA, B_S, B_PSI, B_X, B_W, B_PART, B_L1, B_STATE,
               B_NORMS, B_INFO, B_ERR, B_U, B_Q, B_G, B_USEG, B_XS, B_ABL, B_PSI0, B_FLAGS, B_COUNT };

// checkpoint spacing K = ceil(sqrt(max_terms)) and the number of checkpoints
static int ckpt_every(int max_terms) {
    int k = 1;
    while (k * k < max_terms) k++;
    return k;
}
struct PlanLayout {
    size_t off[B_COUNT];
    size_t total;
};

static PlanLayout plan_layout(const tbs_plan_desc *d) {
    const size_t n = d->n, M = fft_size_for(d), r = d->n_rhs, nn = n * n, T = d->max_terms;
    const bool per = (d->flags & TBS_FLAG_PERIODIC) != 0;
    const bool keep = (d->flags & TBS_FLAG_KEEP_TERMS) != 0;
    size_t sz[B_COUNT];
    sz[B_TW] = M * sizeof(float2);
    sz[B_GHQ] = per ? 0 : (M / 2 + 1) * (size_t)ghat_stride((int)M) * sizeof(float2);
    sz[B_ABL] = per ? M * sizeof(float) : 0;
    sz[B_PSI0] = (d->flags & TBS_FLAG_KSPACE_ABSORPTION) ? r * nn * sizeof(float2) : 0;
    sz[B_FLAGS] = per ? (size_t)(1 + r) * d->n : 0;
    sz[B_V] = nn * sizeof(float2);
    sz[B_C] = nn * sizeof(float);
    sz[B_ALPHA] = nn * sizeof(float);
    sz[B_S] = r * nn * sizeof(float2);
    sz[B_PSI] = r * nn * sizeof(float2);
    sz[B_X] = r * n * M * sizeof(float2);
    sz[B_W] = r * n * M * sizeof(float2);
    sz[B_PART] = r * n * sizeof(double2);
    sz[B_L1] = r * sizeof(double2);
    sz[B_STATE] = r * sizeof(RhsState);
    sz[B_NORMS] = r * T * sizeof(double);
    sz[B_INFO] = r * sizeof(tbs_solve_info);
    sz[B_ERR] = 4 * sizeof(int);
    const bool ckpt = keep && (d->flags & TBS_FLAG_CHECKPOINT_TERMS);
    const size_t K = ckpt ? ckpt_every(d->max_terms) : 0, ncp = ckpt ? (T + K - 1) / K : 0;
    sz[B_U] = keep ? (ckpt ? ncp : T) * r * nn * sizeof(float2) : 0;
    sz[B_USEG] = ckpt ? K * r * nn * sizeof(float2) : 0;
    sz[B_XS] = ckpt ? r * n * M * sizeof(float2) : 0;
    sz[B_Q] = keep ? r * nn * sizeof(float2) : 0;
    sz[B_G] = keep ? r * nn * sizeof(float2) : 0;
    PlanLayout L;
    size_t o = 0;
    for (int b = 0; b < B_COUNT; b++) {
        L.off[b] = o;
        o += (sz[b] + 255) & ~(size_t)255;
    }
    L.total = o;
    return L;
}

static tbs_status check_desc(const tbs_plan_desc *d) {
    if (!d) return fail(TBS_ERR_INVALID_ARG, "desc is NULL");
    if (d->n < 2 || d->n > ((d->flags & TBS_FLAG_PERIODIC) ? TBS_MAX_N_PERIODIC : TBS_MAX_N))
        return fail(TBS_ERR_UNSUPPORTED_SIZE, "n = %d outside [2, %d]", d->n,
                    (d->flags & TBS_FLAG_PERIODIC) ? TBS_MAX_N_PERIODIC : TBS_MAX_N);
    if (!(d->dx > 0) || !(d->freq_hz > 0) || !(d->c0 > 0))
        return fail(TBS_ERR_INVALID_ARG, "dx, freq_hz and c0 must be > 0");
    if (d->n_rhs < 1 || d->n_rhs > 65535) return fail(TBS_ERR_INVALID_ARG, "n_rhs = %d", d->n_rhs);
    if (d->max_terms < 1 || d->max_terms > TBS_MAX_TERMS_CAP)
        return fail(TBS_ERR_INVALID_ARG, "max_terms = %d", d->max_terms);
    if (!(d->tol >= 0)) return fail(TBS_ERR_INVALID_ARG, "tol must be >= 0");
    if (d->stop_mode != TBS_STOP_L2 && d->stop_mode != TBS_STOP_L1_ROW)
        return fail(TBS_ERR_INVALID_ARG, "stop_mode = %d", d->stop_mode);
    if (d->l1_row >= d->n) return fail(TBS_ERR_INVALID_ARG, "l1_row = %d >= n", d->l1_row);
    if (d->div_window < 1 || d->div_grace < 0 || !(d->div_factor > 0))
        return fail(TBS_ERR_INVALID_ARG, "bad divergence parameters");
    if ((d->flags & TBS_FLAG_CHECKPOINT_TERMS) && !(d->flags & TBS_FLAG_KEEP_TERMS))
        return fail(TBS_ERR_INVALID_ARG, "TBS_FLAG_CHECKPOINT_TERMS needs TBS_FLAG_KEEP_TERMS");
    if (d->flags & TBS_FLAG_PERIODIC) {
        if (d->n < 16 || d->n > TBS_MAX_N_PERIODIC || (d->n & (d->n - 1)))
            return fail(TBS_ERR_UNSUPPORTED_SIZE, "periodic grid: n = %d must be a power of two in [16, %d]",
                        d->n, TBS_MAX_N_PERIODIC);
        if (d->flags & TBS_FLAG_KEEP_TERMS)
            return fail(TBS_ERR_INVALID_ARG, "periodic grid: no term storage (the iteration is on psi)");
        if (!(d->eps_factor > 0) && !((d->flags & TBS_FLAG_CBS) && d->eps_factor == 0))
            return fail(TBS_ERR_INVALID_ARG, "eps_factor must be > 0 (or 0 with TBS_FLAG_CBS: chosen from the medium)");
        if (d->abl_width < 0 || d->abl_width > d->n / 2 || (d->abl_width > 0 && !(d->abl_zeta > 0)))
            return fail(TBS_ERR_INVALID_ARG, "absorbing layer: 0 <= abl_width <= n/2 and abl_zeta > 0");
        if ((d->flags & TBS_FLAG_KSPACE_ABSORPTION) &&
            (!(d->kspace_alpha0 >= 0) || !(d->kspace_nu > 0 && d->kspace_nu < 3) ||
             (d->kspace_absorption_only != 0 && d->kspace_absorption_only != 1)))
            return fail(TBS_ERR_INVALID_ARG, "k-space potential: alpha0 >= 0, 0 < nu < 3, absorption_only 0 or 1");
        if ((d->flags & TBS_FLAG_CBS) && (d->flags & TBS_FLAG_KSPACE_ABSORPTION))
            return fail(TBS_ERR_INVALID_ARG, "TBS_FLAG_CBS applies to spatial potentials, not the k-space one");
    } else if (d->flags & (TBS_FLAG_KSPACE_ABSORPTION | TBS_FLAG_CBS)) {
        return fail(TBS_ERR_INVALID_ARG, "TBS_FLAG_KSPACE_ABSORPTION and TBS_FLAG_CBS need TBS_FLAG_PERIODIC");
    }
    return TBS_OK;
}

tbs_status tbs_plan_device_bytes(const tbs_plan_desc *d, size_t *bytes) {
    tbs_status st = check_desc(d);
    if (st != TBS_OK) return st;
    if (!bytes) return fail(TBS_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = plan_layout(d).total;
    return TBS_OK;
}

static tbs_status plan_create(const tbs_plan_desc *d, void *workspace, size_t workspace_bytes, void *stream,
                              tbs_plan_t *out) {
    tbs_status st = check_desc(d);
    if (st != TBS_OK) return st;
    if (!out) return fail(TBS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const PlanLayout lay = plan_layout(d);
    if (workspace) {
        if (reinterpret_cast<uintptr_t>(workspace) & 255)
            return fail(TBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        if (workspace_bytes < lay.total)
            return fail(TBS_ERR_INVALID_ARG, "workspace of %zu bytes < %zu (tbs_plan_device_bytes)",
                        workspace_bytes, lay.total);
        if (!is_device_ptr(workspace)) return fail(TBS_ERR_INVALID_ARG, "workspace must be device memory");
    }
    cudaStream_t s = (cudaStream_t)stream;
    tbs_plan_s *p = new tbs_plan_s();
    p->d = *d;
    if (p->d.stop_mode == TBS_STOP_L1_ROW && p->d.l1_row < 0) p->d.l1_row = d->n / 2;
    p->n = d->n;
    p->M = fft_size_for(d);
    p->periodic = (d->flags & TBS_FLAG_PERIODIC) != 0;
    p->nrhs = d->n_rhs;
    p->omega = 2.0 * M_PI * d->freq_hz;
    p->k0 = p->omega / d->c0;
    p->eps = p->periodic ? d->eps_factor * p->k0 * p->k0 : 0.0;
    p->cbs_auto = p->periodic && (d->flags & TBS_FLAG_CBS) && d->eps_factor == 0;
    const size_t n = p->n, M = p->M, r = p->nrhs, nn = n * n;
    cudaError_t e = cudaSuccess;
    if (workspace) {
        p->base = workspace;
    } else {
        e = cudaMalloc(&p->base, lay.total);
        p->owns_base = (e == cudaSuccess);
    }
    if (e == cudaSuccess) {
        char *b = static_cast<char *>(p->base);
        auto at = [&](int k) { return static_cast<void *>(b + lay.off[k]); };
        p->tw = (float2 *)at(B_TW);
        p->ghq = (float2 *)at(B_GHQ);
        p->V = (float2 *)at(B_V);
        p->c = (float *)at(B_C);
        p->alpha = (float *)at(B_ALPHA);
        p->S = (float2 *)at(B_S);
        p->psi = (float2 *)at(B_PSI);
        p->X = (float2 *)at(B_X);
        p->W = (float2 *)at(B_W);
        p->part = (double2 *)at(B_PART);
        p->l1 = (double2 *)at(B_L1);
        p->state = (RhsState *)at(B_STATE);
        p->norms = (double *)at(B_NORMS);
        p->info_dev = at(B_INFO);
        p->err = (int *)at(B_ERR);
        if (p->periodic) p->abl = (float *)at(B_ABL);
        if (d->flags & TBS_FLAG_KSPACE_ABSORPTION) p->psi0 = (float2 *)at(B_PSI0);
        if (p->periodic) {
            p->vflag = (unsigned char *)at(B_FLAGS);
            p->sflag = p->vflag + d->n;
        }
        if (d->flags & TBS_FLAG_KEEP_TERMS) {
            p->U = (float2 *)at(B_U);
            p->Q = (float2 *)at(B_Q);
            p->G = (float2 *)at(B_G);
            if (d->flags & TBS_FLAG_CHECKPOINT_TERMS) {
                p->ck = ckpt_every(d->max_terms);
                p->ncp = (d->max_terms + p->ck - 1) / p->ck;
                p->Useg = (float2 *)at(B_USEG);
                p->Xs = (float2 *)at(B_XS);
            }
        }
    }
    if (e != cudaSuccess) {
        free_plan(p);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? TBS_ERR_OOM : TBS_ERR_CUDA,
                    "plan allocation failed: %s", cudaGetErrorString(e));
    }
    // periodic grid: the absorbing layer's per-axis profile, the sigmoid
    // 1 / (1 + exp(-zeta (x - mu/2))) at distance x from the nearer edge
    // within mu = abl_width cells (Section 3.1), 1 elsewhere
    std::vector<float> abl_host(p->periodic ? p->M : 0, 1.f);
    for (int i = 0; p->periodic && i < p->M; i++) {
        const int edge = std::min(i, p->M - 1 - i);
        if (edge < d->abl_width) {
            const double mu = d->abl_width * d->dx;
            abl_host[i] = (float)(1.0 / (1.0 + exp(-d->abl_zeta * (edge * d->dx - 0.5 * mu))));
        }
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) == cudaSuccess)
        e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int v = 0; e == cudaSuccess && v < col_variants(p->M, p->periodic); v++) {
        e = col_tensor_maps(&p->cmaps[v], p->X, p->W, p->n, p->M, p->nrhs, v, p->periodic);
        if (e == cudaSuccess && p->Xs) e = col_tensor_maps(&p->cmaps_rc[v], p->Xs, p->W, p->n, p->M, p->nrhs, v);
    }
    if (e == cudaSuccess && (e = set_row_smem_attr(p->M)) == cudaSuccess && (e = set_col_smem_attr(p->M)) == cudaSuccess &&
        ([&] {
            for (int v = 0; v < col_variants(p->M, p->periodic); v++)
                p->col_grid[v] = p->num_sms * col_resident_blocks_per_sm(p->M, v, p->periodic);
            return true;
        })() &&
        (e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&p->body, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = build_twiddles(p->M, p->tw, s)) == cudaSuccess &&
        (p->periodic || (e = build_ghat(p->n, p->M, p->k0, d->dx, p->ghq, s)) == cudaSuccess) &&
        (!p->periodic || (e = cudaMemcpyAsync(p->abl, abl_host.data(), sizeof(float) * p->M,
                                              cudaMemcpyHostToDevice, s)) == cudaSuccess) &&
        (e = cudaMemsetAsync(p->state, 0, r * sizeof(RhsState), s)) == cudaSuccess &&
        (e = cudaMemsetAsync(p->err, 0, 4 * sizeof(int), s)) == cudaSuccess &&
        (e = cudaMemsetAsync(p->psi, 0, r * nn * sizeof(float2), s)) == cudaSuccess) {
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        free_plan(p);
        cudaGetLastError();
        return fail(TBS_ERR_CUDA, "plan build failed: %s", cudaGetErrorString(e));
    }
    *out = p;
    return TBS_OK;
}

tbs_status tbs_plan(const tbs_plan_desc *d, void *stream, tbs_plan_t *out) {
    return plan_create(d, nullptr, 0, stream, out);
}

tbs_status tbs_plan_with_workspace(const tbs_plan_desc *d, void *workspace, size_t workspace_bytes, void *stream,
                                   tbs_plan_t *out) {
    if (!workspace) return fail(TBS_ERR_INVALID_ARG, "workspace is NULL");
    return plan_create(d, workspace, workspace_bytes, stream, out);
}

int32_t tbs_plan_padded_size(tbs_plan_t p) { return p ? p->M : 0; }

// max |U| over the plan's potential, U = V + i eps (synchronous on s)
static tbs_status potential_max_abs(tbs_plan_s *p, cudaStream_t s, double *out) {
    const int nn = p->n * p->n;
    unsigned long long *bits = reinterpret_cast<unsigned long long *>(p->part);  // scratch outside a solve
    TBS_CK(launch_potential_max(nn, p->V, p->eps, bits, s));
    unsigned long long h = 0;
    TBS_CK(cudaMemcpyAsync(&h, bits, sizeof(h), cudaMemcpyDeviceToHost, s));
    TBS_CK(cudaStreamSynchronize(s));
    memcpy(out, &h, sizeof(h));
    return TBS_OK;
}

// A TBS_FLAG_CBS plan made with eps_factor = 0 chooses eps from each medium:
// eps = CBS_EPS_MARGIN max |U|, just above the convergence bound eps >= max|U|
// of the convergent Born series.  V holds U (unshifted) on entry.
static constexpr double CBS_EPS_MARGIN = 1.01;
static tbs_status cbs_auto_eps(tbs_plan_s *p, cudaStream_t s) {
    const double eps_old = p->eps;
    p->eps = 0.0;
    double umax = 0.0;
    tbs_status st = potential_max_abs(p, s, &umax);
    if (st != TBS_OK) return st;
    if (!(umax > 0) || !std::isfinite(umax))
        return fail(TBS_ERR_INVALID_ARG, "automatic CBS epsilon: max |U| = %g (a zero or non-finite medium)", umax);
    p->eps = CBS_EPS_MARGIN * umax;
    if (p->eps != eps_old) drop_graphs(p);  // kernel parameters derived from eps changed
    return TBS_OK;
}

tbs_status tbs_set_medium(tbs_plan_t p, const float *c, const float *alpha, double y_pow,
                          double f_ref_hz, void *stream) {
    if (!p || !c) return fail(TBS_ERR_INVALID_ARG, "plan and c must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemcpyAsync(p->c, c, nn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (alpha) TBS_CK(cudaMemcpyAsync(p->alpha, alpha, nn * sizeof(float), cudaMemcpyDeviceToDevice, s));
    p->have_alpha = alpha != nullptr;
    p->ypow = y_pow;
    p->fref = f_ref_hz;
    double tdel = 0.0;
    if (alpha) {
        const double delta = f_ref_hz > 0 ? 1.0 - pow(f_ref_hz / p->d.freq_hz, y_pow - 1.0) : 1.0;
        tdel = tan(M_PI * y_pow / 2.0) * delta;
    }
    p->tdel = tdel;
    if (p->cbs_auto) {
        TBS_CK(launch_medium((int)nn, p->c, alpha ? p->alpha : nullptr, p->omega, p->d.c0, tdel, 0.0, p->V, s));
        tbs_status st = cbs_auto_eps(p, s);
        if (st != TBS_OK) return st;
        TBS_CK(launch_shift_potential((int)nn, p->eps, p->V, s));  // U - i eps
    } else {
        TBS_CK(launch_medium((int)nn, p->c, alpha ? p->alpha : nullptr, p->omega, p->d.c0, tdel, p->eps, p->V, s));
    }
    p->have_medium = true;
    p->medium_from_c = true;
    return TBS_OK;
}

tbs_status tbs_set_potential(tbs_plan_t p, const float *V, void *stream) {
    if (!p || !V) return fail(TBS_ERR_INVALID_ARG, "plan and V must not be NULL");
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemcpyAsync(p->V, V, nn * sizeof(float2), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (p->cbs_auto) {
        tbs_status st = cbs_auto_eps(p, (cudaStream_t)stream);
        if (st != TBS_OK) return st;
    }
    if (p->periodic) TBS_CK(launch_shift_potential((int)nn, p->eps, p->V, (cudaStream_t)stream));  // U - i eps
    p->have_medium = true;
    p->medium_from_c = false;
    return TBS_OK;
}

tbs_status tbs_set_sources(tbs_plan_t p, int32_t n_pts, const int32_t *ix, const int32_t *iy,
                           const float *amp, void *stream) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (n_pts < 0) return fail(TBS_ERR_INVALID_ARG, "n_pts < 0");
    if (n_pts > 0 && (!ix || !iy || !amp)) return fail(TBS_ERR_INVALID_ARG, "NULL source arrays");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n;
    for (int j = 0; j < n_pts; j++)
        if (ix[j] < 0 || ix[j] >= n || iy[j] < 0 || iy[j] >= n)
            return fail(TBS_ERR_INVALID_ARG, "source %d at (%d, %d) outside the %d x %d grid", j,
                        ix[j], iy[j], n, n);
    // group elements by cell (bookkeeping only; the sums run on the device)
    std::vector<int> perm(n_pts);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        return (int64_t)iy[a] * n + ix[a] < (int64_t)iy[b] * n + ix[b];
    });
    std::vector<int> &cell = p->h_cell, &seg = p->h_seg;
    cell.clear();
    seg.clear();
    for (int k = 0; k < n_pts; k++) {
        const int ci = iy[perm[k]] * n + ix[perm[k]];
        if (cell.empty() || cell.back() != ci) {
            cell.push_back(ci);
            seg.push_back(k);
        }
    }
    seg.push_back(n_pts);
    std::vector<float2> &amps = p->h_amp;
    amps.assign((size_t)p->nrhs * n_pts, make_float2(0.f, 0.f));
    const float2 *a2 = (const float2 *)amp;
    for (int r = 0; r < p->nrhs; r++)
        for (int k = 0; k < n_pts; k++) amps[(size_t)r * n_pts + k] = a2[(size_t)r * n_pts + perm[k]];
    if (n_pts > p->src_cap) {
        cudaFree(p->src_cell);
        cudaFree(p->src_seg);
        cudaFree(p->src_amp);
        p->src_cell = nullptr;
        p->src_seg = nullptr;
        p->src_amp = nullptr;
        p->src_cap = 0;
        TBS_CK(cudaMalloc(&p->src_cell, sizeof(int) * n_pts));
        TBS_CK(cudaMalloc(&p->src_seg, sizeof(int) * (n_pts + 1)));
        TBS_CK(cudaMalloc(&p->src_amp, sizeof(float2) * (size_t)p->nrhs * n_pts));
        p->src_cap = n_pts;
    }
    const size_t nn = (size_t)n * n;
    TBS_CK(cudaMemsetAsync(p->S, 0, sizeof(float2) * p->nrhs * nn, s));
    if (n_pts > 0) {
        TBS_CK(cudaMemcpyAsync(p->src_cell, cell.data(), sizeof(int) * cell.size(), cudaMemcpyHostToDevice, s));
        TBS_CK(cudaMemcpyAsync(p->src_seg, seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice, s));
        TBS_CK(cudaMemcpyAsync(p->src_amp, amps.data(), sizeof(float2) * amps.size(), cudaMemcpyHostToDevice, s));
        TBS_CK(launch_deposit(p->nrhs, n, (int)cell.size(), p->src_cell, p->src_seg, p->src_amp, n_pts,
                              1.0 / (p->d.dx * p->d.dx), p->S, s));
    }
    p->have_sources = true;
    return TBS_OK;
}

tbs_status tbs_set_source_field(tbs_plan_t p, const float *S, void *stream) {
    if (!p || !S) return fail(TBS_ERR_INVALID_ARG, "plan and S must not be NULL");
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemcpyAsync(p->S, S, sizeof(float2) * p->nrhs * nn, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
    p->have_sources = true;
    return TBS_OK;
}

tbs_status tbs_set_harmonic2_source(tbs_plan_t p, const float *psi1, const float *beta,
                                    const float *rho, const float *c, double omega_fundamental,
                                    void *stream) {
    if (!p || !psi1 || !beta || !rho || !c)
        return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_set_harmonic2_source");
    const int count = p->n * p->n;
    TBS_CK(launch_harmonic2(p->nrhs, count, (const float2 *)psi1, beta, rho, c, omega_fundamental, p->S,
                            (cudaStream_t)stream));
    p->have_sources = true;
    return TBS_OK;
}

tbs_status tbs_set_harmonic_source(tbs_plan_t p, int32_t order, const float *const *psi_lower,
                                   const double *psi_scale, const float *beta, const float *rho, const float *c,
                                   double omega_fundamental, double source_scale, void *stream) {
    if (!p || !psi_lower || !beta || !rho || !c)
        return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_set_harmonic_source");
    if (order < 2 || order > 5) return fail(TBS_ERR_INVALID_ARG, "order = %d outside [2, 5]", order);
    if (!(source_scale > 0) || !std::isfinite(source_scale))
        return fail(TBS_ERR_INVALID_ARG, "source_scale must be finite and > 0");
    HarmonicInputs in;
    memset(&in, 0, sizeof(in));
    for (int k = 0; k < order - 1; k++) {
        if (!psi_lower[k]) return fail(TBS_ERR_INVALID_ARG, "psi_lower[%d] is NULL", k);
        in.psi[k] = (const float2 *)psi_lower[k];
        in.scale[k] = psi_scale ? psi_scale[k] : 1.0;
        if (!(in.scale[k] > 0) || !std::isfinite(in.scale[k]))
            return fail(TBS_ERR_INVALID_ARG, "psi_scale[%d] must be finite and > 0", k);
    }
    in.source_scale = source_scale;
    TBS_CK(launch_harmonic(p->nrhs, p->n * p->n, order, in, beta, rho, c, omega_fundamental, p->S,
                           (cudaStream_t)stream));
    p->have_sources = true;
    return TBS_OK;
}

tbs_status tbs_solve(tbs_plan_t p, float *psi, tbs_solve_info *info, void *stream) {
    if (!p || !psi || !info) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_solve");
    if (!p->have_medium) return fail(TBS_ERR_STATE, "no medium: call tbs_set_medium or tbs_set_potential");
    if (!p->have_sources) return fail(TBS_ERR_STATE, "no sources: call tbs_set_sources first");
    cudaStream_t s = (cudaStream_t)stream;
    const bool use_graph = !p->timing && !(p->d.flags & TBS_FLAG_NO_GRAPH);
    if (use_graph) {
        if (!p->exec) {
            tbs_status st = capture_graph(p->cap, &p->exec, [&](cudaStream_t c) { return enqueue_solve(p, c, true); });
            if (st != TBS_OK) return st;
        }
        TBS_CK(cudaGraphLaunch(p->exec, s));
    } else {
        tbs_status st = enqueue_solve(p, s, false);
        if (st != TBS_OK) return st;
    }
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemcpyAsync(psi, p->psi, sizeof(float2) * p->nrhs * nn, cudaMemcpyDeviceToDevice, s));
    TBS_CK(cudaMemcpyAsync(info, p->info_dev, sizeof(tbs_solve_info) * p->nrhs,
                           is_device_ptr(info) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    p->solved = true;
    return TBS_OK;
}

}  // extern "C"

struct tbs_batch_s {
    std::vector<tbs_plan_s *> plans;
    cudaStream_t origin = nullptr;
    std::vector<cudaEvent_t> events;  // fork + one join per plan
    cudaGraphExec_t exec = nullptr;
};

static void free_batch(tbs_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

extern "C" {

tbs_status tbs_batch_create(const tbs_plan_t *plans, int32_t n_plans, float *const *psi,
                            tbs_solve_info *const *info, tbs_batch_t *out) {
    if (!plans || !psi || !info || !out || n_plans < 1)
        return fail(TBS_ERR_INVALID_ARG, "tbs_batch_create: NULL argument or n_plans < 1");
    *out = nullptr;
    for (int i = 0; i < n_plans; i++) {
        if (!plans[i] || !psi[i] || !info[i]) return fail(TBS_ERR_INVALID_ARG, "tbs_batch_create: NULL entry %d", i);
        if (!is_device_ptr(info[i]))
            return fail(TBS_ERR_INVALID_ARG, "tbs_batch_create: info[%d] must be device memory", i);
        if (plans[i]->timing) return fail(TBS_ERR_STATE, "tbs_batch_create: plan %d has timing enabled", i);
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return fail(TBS_ERR_INVALID_ARG, "tbs_batch_create: plan %d repeated", i);
    }
    tbs_batch_s *b = new tbs_batch_s();
    b->plans.assign(plans, plans + n_plans);
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i <= n_plans; i++) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->events.push_back(ev);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return fail(TBS_ERR_CUDA, "tbs_batch_create: %s", cudaGetErrorString(e));
    }
    cudaGraph_t g = nullptr;
    tbs_status st = TBS_OK;
    e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->events[0], b->origin);
    for (int i = 0; e == cudaSuccess && st == TBS_OK && i < n_plans; i++) {
        tbs_plan_s *p = b->plans[i];
        const size_t nn = (size_t)p->n * p->n;
        if ((e = cudaStreamWaitEvent(p->cap, b->events[0], 0)) != cudaSuccess) break;
        if ((st = enqueue_solve(p, p->cap, true)) != TBS_OK) break;
        if ((e = cudaMemcpyAsync(psi[i], p->psi, sizeof(float2) * p->nrhs * nn, cudaMemcpyDeviceToDevice,
                                 p->cap)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(info[i], p->info_dev, sizeof(tbs_solve_info) * p->nrhs,
                                 cudaMemcpyDeviceToDevice, p->cap)) != cudaSuccess)
            break;
        if ((e = cudaEventRecord(b->events[i + 1], p->cap)) != cudaSuccess) break;
        e = cudaStreamWaitEvent(b->origin, b->events[i + 1], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == TBS_OK) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != TBS_OK || e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return st != TBS_OK ? st : fail(TBS_ERR_CUDA, "tbs_batch_create: capture failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return TBS_OK;
}

tbs_status tbs_batch_solve(tbs_batch_t b, void *stream) {
    if (!b) return fail(TBS_ERR_INVALID_ARG, "batch is NULL");
    for (size_t i = 0; i < b->plans.size(); i++) {
        tbs_plan_s *p = b->plans[i];
        if (!p->have_medium || !p->have_sources)
            return fail(TBS_ERR_STATE, "tbs_batch_solve: plan %zu has no medium or no sources", i);
    }
    TBS_CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    for (tbs_plan_s *p : b->plans) p->solved = true;
    return TBS_OK;
}

tbs_status tbs_batch_destroy(tbs_batch_t b) {
    if (!b) return fail(TBS_ERR_INVALID_ARG, "batch is NULL");
    free_batch(b);
    return TBS_OK;
}

tbs_status tbs_solve_adjoint(tbs_plan_t p, const float *grad_psi, float *grad_c, float *grad_alpha,
                             void *stream) {
    if (!p || !grad_psi) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_solve_adjoint");
    if (!(p->d.flags & TBS_FLAG_KEEP_TERMS))
        return fail(TBS_ERR_STATE, "the plan was created without TBS_FLAG_KEEP_TERMS");
    if (!p->solved) return fail(TBS_ERR_STATE, "no forward solve to differentiate");
    if (!p->medium_from_c) return fail(TBS_ERR_STATE, "medium not set by tbs_set_medium");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nn = (size_t)p->n * p->n;
    TBS_CK(cudaMemsetAsync(p->err, 0, sizeof(int), s));  // read back by tbs_device_error
    TBS_CK(cudaMemcpyAsync(p->G, grad_psi, sizeof(float2) * p->nrhs * nn, cudaMemcpyDeviceToDevice, s));
    const bool use_graph = !p->timing && !(p->d.flags & TBS_FLAG_NO_GRAPH);
    if (p->ck) {
        std::vector<RhsState> st(p->nrhs);
        TBS_CK(cudaMemcpyAsync(st.data(), p->state, sizeof(RhsState) * p->nrhs, cudaMemcpyDeviceToHost, s));
        TBS_CK(cudaStreamSynchronize(s));
        int tmax = 0;
        for (const RhsState &r : st) tmax = std::max(tmax, r.terms);
        tbs_status st2 = enqueue_adjoint_ckpt(p, s, tmax);
        if (st2 != TBS_OK) return st2;
    } else if (use_graph) {
        if (!p->exec_adj) {
            tbs_status st = capture_graph(p->cap, &p->exec_adj, [&](cudaStream_t c) { return enqueue_adjoint(p, c, true); });
            if (st != TBS_OK) return st;
        }
        TBS_CK(cudaGraphLaunch(p->exec_adj, s));
    } else {
        tbs_status st = enqueue_adjoint(p, s, false);
        if (st != TBS_OK) return st;
    }
    if (grad_c || grad_alpha)
        TBS_CK(launch_gradient(p->nrhs, (int)nn, p->Q, p->c, p->have_alpha ? p->alpha : nullptr, p->omega,
                               p->tdel, grad_c, grad_alpha, s));
    return TBS_OK;
}

tbs_status tbs_apply_green(tbs_plan_t p, const float *f, float *out, int32_t conj_kernel, void *stream) {
    if (!p || !f || !out) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_apply_green");
    if (f == out) return fail(TBS_ERR_INVALID_ARG, "f and out may not alias");
    cudaStream_t s = (cudaStream_t)stream;
    TBS_CK(cudaMemsetAsync(p->err, 0, sizeof(int), s));  // read back by tbs_device_error
    RowArgs ra = row_args(p);
    ra.src = (const float2 *)f;
    ra.psi = (float2 *)out;
    ColArgs ca = col_args(p);
    TBS_CK(timed_row(p, ROW_SRC, ra, s));
    TBS_CK(timed_col(p, conj_kernel != 0, ca, s));
    TBS_CK(timed_row(p, ROW_OUT, ra, s));
    return TBS_OK;
}

tbs_status tbs_potential_max_abs(tbs_plan_t p, double *out_host, void *stream) {
    if (!p || !out_host) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_potential_max_abs");
    if (!p->have_medium) return fail(TBS_ERR_STATE, "no medium: call tbs_set_medium or tbs_set_potential");
    return potential_max_abs(p, (cudaStream_t)stream, out_host);
}

double tbs_plan_eps(tbs_plan_t p) { return p ? p->eps : 0.0; }

tbs_status tbs_device_error(tbs_plan_t p, int32_t *code, void *stream) {
    if (!p || !code) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_device_error");
    int h = 0;
    TBS_CK(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TBS_CK(cudaStreamSynchronize((cudaStream_t)stream));
    *code = h == 1 ? TBS_WAIT_TIMEOUT : h == 2 ? TBS_COPY_CHECK_FAILED : 0;
    return TBS_OK;
}

tbs_status tbs_get_ghat(tbs_plan_t p, float *out_host) {
    if (!p || !out_host) return fail(TBS_ERR_INVALID_ARG, "NULL argument to tbs_get_ghat");
    if (p->periodic) return fail(TBS_ERR_STATE, "periodic plan: the spectrum is formed in the kernel");
    const size_t q = (size_t)(p->M / 2 + 1);
    TBS_CK(cudaMemcpy2D(out_host, q * sizeof(float2), p->ghq, (size_t)ghat_stride(p->M) * sizeof(float2),
                        q * sizeof(float2), q, cudaMemcpyDeviceToHost));
    return TBS_OK;
}

tbs_status tbs_set_timing(tbs_plan_t p, int32_t enable) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    p->timing = enable != 0;
    p->tev_used = 0;
    p->row_ms = p->col_ms = 0;
    p->row_n = p->col_n = 0;
    return TBS_OK;
}

tbs_status tbs_get_timing(tbs_plan_t p, double *row_ms, int32_t *row_launches, double *col_ms,
                          int32_t *col_launches) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    for (size_t i = 0; i < p->tev_used; i++) {
        float ms = 0.f;
        TBS_CK(cudaEventSynchronize(p->tev[i].b));
        TBS_CK(cudaEventElapsedTime(&ms, p->tev[i].a, p->tev[i].b));
        if (p->tev[i].col) {
            p->col_ms += ms;
            p->col_n++;
        } else {
            p->row_ms += ms;
            p->row_n++;
        }
    }
    p->tev_used = 0;
    if (row_ms) *row_ms = p->row_ms;
    if (row_launches) *row_launches = p->row_n;
    if (col_ms) *col_ms = p->col_ms;
    if (col_launches) *col_launches = p->col_n;
    return TBS_OK;
}

int32_t tbs_col_variants(tbs_plan_t p) { return p ? col_variants(p->M, p->periodic) : 0; }

const char *tbs_col_variant_name(tbs_plan_t p, int32_t variant) {
    if (!p) return nullptr;
    return col_variant_name(p->M, p->periodic, variant < 0 ? p->col_variant : variant);
}

tbs_status tbs_set_col_variant(tbs_plan_t p, int32_t variant) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (variant < 0 || variant >= tbs_col_variants(p))
        return fail(TBS_ERR_INVALID_ARG, "variant %d outside [0, %d)", variant, tbs_col_variants(p));
    if (variant != p->col_variant) drop_graphs(p);
    p->col_variant = variant;
    return TBS_OK;
}

tbs_status tbs_autotune(tbs_plan_t p, int32_t reps, double *times_ms, int32_t *best, void *stream) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (reps < 1) return fail(TBS_ERR_INVALID_ARG, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    TBS_CK(cudaEventCreate(&e0));
    TBS_CK(cudaEventCreate(&e1));
    const int nv = tbs_col_variants(p);
    int bi = 0;
    double bt = 1e300;
    for (int v = 0; v < nv; v++) {
        ColArgs ca = col_args(p);
        ca.num_sms = p->col_grid[v];
        cudaError_t e = launch_col(p->M, p->nrhs, false, ca, &p->cmaps[v], v, s);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; e == cudaSuccess && r < reps; r++) e = launch_col(p->M, p->nrhs, false, ca, &p->cmaps[v], v, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(TBS_ERR_CUDA, "tbs_autotune: %s", cudaGetErrorString(e));
        }
        const double t = ms / reps;
        if (times_ms) times_ms[v] = t;
        if (t < bt) {
            bt = t;
            bi = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best) *best = bi;
    return tbs_set_col_variant(p, bi);
}

int32_t tbs_row_variants(tbs_plan_t p) {
    if (!p) return 0;
    // the persistent steady-state passes exist for M >= 512 with an even N
    // (padded grid) or N = M (periodic grid)
    const bool persistent = p->M >= 512 && (p->periodic ? p->n == p->M : (p->n & 1) == 0);
    return persistent ? 2 : 1;
}

const char *tbs_row_variant_name(tbs_plan_t p, int32_t variant) {
    if (!p) return nullptr;
    if (variant < 0) variant = p->row_variant;
    if (variant >= tbs_row_variants(p)) return nullptr;
    if (tbs_row_variants(p) == 1) return "one block per row";
    return variant == 0 ? "persistent, rows prefetched a row ahead" : "one block per row";
}

tbs_status tbs_set_row_variant(tbs_plan_t p, int32_t variant) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (variant < 0 || variant >= tbs_row_variants(p))
        return fail(TBS_ERR_INVALID_ARG, "variant %d outside [0, %d)", variant, tbs_row_variants(p));
    if (variant != p->row_variant) drop_graphs(p);
    p->row_variant = variant;
    return TBS_OK;
}

tbs_status tbs_autotune_rows(tbs_plan_t p, int32_t reps, double *times_ms, int32_t *best, void *stream) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (reps < 1) return fail(TBS_ERR_INVALID_ARG, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int nv = tbs_row_variants(p);
    const int rk = !p->periodic ? ROW_FWD : p->psi0 ? ROW_EPSK : ROW_EPS;
    // The steady pass accumulates into psi: the timed launches write a
    // scratch field instead of the plan's result, and store no terms.
    const size_t bytes = (size_t)p->nrhs * p->n * p->n * sizeof(float2);
    float2 *scratch = nullptr;
    TBS_CK(cudaMalloc(&scratch, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && rk == ROW_EPS) e = launch_row_flags(p->n, p->nrhs, p->V, p->S, p->vflag, p->sflag, s);
    int bi = 0;
    double bt = 1e300;
    for (int v = 0; e == cudaSuccess && v < nv; v++) {
        RowArgs ra = row_args(p);
        ra.num_sms = v == 0 && nv > 1 ? p->num_sms : 0;
        ra.psi = scratch;
        ra.U = nullptr;
        ra.term = 1;  // a steady-state term: inverse transform, epilogue, forward transform
        ra.l1_row = -1;
        ra.gate.mode = GATE_ALL;
        e = launch_row(rk, p->M, p->nrhs, ra, s);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; e == cudaSuccess && r < reps; r++) e = launch_row(rk, p->M, p->nrhs, ra, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double t = ms / reps;
        if (times_ms) times_ms[v] = t;
        if (t < bt) {
            bt = t;
            bi = v;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const cudaError_t ef = cudaFree(scratch);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return fail(TBS_ERR_CUDA, "tbs_autotune_rows: %s", cudaGetErrorString(e));
    if (best) *best = bi;
    return tbs_set_row_variant(p, bi);
}

tbs_status tbs_debug_set(tbs_plan_t p, int32_t key, int64_t value) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    if (key == TBS_DEBUG_WAIT_LIMIT_NS) {
        if (value <= 0) return fail(TBS_ERR_INVALID_ARG, "wait limit must be > 0");
        p->wait_ns = (unsigned long long)value;
    } else if (key == TBS_DEBUG_EXTRA_TX) {
        if (value < 0 || value > (1 << 20)) return fail(TBS_ERR_INVALID_ARG, "extra_tx out of range");
        p->extra_tx = (unsigned)value;
    } else {
        return fail(TBS_ERR_INVALID_ARG, "unknown debug key %d", key);
    }
    drop_graphs(p);  // kernel arguments changed: recapture on the next solve
    return TBS_OK;
}

tbs_status tbs_destroy(tbs_plan_t p) {
    if (!p) return fail(TBS_ERR_INVALID_ARG, "plan is NULL");
    free_plan(p);
    return TBS_OK;
}

const char *tbs_status_string(tbs_status s) {
    switch (s) {
    case TBS_OK: return "TBS_OK";
    case TBS_ERR_INVALID_ARG: return "TBS_ERR_INVALID_ARG";
    case TBS_ERR_UNSUPPORTED_SIZE: return "TBS_ERR_UNSUPPORTED_SIZE";
    case TBS_ERR_OOM: return "TBS_ERR_OOM";
    case TBS_ERR_CUDA: return "TBS_ERR_CUDA";
    case TBS_ERR_STATE: return "TBS_ERR_STATE";
    }
    return "TBS_ERR_UNKNOWN";
}

const char *tbs_last_error(void) { return g_err; }

}  // extern "C"
