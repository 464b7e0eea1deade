// tbs_synth.cu -- broadband synthesis: the time signal at a lattice of
// receivers from a set of single-frequency fields (one per frequency of a
// sweep, each on its own grid over the same physical domain):
//     s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t)
// (e^{-i omega t} convention of the outgoing Green's function, Section 2.2).
//
// One block takes SY_RB receivers of one right-hand side: it first gathers
// the weighted bilinear samples w_k psi_k(X_r) of its receivers into shared
// memory, then each thread produces time samples t_j, forming each phase
// factor once for all SY_RB receivers.  Phases f_k t_j are reduced modulo
// one cycle in FP64 (f t reaches thousands of cycles, beyond FP32's
// resolution), the rest is FP32.  Frequencies go in chunks of SY_CHUNK per
// launch (the per-frequency table rides in the kernel parameters, so the
// call allocates nothing); later chunks add to the output.
#include "tbs.h"
#include "tbs_internal.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

namespace {

constexpr int SY_CHUNK = 64;     // frequencies per launch
constexpr int SY_RB = 8;         // receivers per block
constexpr int SY_THREADS = 256;

struct SynthArgs {
    const float2 *field[SY_CHUNK];
    double dx[SY_CHUNK];
    double f[SY_CHUNK];
    float w[SY_CHUNK];
    int n[SY_CHUNK];
    int count;       // frequencies in this chunk
    int accumulate;  // add to out (chunks after the first)
    int nx, ny, n_t;
    double x0, y0, sx, sy, t0, dt;
    float2 *out;
};
static_assert(sizeof(SynthArgs) <= 4000, "kernel parameter space");

// fractional cell index of coordinate p on a grid of n cell centres i * dx,
// clamped to [0, n - 1]; i0 <= n - 2 so that i0 + 1 is a cell too
__device__ __forceinline__ void cell_of(double p, double dx, int n, int &i0, float &fr) {
    const double u = fmin(fmax(p / dx, 0.0), (double)(n - 1));
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    i0 = i;
    fr = (float)(u - (double)i);
}

__global__ void __launch_bounds__(SY_THREADS) synth_kernel(const __grid_constant__ SynthArgs a) {
    __shared__ float2 A[SY_RB][SY_CHUNK];
    const int nr = a.nx * a.ny;
    const int r0 = blockIdx.x * SY_RB;
    const int rhs = blockIdx.y;
    for (int idx = threadIdx.x; idx < SY_RB * SY_CHUNK; idx += SY_THREADS) {
        const int rr = idx / SY_CHUNK, k = idx % SY_CHUNK;
        const int r = r0 + rr;
        float2 s = make_float2(0.f, 0.f);
        if (r < nr && k < a.count) {
            const int n = a.n[k];
            int i0, j0;
            float fx, fy;
            cell_of(a.x0 + (double)(r % a.nx) * a.sx, a.dx[k], n, i0, fx);
            cell_of(a.y0 + (double)(r / a.nx) * a.sy, a.dx[k], n, j0, fy);
            const float2 *p = a.field[k] + ((size_t)rhs * n + j0) * n + i0;
            const float2 p00 = p[0], p01 = p[1], p10 = p[n], p11 = p[n + 1];
            const float ax = 1.f - fx, ay = 1.f - fy;
            const float re = ay * (ax * p00.x + fx * p01.x) + fy * (ax * p10.x + fx * p11.x);
            const float im = ay * (ax * p00.y + fx * p01.y) + fy * (ax * p10.y + fx * p11.y);
            s = make_float2(a.w[k] * re, a.w[k] * im);
        }
        A[rr][k] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < a.n_t; j += SY_THREADS) {
        const double t = a.t0 + (double)j * a.dt;
        float2 acc[SY_RB];
#pragma unroll
        for (int rr = 0; rr < SY_RB; rr++) acc[rr] = make_float2(0.f, 0.f);
        for (int k = 0; k < a.count; k++) {
            const double cyc = a.f[k] * t;
            const float ph = (float)(cyc - rint(cyc));  // in [-1/2, 1/2] cycles
            float sn, cs;
            sincospif(2.f * ph, &sn, &cs);  // exp(-2 pi i ph) = cs - i sn
#pragma unroll
            for (int rr = 0; rr < SY_RB; rr++) {
                const float2 v = A[rr][k];
                acc[rr].x = fmaf(v.x, cs, fmaf(v.y, sn, acc[rr].x));
                acc[rr].y = fmaf(v.y, cs, fmaf(-v.x, sn, acc[rr].y));
            }
        }
#pragma unroll
        for (int rr = 0; rr < SY_RB; rr++) {
            if (r0 + rr >= nr) break;
            float2 *o = a.out + ((size_t)rhs * nr + (r0 + rr)) * a.n_t + j;
            if (a.accumulate) {
                const float2 prev = *o;
                *o = make_float2(prev.x + acc[rr].x, prev.y + acc[rr].y);
            } else {
                *o = acc[rr];
            }
        }
    }
}

tbs_status sy_fail(tbs_status s, const char *msg) {
    tbs::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" tbs_status tbs_synthesize(const tbs_synth_freq *freqs, int32_t n_freq, int32_t n_rhs, double x0,
                                     double y0, double sx, double sy, int32_t nx, int32_t ny, double t0, double dt,
                                     int32_t n_t, float *out, void *stream) {
    if (!freqs || !out) return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: NULL pointer");
    if (n_freq < 1 || n_rhs < 1 || n_rhs > 65535 || nx < 1 || ny < 1 || n_t < 1)
        return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: counts must be >= 1 (n_rhs <= 65535)");
    if ((long long)nx * ny > (1ll << 30))
        return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: more than 2^30 receivers");
    if (!isfinite(x0) || !isfinite(y0) || !isfinite(sx) || !isfinite(sy) || !isfinite(t0) || !isfinite(dt))
        return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: receiver lattice and times must be finite");
    for (int k = 0; k < n_freq; k++) {
        const tbs_synth_freq &q = freqs[k];
        if (!q.field || q.n < 2 || !(q.dx > 0) || !isfinite(q.dx) || !isfinite(q.freq_hz) || !isfinite(q.weight))
            return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: bad frequency entry (field, n >= 2, dx > 0, finite)");
        if ((const void *)q.field == (const void *)out)
            return sy_fail(TBS_ERR_INVALID_ARG, "tbs_synthesize: out may not alias a field");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nr = nx * ny;
    const dim3 grid((nr + SY_RB - 1) / SY_RB, n_rhs);
    for (int c = 0; c < n_freq; c += SY_CHUNK) {
        SynthArgs a;
        memset(&a, 0, sizeof(a));
        a.count = n_freq - c < SY_CHUNK ? n_freq - c : SY_CHUNK;
        for (int k = 0; k < a.count; k++) {
            const tbs_synth_freq &q = freqs[c + k];
            a.field[k] = (const float2 *)q.field;
            a.dx[k] = q.dx;
            a.f[k] = q.freq_hz;
            a.w[k] = (float)q.weight;
            a.n[k] = q.n;
        }
        a.accumulate = c > 0;
        a.nx = nx;
        a.ny = ny;
        a.n_t = n_t;
        a.x0 = x0;
        a.y0 = y0;
        a.sx = sx;
        a.sy = sy;
        a.t0 = t0;
        a.dt = dt;
        a.out = (float2 *)out;
        synth_kernel<<<grid, SY_THREADS, 0, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof(buf), "tbs_synthesize: launch failed: %s", cudaGetErrorString(e));
            return sy_fail(TBS_ERR_CUDA, buf);
        }
    }
    return TBS_OK;
}
