// tbs_plan.cu -- plan-time tables: FFT twiddles and the spectrum of the
// cell-averaged free-space Green's function.
//
// The operator G of arxiv 2507.13754 (Section 2.2: G = F^-1 g~ F below
// Eq. 17) is realised with the free-space Green's function of Eq. 16 at
// epsilon -> 0, g(r) = (i/4) H0^(1)(k0 r) = (i/4) J0(k0 r) - (1/4) Y0(k0 r),
// averaged over each cell:
//     Gc[d] = (1/dx^2) * integral over cell d of g(|r|) d^2r.
// Everything here runs in FP64 (J0 and Y0 are CUDA's j0/y0); only the final
// spectrum is rounded to complex64.
//
//  * Cells with max(|a|,|b|) >= 4: 6 x 6 tensor Gauss-Legendre; the nearest
//    singularity is >= 3.5 cells away, so the rule is exact to ~1e-14.
//  * 1 <= max(|a|,|b|) <= 3: 16 x 16 tensor Gauss-Legendre.
//  * The self cell: subtract the logarithm.  Near r = 0,
//    Y0(z) = (2/pi)(ln(z/2) + gamma) J0(z) + O(z^2), so
//    g_s(r) = g(r) + ln(r)/(2 pi) is continuous; its mean is integrated in
//    polar coordinates over the 8 triangles of the square (24 x 24 points),
//    and the mean of ln r over a square of side h has the closed form
//    ln(h/2) + (ln 2 - 3 + pi/2)/2.
//
// The table is wrapped into M x M (offset d at index d mod M, zero where no
// pair of grid cells has that offset), transformed in FP64 (radix-2
// Stockham, rows, transpose, rows, transpose back), scaled by dx^2/M^2 and the
// quadrant 0 <= kx, ky <= M/2 is stored (the spectrum is even in both axes).
#include "tbs_fft.cuh"
#include "tbs_internal.h"

#include <math.h>
#include <stdio.h>
#include <vector>

namespace tbs {

#define TBS_NQ_SELF 24
#define TBS_NQ_NEAR 16
#define TBS_NQ_FAR 6

__constant__ double c_gl_self_x[TBS_NQ_SELF], c_gl_self_w[TBS_NQ_SELF];
__constant__ double c_gl_near_x[TBS_NQ_NEAR], c_gl_near_w[TBS_NQ_NEAR];
__constant__ double c_gl_far_x[TBS_NQ_FAR], c_gl_far_w[TBS_NQ_FAR];

// Gauss-Legendre rule on [-1, 1] by Newton's method on the Legendre
// polynomial, evaluated with Bonnet's recurrence; initial guesses from the
// asymptotic formula cos(pi (4i + 3) / (4n + 2)).
static void gauss_legendre_rule(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double pkm1 = 1.0, pk = z;  // P_0, P_1
            for (int k = 1; k < n; k++) {
                const double pkp1 = ((2.0 * k + 1.0) * z * pk - k * pkm1) / (k + 1.0);
                pkm1 = pk;
                pk = pkp1;
            }
            if (n == 1) { pk = z; pkm1 = 1.0; }
            dp = n * (pkm1 - z * pk) / (1.0 - z * z);
            const double step = pk / dp;
            z -= step;
            if (fabs(step) < 1e-15) {
                // refresh the derivative at the final node
                double a = 1.0, b = z;
                for (int k = 1; k < n; k++) {
                    const double c = ((2.0 * k + 1.0) * z * b - k * a) / (k + 1.0);
                    a = b;
                    b = c;
                }
                if (n == 1) { b = z; a = 1.0; }
                dp = n * (a - z * b) / (1.0 - z * z);
                break;
            }
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

__device__ __forceinline__ double2 green_fp64(double k0, double r) {
    const double z = k0 * r;
    return make_double2(-0.25 * y0(z), 0.25 * j0(z));
}

__global__ void green_quadrant_kernel(int n, double k0, double dx, double2 *__restrict__ gc) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a >= n) return;
    double re = 0.0, im = 0.0;
    if (a == 0 && b == 0) {
        const double inv2pi = 1.0 / (2.0 * M_PI);
        const double mean_ln = log(0.5 * dx) + 0.5 * (log(2.0) - 3.0 + 0.5 * M_PI);
        double sre = 0.0, sim = 0.0;
        for (int p = 0; p < TBS_NQ_SELF; p++) {
            const double th = (c_gl_self_x[p] + 1.0) * (M_PI / 8.0);
            const double wth = c_gl_self_w[p] * (M_PI / 8.0);
            const double R = 0.5 * dx / cos(th);
            double ire = 0.0, iim = 0.0;
            for (int q = 0; q < TBS_NQ_SELF; q++) {
                const double r = 0.5 * R * (c_gl_self_x[q] + 1.0);
                const double wr = 0.5 * R * c_gl_self_w[q];
                const double2 g = green_fp64(k0, r);
                ire += wr * r * (g.x + log(r) * inv2pi);
                iim += wr * r * g.y;
            }
            sre += wth * ire;
            sim += wth * iim;
        }
        re = -inv2pi * mean_ln + 8.0 * sre / (dx * dx);
        im = 8.0 * sim / (dx * dx);
    } else {
        const bool near = (a <= 3 && b <= 3);
        const int nq = near ? TBS_NQ_NEAR : TBS_NQ_FAR;
        const double *gx = near ? c_gl_near_x : c_gl_far_x;
        const double *gw = near ? c_gl_near_w : c_gl_far_w;
        for (int i = 0; i < nq; i++) {
            const double px = (a + 0.5 * gx[i]) * dx;
            double rre = 0.0, rim = 0.0;
            for (int j = 0; j < nq; j++) {
                const double py = (b + 0.5 * gx[j]) * dx;
                const double2 g = green_fp64(k0, sqrt(px * px + py * py));
                rre += gw[j] * g.x;
                rim += gw[j] * g.y;
            }
            re += gw[i] * rre;
            im += gw[i] * rim;
        }
        re *= 0.25;
        im *= 0.25;
    }
    gc[(size_t)b * n + a] = make_double2(re, im);
}

__global__ void wrap_kernel(int n, int M, const double2 *__restrict__ gc, double2 *__restrict__ full) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= M) return;
    const int dy = y < n ? y : (y > M - n ? M - y : -1);
    const int dxo = x < n ? x : (x > M - n ? M - x : -1);
    full[(size_t)y * M + x] = (dy >= 0 && dxo >= 0) ? gc[(size_t)dy * n + dxo] : make_double2(0.0, 0.0);
}

__global__ void twiddle64_kernel(int M, double2 *__restrict__ tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)M, &s, &c);
    tw[k] = make_double2(c, -s);  // exp(-2 pi i k / M)
}

__global__ void twiddle32_kernel(int M, const double2 *__restrict__ tw64, float2 *__restrict__ tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    tw[k] = make_float2((float)tw64[k].x, (float)tw64[k].y);
}

// Forward FFT of every row of an M x M FP64 array, one block per row,
// radix-2 Stockham ping-pong in shared memory (2 M double2).
__global__ void fft64_rows_kernel(int M, double2 *__restrict__ a, const double2 *__restrict__ tw) {
    extern __shared__ double2 sh64[];
    double2 *src = sh64, *dst = sh64 + M;
    double2 *row = a + (size_t)blockIdx.x * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) src[i] = row[i];
    __syncthreads();
    const int half = M / 2;
    for (int Ns = 1; Ns < M; Ns <<= 1) {
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (Ns - 1);
            const double2 a0 = src[j], a1 = src[j + half];
            const double2 w = tw[k * (M / (2 * Ns))];
            const double2 b1 = make_double2(a1.x * w.x - a1.y * w.y, a1.x * w.y + a1.y * w.x);
            const int d = (j / Ns) * 2 * Ns + k;
            dst[d] = make_double2(a0.x + b1.x, a0.y + b1.y);
            dst[d + Ns] = make_double2(a0.x - b1.x, a0.y - b1.y);
        }
        __syncthreads();
        double2 *t = src;
        src = dst;
        dst = t;
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) row[i] = src[i];
}

__global__ void transpose64_kernel(int M, const double2 *__restrict__ in, double2 *__restrict__ out) {
    __shared__ double2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y)
        if (by + j < M && bx + (int)threadIdx.x < M)
            tile[j][threadIdx.x] = in[(size_t)(by + j) * M + bx + threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y)
        if (bx + j < M && by + (int)threadIdx.x < M)
            out[(size_t)(bx + j) * M + by + threadIdx.x] = tile[threadIdx.x][j];
}

// quadrant 0 <= kx, ky <= M/2, stored with row stride ghat_stride(M) (the
// padding column is zero)
__global__ void pack_quadrant_kernel(int M, double scale, const double2 *__restrict__ full,
                                     float2 *__restrict__ ghq) {
    const int kx = blockIdx.x * blockDim.x + threadIdx.x;
    const int ky = blockIdx.y;
    const int qs = M / 2 + 1, qsp = ghat_stride(M);
    if (kx >= qsp) return;
    float2 out = make_float2(0.f, 0.f);
    if (kx < qs) {
        const double2 v = full[(size_t)ky * M + kx];
        out = make_float2((float)(v.x * scale), (float)(v.y * scale));
    }
    ghq[(size_t)ky * qsp + kx] = out;
}

cudaError_t build_twiddles(int M, float2 *tw, cudaStream_t s) {
    double2 *tw64 = nullptr;
    cudaError_t e = cudaMalloc(&tw64, sizeof(double2) * M);
    if (e != cudaSuccess) return e;
    twiddle64_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, tw64);
    twiddle32_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, tw64, tw);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tw64);
    return e;
}

cudaError_t build_ghat(int n, int M, double k0, double dx, float2 *ghq, cudaStream_t s) {
    {
        double xs[TBS_NQ_SELF], ws[TBS_NQ_SELF], xn[TBS_NQ_NEAR], wn[TBS_NQ_NEAR];
        double xf[TBS_NQ_FAR], wf[TBS_NQ_FAR];
        gauss_legendre_rule(TBS_NQ_SELF, xs, ws);
        gauss_legendre_rule(TBS_NQ_NEAR, xn, wn);
        gauss_legendre_rule(TBS_NQ_FAR, xf, wf);
        cudaError_t e;
        if ((e = cudaMemcpyToSymbol(c_gl_self_x, xs, sizeof(xs)))) return e;
        if ((e = cudaMemcpyToSymbol(c_gl_self_w, ws, sizeof(ws)))) return e;
        if ((e = cudaMemcpyToSymbol(c_gl_near_x, xn, sizeof(xn)))) return e;
        if ((e = cudaMemcpyToSymbol(c_gl_near_w, wn, sizeof(wn)))) return e;
        if ((e = cudaMemcpyToSymbol(c_gl_far_x, xf, sizeof(xf)))) return e;
        if ((e = cudaMemcpyToSymbol(c_gl_far_w, wf, sizeof(wf)))) return e;
    }
    double2 *gc = nullptr, *full = nullptr, *tmp = nullptr, *tw64 = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t mm = (size_t)M * M;
    if ((e = cudaMalloc(&gc, sizeof(double2) * (size_t)n * n))) goto done;
    if ((e = cudaMalloc(&full, sizeof(double2) * mm))) goto done;
    if ((e = cudaMalloc(&tmp, sizeof(double2) * mm))) goto done;
    if ((e = cudaMalloc(&tw64, sizeof(double2) * M))) goto done;
    if ((e = cudaFuncSetAttribute(fft64_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * M * sizeof(double2)))))
        goto done;
    green_quadrant_kernel<<<dim3((n + 127) / 128, n), 128, 0, s>>>(n, k0, dx, gc);
    wrap_kernel<<<dim3((M + 255) / 256, M), 256, 0, s>>>(n, M, gc, full);
    twiddle64_kernel<<<(M + 255) / 256, 256, 0, s>>>(M, tw64);
    {
        const size_t sh = 2 * (size_t)M * sizeof(double2);
        const int thr = M / 2 < 512 ? (M / 2 < 32 ? 32 : M / 2) : 512;
        const dim3 tg((M + 31) / 32, (M + 31) / 32);
        fft64_rows_kernel<<<M, thr, sh, s>>>(M, full, tw64);
        transpose64_kernel<<<tg, dim3(32, 8), 0, s>>>(M, full, tmp);
        fft64_rows_kernel<<<M, thr, sh, s>>>(M, tmp, tw64);
        transpose64_kernel<<<tg, dim3(32, 8), 0, s>>>(M, tmp, full);
    }
    pack_quadrant_kernel<<<dim3((ghat_stride(M) + 255) / 256, M / 2 + 1), 256, 0, s>>>(
        M, dx * dx / ((double)M * (double)M), full, ghq);
    if ((e = cudaGetLastError())) goto done;
    e = cudaStreamSynchronize(s);
done:
    cudaFree(gc);
    cudaFree(full);
    cudaFree(tmp);
    cudaFree(tw64);
    return e;
}

}  // namespace tbs
