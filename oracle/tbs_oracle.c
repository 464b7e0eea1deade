/*
 * tbs_oracle.c -- plain, slow, complex128 reference implementation of the
 * traditional Born series (TBS) for the 2D inhomogeneous Helmholtz equation
 * (arxiv 2507.13754, Section 2.2 "Derivation of the Born series").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only at the seeded synthetic
 * inputs.
 *
 * What it computes, in the paper's notation with the free-space
 * discretisation used by this project (zero padding instead of the paper's
 * periodic grid + absorbing layer, epsilon = 0):
 *
 *   Helmholtz form            lap(psi) + k0^2 psi = -S - V psi          (Eq. 13)
 *   Lippmann-Schwinger        psi = G (V psi + S)                       (Eqs. 15, 17)
 *   Born series               psi = sum_n (G V)^n G S                   (Eq. 18)
 *   term recurrence           u_0 = G S,  u_{n+1} = G (V u_n)           (Eqs. 19, 20)
 *
 * G is convolution with the 2D outgoing free-space Green's function
 * g(r) = (i/4) H0^(1)(k0 r), the solution of lap g + k0^2 g = -delta
 * (Eq. 16 with epsilon -> 0), averaged over each grid cell:
 *
 *   (G f)[m] = dx^2 * sum_n Gc[m - n] f[n],
 *   Gc[d]    = (1/dx^2) * integral over cell d of g(|r|) d^2r.
 *
 * A second part, at the end of the file, follows the paper's own
 * discretisation (periodic grid, epsilon-shifted spectral G, absorbing
 * layer, Eq. 30 row stop; Section 3.1 and Algorithm 1).
 *
 * Every routine is the plain definition: an iterative radix-2 FFT with
 * twiddles from cos/sin in double, a cyclic convolution of size M >= 2N-1
 * (exact linear convolution on the N x N crop), and the recurrence written
 * term by term.  OpenMP only splits independent rows/columns; it does not
 * reorder any sum.
 */
#define _DEFAULT_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n with  */
/* the three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}.        */
/* ------------------------------------------------------------------------ */
int ora_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0.0, pm = 0.0, dp = 1.0;
        for (int it = 0; it < 200; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pn = p1;
            pm = p0;
            if (n == 1) { pn = z; pm = 1.0; }
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) <= 1e-16) break;
        }
        /* derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pn = (n == 1) ? z : p1;
            pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Green's function (Eq. 16, epsilon -> 0): g(r) = (i/4) H0^(1)(k0 r),        */
/* H0^(1) = J0 + i Y0, so g = (i/4) J0 - (1/4) Y0.  J0, Y0 from libm.         */
/* ------------------------------------------------------------------------ */
void ora_green_point(double k0, double r, double *re, double *im)
{
    double z = k0 * r;
    double j = j0(z), y = y0(z);
    *re = -0.25 * y;
    *im = 0.25 * j;
}

static cplx green_point(double k0, double r)
{
    double re, im;
    ora_green_point(k0, r, &re, &im);
    return re + I * im;
}

#define ORA_NQ_SELF 40   /* polar rule for the self cell, per direction   */
#define ORA_NQ_NEAR 20   /* tensor rule for cells with max(|a|,|b|) <= 3  */
#define ORA_NQ_FAR 8     /* tensor rule for all other cells               */

/* Mean of g over the square cell centred at (a dx, b dx), side dx. */
static cplx green_cell_mean(double k0, double dx, int a, int b,
                            const double *xs, const double *ws,
                            const double *xn, const double *wn,
                            const double *xf, const double *wf)
{
    if (a == 0 && b == 0) {
        /* Self cell: the log singularity sits at the centre.  Split the
         * square into 8 congruent right triangles with apex at the centre;
         * on the one with 0 <= theta <= pi/4 the radius runs to
         * R(theta) = (dx/2)/cos(theta).  Substituting r = R t^2 turns the
         * r dr ln r integrand into a smooth one (2 R^2 t^3 dt), so
         * Gauss-Legendre converges fast in both t and theta. */
        cplx acc = 0.0;
        for (int p = 0; p < ORA_NQ_SELF; p++) {
            double th = 0.5 * (xs[p] + 1.0) * (M_PI / 4.0);
            double wth = 0.5 * ws[p] * (M_PI / 4.0);
            double R = 0.5 * dx / cos(th);
            cplx inner = 0.0;
            for (int q = 0; q < ORA_NQ_SELF; q++) {
                double t = 0.5 * (xs[q] + 1.0);
                double wt = 0.5 * ws[q];
                inner += wt * green_point(k0, R * t * t) * (2.0 * R * R * t * t * t);
            }
            acc += wth * inner;
        }
        return 8.0 * acc / (dx * dx);
    }
    int aa = abs(a), bb = abs(b);
    int near = (aa <= 3 && bb <= 3);
    int nq = near ? ORA_NQ_NEAR : ORA_NQ_FAR;
    const double *x = near ? xn : xf;
    const double *w = near ? wn : wf;
    cplx acc = 0.0;
    for (int i = 0; i < nq; i++) {
        double px = (a + 0.5 * x[i]) * dx;
        cplx row = 0.0;
        for (int j = 0; j < nq; j++) {
            double py = (b + 0.5 * x[j]) * dx;
            row += 0.5 * w[j] * green_point(k0, sqrt(px * px + py * py));
        }
        acc += 0.5 * w[i] * row;
    }
    return acc;
}

/* Cell-averaged Green's function Gc[d] for one offset d = (a, b). */
void ora_green_cell(double k0, double dx, int a, int b, double *re, double *im)
{
    double xs[ORA_NQ_SELF], ws[ORA_NQ_SELF], xn[ORA_NQ_NEAR], wn[ORA_NQ_NEAR];
    double xf[ORA_NQ_FAR], wf[ORA_NQ_FAR];
    ora_gauss_legendre(ORA_NQ_SELF, xs, ws);
    ora_gauss_legendre(ORA_NQ_NEAR, xn, wn);
    ora_gauss_legendre(ORA_NQ_FAR, xf, wf);
    cplx v = green_cell_mean(k0, dx, a, b, xs, ws, xn, wn, xf, wf);
    *re = creal(v);
    *im = cimag(v);
}

/* Quadrant table gc[b*n + a] = Gc[(a, b)] for a, b in [0, n).  The full
 * table follows from Gc[(+-a, +-b)] = Gc[(a, b)] (g depends on |r| only). */
void ora_green_table(int n, double k0, double dx, cplx *gc)
{
    double xs[ORA_NQ_SELF], ws[ORA_NQ_SELF], xn[ORA_NQ_NEAR], wn[ORA_NQ_NEAR];
    double xf[ORA_NQ_FAR], wf[ORA_NQ_FAR];
    ora_gauss_legendre(ORA_NQ_SELF, xs, ws);
    ora_gauss_legendre(ORA_NQ_NEAR, xn, wn);
    ora_gauss_legendre(ORA_NQ_FAR, xf, wf);
#pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < n; b++)
        for (int a = 0; a < n; a++)
            gc[(size_t)b * n + a] = green_cell_mean(k0, dx, a, b, xs, ws, xn, wn, xf, wf);
}

/* ------------------------------------------------------------------------ */
/* Iterative radix-2 FFT (bit reversal + Cooley-Tukey butterflies),          */
/* unnormalised: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n).               */
/* ------------------------------------------------------------------------ */
static int is_pow2(long n) { return n > 0 && (n & (n - 1)) == 0; }

static void fft1_with_table(cplx *a, long n, const cplx *tw)
{
    /* tw[k] = exp(sign 2 pi i k / n), k < n/2 */
    for (long i = 1, j = 0; i < n; i++) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (long len = 2; len <= n; len <<= 1) {
        long half = len >> 1, step = n / len;
        for (long i = 0; i < n; i += len)
            for (long k = 0; k < half; k++) {
                cplx u = a[i + k];
                cplx v = a[i + k + half] * tw[k * step];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

static cplx *twiddle_table(long n, int sign)
{
    long h = n / 2 > 0 ? n / 2 : 1;
    cplx *tw = (cplx *)malloc(sizeof(cplx) * h);
    for (long k = 0; k < h; k++) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        tw[k] = cos(ang) + I * sin(ang);
    }
    return tw;
}

int ora_fft(cplx *a, long n, int sign)
{
    if (!is_pow2(n)) return -1;
    if (n == 1) return 0;
    cplx *tw = twiddle_table(n, sign);
    fft1_with_table(a, n, tw);
    free(tw);
    return 0;
}

/* 2D FFT of a row-major m x m array: every row, then every column. */
int ora_fft2(cplx *a, long m, int sign)
{
    if (!is_pow2(m)) return -1;
    if (m == 1) return 0;
    cplx *tw = twiddle_table(m, sign);
#pragma omp parallel for schedule(static)
    for (long r = 0; r < m; r++) fft1_with_table(a + r * m, m, tw);
#pragma omp parallel
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * m);
#pragma omp for schedule(static)
        for (long c = 0; c < m; c++) {
            for (long r = 0; r < m; r++) col[r] = a[r * m + c];
            fft1_with_table(col, m, tw);
            for (long r = 0; r < m; r++) a[r * m + c] = col[r];
        }
        free(col);
    }
    free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* G as a zero-padded cyclic convolution.  With M >= 2N - 1 the cyclic      */
/* convolution of the wrapped table with the zero-extended field equals the  */
/* linear convolution on the N x N crop.                                     */
/* ------------------------------------------------------------------------ */

/* Spectrum of the wrapped table, scaled so that apply = IFFT(ghat * FFT(f))
 * with an unnormalised inverse:  ghat = FFT_M(T) * dx^2 / M^2, where
 * T[y][x] = Gc[(dx(x), dy(y))], d(i) = i for i < N, i - M for i > M - N,
 * and T = 0 elsewhere (offsets that never occur between two grid cells). */
int ora_ghat(int n, int m, double dx, const cplx *gc, cplx *ghat)
{
    if (!is_pow2(m) || m < 2 * n - 1) return -1;
    for (long y = 0; y < m; y++) {
        long dy = (y < n) ? y : (y > m - n ? m - y : -1);
        for (long x = 0; x < m; x++) {
            long dxo = (x < n) ? x : (x > m - n ? m - x : -1);
            ghat[y * m + x] = (dy >= 0 && dxo >= 0) ? gc[dy * n + dxo] : 0.0;
        }
    }
    ora_fft2(ghat, m, -1);
    double s = dx * dx / ((double)m * (double)m);
    for (long i = 0; i < (long)m * m; i++) ghat[i] *= s;
    return 0;
}

/* out = G f on the N x N grid; with conj_kernel != 0 the kernel is conj(Gc),
 * i.e. the Hermitian adjoint G^H (Gc is even, so G is symmetric).
 * work: m*m scratch. */
static void apply_g_work(int n, int m, const cplx *ghat, const cplx *f, cplx *out,
                         int conj_kernel, cplx *work)
{
    memset(work, 0, sizeof(cplx) * (size_t)m * m);
    for (long y = 0; y < n; y++)
        for (long x = 0; x < n; x++) work[y * m + x] = f[y * n + x];
    ora_fft2(work, m, -1);
    if (conj_kernel) {
        for (long i = 0; i < (long)m * m; i++) work[i] *= conj(ghat[i]);
    } else {
        for (long i = 0; i < (long)m * m; i++) work[i] *= ghat[i];
    }
    ora_fft2(work, m, +1);
    for (long y = 0; y < n; y++)
        for (long x = 0; x < n; x++) out[y * n + x] = work[y * m + x];
}

int ora_apply_g(int n, int m, const cplx *ghat, const cplx *f, cplx *out, int conj_kernel)
{
    if (!is_pow2(m) || m < 2 * n - 1) return -1;
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    if (!work) return -2;
    apply_g_work(n, m, ghat, f, out, conj_kernel, work);
    free(work);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Potential V = p^2 - k0^2 (Eq. 13: lap psi + k0^2 psi = -S - V psi with    */
/* V = k(x)^2 - k0^2; Eq. 25 for the disk scatterer).  Absorption and its    */
/* dispersion follow the power-law model of Eqs. 3, 4 and 7: to first order */
/* alpha0 a plane wave has p = omega/v + alpha0 omega^y (tan(pi y/2) + i).   */
/* Here c(x) is the phase speed at f_ref, alpha(x) = alpha0 omega^y is the   */
/* absorption in Np/m at the solve frequency, and                           */
/*   p = omega/c + alpha (tan(pi y / 2) * delta + i),                       */
/*   delta = 1 - (f_ref / f)^(y - 1)  (delta = 1 when f_ref <= 0).          */
/* ------------------------------------------------------------------------ */
static cplx slowness_p(double omega, double c, double alpha, double tdel)
{
    return omega / c + alpha * (tdel + I);
}

static double disp_factor(double f, double ypow, double f_ref)
{
    double delta = (f_ref > 0.0) ? 1.0 - pow(f_ref / f, ypow - 1.0) : 1.0;
    return tan(M_PI * ypow / 2.0) * delta;
}

void ora_potential(long count, double f, double c0, const double *c, const double *alpha,
                   double ypow, double f_ref, cplx *V)
{
    double omega = 2.0 * M_PI * f, k0 = omega / c0;
    double tdel = alpha ? disp_factor(f, ypow, f_ref) : 0.0;
    for (long i = 0; i < count; i++) {
        cplx p = slowness_p(omega, c[i], alpha ? alpha[i] : 0.0, tdel);
        V[i] = p * p - k0 * k0;
    }
}

/* dV/dc = 2 p (-omega / c^2),  dV/dalpha = 2 p (tan(pi y/2) delta + i). */
void ora_potential_derivs(long count, double f, const double *c, const double *alpha,
                          double ypow, double f_ref, cplx *dVdc, cplx *dVdalpha)
{
    double omega = 2.0 * M_PI * f;
    double tdel = alpha ? disp_factor(f, ypow, f_ref) : 0.0;
    for (long i = 0; i < count; i++) {
        cplx p = slowness_p(omega, c[i], alpha ? alpha[i] : 0.0, tdel);
        dVdc[i] = 2.0 * p * (-omega / (c[i] * c[i]));
        dVdalpha[i] = 2.0 * p * (tdel + I);
    }
}

/* Point sources (Section 3.1, Algorithm 1's source table):
 * S = sum_j a_j delta_{cell_j} / dx^2 (a discrete delta of unit integral), so the field of one isolated element is u_0 = a_j Gc[. - n_j]. */
int ora_deposit_points(int n, double dx, int npts, const int32_t *ix, const int32_t *iy,
                       const cplx *amp, cplx *s)
{
    for (int j = 0; j < npts; j++) {
        if (ix[j] < 0 || ix[j] >= n || iy[j] < 0 || iy[j] >= n) return -1;
        s[(size_t)iy[j] * n + ix[j]] += amp[j] / (dx * dx);
    }
    return 0;
}

/* Second-harmonic source of the sum-term series (Eq. 28b):
 *   S2 = -(1/2) xi (2 omega)^2 psi1^2,   xi = beta / (rho c^4),
 * beta = 1 + B/(2A) (Eq. 11). */
void ora_harmonic2_source(long count, double omega, const double *beta, const double *rho,
                          const double *c, const cplx *psi1, cplx *s2)
{
    for (long i = 0; i < count; i++) {
        double c2 = c[i] * c[i];
        double xi = beta[i] / (rho[i] * c2 * c2);
        double w2 = 2.0 * omega;
        s2[i] = -0.5 * xi * w2 * w2 * psi1[i] * psi1[i];
    }
}

/* Sum-term source of harmonic n = order (2 .. 5) from the lower harmonics  */
/* psi_1 .. psi_{n-1} (Eqs. 28b-28e): with                                 */
/* P = Re sum_k psi_k e^{-i k w t}, the e^{-i n w t} phasor of the          */
/* nonlinear term keeps the products psi_i psi_j with i + j = n,            */
/*   S_n = -xi (n w)^2 [ sum_{i<j, i+j=n} psi_i psi_j + (1/2) psi_{n/2}^2 ], */
/* xi = beta / (rho c^4).  psi: [order - 1][count], psi_k at (k-1)*count.   */
int ora_harmonic_source(long count, int order, double omega, const double *beta, const double *rho,
                        const double *c, const cplx *psi, cplx *sn)
{
    if (order < 2 || order > 5) return -1;
    const double wn = order * omega;
    for (long i = 0; i < count; i++) {
        const double c2 = c[i] * c[i];
        const double xi = beta[i] / (rho[i] * c2 * c2);
        cplx acc = 0.0;
        for (int a = 1; 2 * a <= order; a++) {
            const int b = order - a;
            const cplx pa = psi[(size_t)(a - 1) * count + i], pb = psi[(size_t)(b - 1) * count + i];
            acc += (a == b ? 0.5 : 1.0) * pa * pb;
        }
        sn[i] = -xi * wn * wn * acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The series.                                                               */
/* ------------------------------------------------------------------------ */
enum { ORA_CONVERGED = 0, ORA_MAX_TERMS = 1, ORA_DIVERGED = 2, ORA_NONFINITE = 3 };
enum { ORA_STOP_L2 = 0, ORA_STOP_L1_ROW = 1 };

typedef struct {
    int max_terms;       /* cap on the number of terms u_0 .. u_{T-1}          */
    double tol;          /* stop when the residual falls below tol             */
    int stop_mode;       /* ORA_STOP_L2 or ORA_STOP_L1_ROW                      */
    int l1_row;          /* row of the L1 test (Eq. 30), 0-based                */
    int div_grace;       /* no growth test before this term index               */
    int div_window;      /* consecutive growing terms that flag divergence      */
    double div_factor;   /* |u_n| > div_factor |u_0| flags divergence           */
} ora_stop_params;

typedef struct {
    int terms;           /* number of terms summed into psi                    */
    int status;
    double residual;     /* last residual evaluated                            */
    double term_norm_max;
    double psi_norm;
} ora_solve_info;

static double l2sq(const cplx *a, long count)
{
    double s = 0.0;
    for (long i = 0; i < count; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static double l1row(const cplx *a, int n, int row)
{
    double s = 0.0;
    for (int x = 0; x < n; x++) s += cabs(a[(size_t)row * n + x]);
    return s;
}

/* u_0 = G s; u_{n+1} = G (V u_n); psi_n = sum_{k<=n} u_k (Eqs. 18-20).
 * After term n the stop test runs on (u_n, psi_n):
 *   L2 mode:     r_n = |u_n|_2 / |psi_n|_2 over the whole grid;
 *   L1_ROW mode: r_n = sum_m |u_n(row, m)| / sum_m |psi_{n-1}(row, m)|, n >= 1,
 *                which is Eq. 30's |psi_{l+1} - psi_l| / |psi_l| on one row.
 * Checks in order: non-finite norms, r_n < tol, divergence, term cap.
 * u_all (optional) receives every term [max_terms][N*N]; norms (optional)
 * receives |u_n|_2 per term. */
int ora_tbs_solve(int n, int m, const cplx *ghat, const cplx *V, const cplx *s,
                  const ora_stop_params *sp, cplx *psi, ora_solve_info *info,
                  double *norms, cplx *u_all)
{
    if (!is_pow2(m) || m < 2 * n - 1 || sp->max_terms < 1) return -1;
    long nn = (long)n * n;
    cplx *u = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *vu = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    if (!u || !vu || !work) { free(u); free(vu); free(work); return -2; }

    apply_g_work(n, m, ghat, s, u, 0, work); /* u_0 = G S (Eq. 20) */
    memcpy(psi, u, sizeof(cplx) * nn);
    double u0 = sqrt(l2sq(u, nn)), prev = u0, tmax = u0;
    double psi_prev_l1 = 0.0;
    int grow = 0;
    info->status = ORA_MAX_TERMS;
    info->residual = INFINITY;
    for (int t = 0;; t++) {
        if (u_all) memcpy(u_all + (size_t)t * nn, u, sizeof(cplx) * nn);
        double un = sqrt(l2sq(u, nn));
        double pn = sqrt(l2sq(psi, nn));
        if (norms) norms[t] = un;
        if (un > tmax) tmax = un;
        info->terms = t + 1;
        info->psi_norm = pn;
        double r;
        int have_r = 1;
        if (sp->stop_mode == ORA_STOP_L1_ROW) {
            if (t == 0) { have_r = 0; r = INFINITY; }
            else r = l1row(u, n, sp->l1_row) / psi_prev_l1;
        } else {
            r = (pn > 0.0) ? un / pn : (un > 0.0 ? INFINITY : 0.0);
        }
        if (have_r) info->residual = r;
        if (t > 0) grow = (un > prev) ? grow + 1 : 0;
        if (!isfinite(un) || !isfinite(pn)) { info->status = ORA_NONFINITE; break; }
        if (have_r && r < sp->tol) { info->status = ORA_CONVERGED; break; }
        if ((t >= sp->div_grace && grow >= sp->div_window) || un > sp->div_factor * u0) {
            info->status = ORA_DIVERGED;
            break;
        }
        if (t + 1 >= sp->max_terms) { info->status = ORA_MAX_TERMS; break; }
        if (sp->stop_mode == ORA_STOP_L1_ROW) psi_prev_l1 = l1row(psi, n, sp->l1_row);
        prev = un;
        /* next term: u_{t+1} = G (V u_t) (Eq. 19) */
        for (long i = 0; i < nn; i++) vu[i] = V[i] * u[i];
        apply_g_work(n, m, ghat, vu, u, 0, work);
        for (long i = 0; i < nn; i++) psi[i] += u[i];
    }
    info->term_norm_max = tmax;
    free(u);
    free(vu);
    free(work);
    return 0;
}

/* Adjoint of the truncated series psi = sum_{n<T} u_n with respect to V.
 * For a real loss L with complex gradient g = dL/dRe(psi) + i dL/dIm(psi):
 *   ubar_{T-1} = g,  lambda_{j+1} = G^H ubar_{j+1},  ubar_j = g + conj(V) lambda_{j+1},
 *   Q = sum_{j=0}^{T-2} conj(lambda_{j+1}) u_j,
 * and dL/dtheta(x) = Re(Q(x) dV/dtheta(x)) for any real medium parameter theta.
 * u_all holds the T forward terms [T][N*N].  Q receives N*N values. */
int ora_tbs_adjoint(int n, int m, const cplx *ghat, const cplx *V, int T, const cplx *u_all,
                    const cplx *g, cplx *Q)
{
    if (!is_pow2(m) || m < 2 * n - 1 || T < 1) return -1;
    long nn = (long)n * n;
    cplx *ubar = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *lam = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)m * m);
    if (!ubar || !lam || !work) { free(ubar); free(lam); free(work); return -2; }
    memcpy(ubar, g, sizeof(cplx) * nn);
    memset(Q, 0, sizeof(cplx) * nn);
    for (int j = T - 2; j >= 0; j--) {
        apply_g_work(n, m, ghat, ubar, lam, 1, work);
        const cplx *uj = u_all + (size_t)j * nn;
        for (long i = 0; i < nn; i++) {
            Q[i] += conj(lam[i]) * uj[i];
            ubar[i] = g[i] + conj(V[i]) * lam[i];
        }
    }
    free(ubar);
    free(lam);
    free(work);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own discretisation (Section 2.2 with finite epsilon, Section  */
/* 3.1 and Algorithm 1): a periodic N x N grid without padding, the        */
/* spectral Green's function of the epsilon-shifted equation                */
/*     lap g + (k0^2 + i eps) g = -delta,   g~(p) = 1 / (|p|^2 - k0^2 - i eps), */
/* applied as  G f = IDFT(g~ . DFT(f))  (the IDFT carries 1/N^2, which     */
/* makes the sum over p the dx^2-weighted convolution with g), and         */
/* V = U - i eps, so that a fixed point of psi = G (V psi + S) solves      */
/* lap psi + (k0^2 + U) psi = -S: the i eps cancels.  The paper iterates    */
/*     psi^0 = G S,   psi^{l+1} = A . G (V psi^l + S)                      */
/* with A an absorbing layer: within mu = `width` cells of an edge the     */
/* field is multiplied by the sigmoid 1 / (1 + exp(-zeta (x - mu/2))), x   */
/* the distance from that edge (x, y profiles multiplied at the corners),   */
/* and stops when Eq. 30's row ratio                                        */
/*     sum_m |psi^{l+1}(r, m) - psi^l(r, m)| / sum_m |psi^l(r, m)|          */
/* falls below tol.                                                         */
/* ------------------------------------------------------------------------ */

/* g~(p) / N^2 on the DFT wavenumbers p = 2 pi (j, i) / (N dx), j, i taken  */
/* in [-N/2, N/2), row-major [ky][kx], for the unnormalised transforms.    */
int ora_ghat_eps(int n, double dx, double k0, double eps, cplx *gh)
{
    if (!is_pow2(n)) return -1;
    const double dp = 2.0 * M_PI / (n * dx), inv = 1.0 / ((double)n * (double)n);
    for (int j = 0; j < n; j++) {
        const double py = dp * (j < n / 2 ? j : j - n);
        for (int i = 0; i < n; i++) {
            const double px = dp * (i < n / 2 ? i : i - n);
            gh[(size_t)j * n + i] = inv / (px * px + py * py - k0 * k0 - I * eps);
        }
    }
    return 0;
}

/* Absorbing-layer profile along one axis (the sigmoid above; 1 outside).  */
void ora_abl_profile(int n, double dx, double zeta, int width, double *prof)
{
    const double mu = width * dx;
    for (int i = 0; i < n; i++) {
        const int e = i < n - 1 - i ? i : n - 1 - i;  /* cells to the nearer edge */
        prof[i] = e < width ? 1.0 / (1.0 + exp(-zeta * (e * dx - 0.5 * mu))) : 1.0;
    }
}

typedef struct {
    int iters;           /* iterations l run (psi^iters returned)              */
    int status;          /* 0 converged, 1 iteration cap, 3 non-finite         */
    double error;        /* last row ratio                                     */
} ora_eps_info;

/* psi: out, N x N.  abl: per-axis profile or NULL (no layer).  errs:      */
/* optional, the row ratio of every iteration.                             */
int ora_eps_solve(int n, const cplx *gh, const cplx *V, const cplx *S, const double *abl,
                  int max_iter, double tol, int row, cplx *psi, ora_eps_info *info, double *errs)
{
    if (!is_pow2(n) || row < 0 || row >= n) return -1;
    const long nn = (long)n * n;
    cplx *w = (cplx *)malloc(sizeof(cplx) * nn);
    if (!w) return -2;
    /* psi^0 = G S */
    memcpy(w, S, sizeof(cplx) * nn);
    ora_fft2(w, n, -1);
    for (long i = 0; i < nn; i++) w[i] *= gh[i];
    ora_fft2(w, n, +1);
    memcpy(psi, w, sizeof(cplx) * nn);
    info->iters = 0;
    info->status = 1;
    info->error = INFINITY;
    for (int it = 1; it <= max_iter; it++) {
        for (long i = 0; i < nn; i++) w[i] = V[i] * psi[i] + S[i];
        ora_fft2(w, n, -1);
        for (long i = 0; i < nn; i++) w[i] *= gh[i];
        ora_fft2(w, n, +1);
        if (abl)
            for (long y = 0; y < n; y++)
                for (long x = 0; x < n; x++) w[y * n + x] *= abl[y] * abl[x];
        double num = 0.0, den = 0.0;
        for (int x = 0; x < n; x++) {
            num += cabs(w[(size_t)row * n + x] - psi[(size_t)row * n + x]);
            den += cabs(psi[(size_t)row * n + x]);
        }
        const double err = num / den;
        if (errs) errs[it - 1] = err;
        memcpy(psi, w, sizeof(cplx) * nn);
        info->iters = it;
        info->error = err;
        if (!isfinite(err)) {
            info->status = 3;
            break;
        }
        if (err < tol) {
            info->status = 0;
            break;
        }
    }
    free(w);
    return 0;
}

/* The convergent Born series preconditioner (Osnabrugge, Leedumrongwatthanakun
 * and Vellekoop, J. Comput. Phys. 322 (2016); the paper names it as future
 * work in Section 5) on the paper's periodic iteration: with
 * gamma = i V / eps, V = U - i eps and eps >= max |U|,
 *     psi^0 = G S,
 *     psi^{l+1} = A . (psi^l + gamma (G (V psi^l + S) - psi^l)),
 * stopped by Eq. 30 on `row` as in ora_eps_solve.  The fixed point without
 * a layer is the plain iteration's (gamma vanishes nowhere). */
int ora_eps_solve_cbs(int n, const cplx *gh, const cplx *V, const cplx *S, const double *abl, double eps,
                      int max_iter, double tol, int row, cplx *psi, ora_eps_info *info, double *errs)
{
    if (!is_pow2(n) || row < 0 || row >= n || !(eps > 0.0)) return -1;
    const long nn = (long)n * n;
    cplx *w = (cplx *)malloc(sizeof(cplx) * nn);
    if (!w) return -2;
    memcpy(w, S, sizeof(cplx) * nn);
    ora_fft2(w, n, -1);
    for (long i = 0; i < nn; i++) w[i] *= gh[i];
    ora_fft2(w, n, +1);
    memcpy(psi, w, sizeof(cplx) * nn);
    info->iters = 0;
    info->status = 1;
    info->error = INFINITY;
    for (int it = 1; it <= max_iter; it++) {
        for (long i = 0; i < nn; i++) w[i] = V[i] * psi[i] + S[i];
        ora_fft2(w, n, -1);
        for (long i = 0; i < nn; i++) w[i] *= gh[i];
        ora_fft2(w, n, +1);
        for (long i = 0; i < nn; i++) {
            const cplx gamma = I * V[i] / eps;
            w[i] = psi[i] + gamma * (w[i] - psi[i]);
        }
        if (abl)
            for (long y = 0; y < n; y++)
                for (long x = 0; x < n; x++) w[y * n + x] *= abl[y] * abl[x];
        double num = 0.0, den = 0.0;
        for (int x = 0; x < n; x++) {
            num += cabs(w[(size_t)row * n + x] - psi[(size_t)row * n + x]);
            den += cabs(psi[(size_t)row * n + x]);
        }
        const double err = num / den;
        if (errs) errs[it - 1] = err;
        memcpy(psi, w, sizeof(cplx) * nn);
        info->iters = it;
        info->error = err;
        if (!isfinite(err)) {
            info->status = 3;
            break;
        }
        if (err < tol) {
            info->status = 0;
            break;
        }
    }
    free(w);
    return 0;
}

/* k-space absorbing-dispersive potential (Section 2.3, Eq. 24 and         */
/* Algorithm 1, case II) on the DFT wavenumbers, row-major [ky][kx]:        */
/*     VV(p) = eta |p|^(nu+1) - i (tau omega |p|^nu + eps),                  */
/* with tau = -2 alpha0 v^(nu-1), eta = 2 alpha0 v^nu tan(pi nu / 2).        */
int ora_vv_kspace(int n, double dx, double omega, double eta, double tau, double nu, double eps, cplx *vv)
{
    if (!is_pow2(n)) return -1;
    const double dp = 2.0 * M_PI / (n * dx);
    for (int j = 0; j < n; j++) {
        const double py = dp * (j < n / 2 ? j : j - n);
        for (int i = 0; i < n; i++) {
            const double px = dp * (i < n / 2 ? i : i - n);
            const double p = sqrt(px * px + py * py);
            vv[(size_t)j * n + i] = eta * pow(p, nu + 1.0) - I * (tau * omega * pow(p, nu) + eps);
        }
    }
    return 0;
}

/* The paper's case-II iteration (Algorithm 1):                            */
/*     psi^0 = IDFT(g~ DFT(S)),                                            */
/*     psi^{l+1} = A . IDFT(g~ (VV DFT(psi^l) + DFT(S))),                   */
/* stopped by Eq. 30 on `row` as in ora_eps_solve.  gh = g~ / N^2.          */
int ora_eps_solve_kspace(int n, const cplx *gh, const cplx *vv, const cplx *S, const double *abl,
                         int max_iter, double tol, int row, cplx *psi, ora_eps_info *info, double *errs)
{
    if (!is_pow2(n) || row < 0 || row >= n) return -1;
    const long nn = (long)n * n;
    cplx *w = (cplx *)malloc(sizeof(cplx) * nn), *sh = (cplx *)malloc(sizeof(cplx) * nn);
    if (!w || !sh) {
        free(w);
        free(sh);
        return -2;
    }
    memcpy(sh, S, sizeof(cplx) * nn);
    ora_fft2(sh, n, -1); /* DFT(S) */
    for (long i = 0; i < nn; i++) w[i] = gh[i] * sh[i];
    ora_fft2(w, n, +1);
    memcpy(psi, w, sizeof(cplx) * nn);
    info->iters = 0;
    info->status = 1;
    info->error = INFINITY;
    for (int it = 1; it <= max_iter; it++) {
        memcpy(w, psi, sizeof(cplx) * nn);
        ora_fft2(w, n, -1);
        for (long i = 0; i < nn; i++) w[i] = gh[i] * (vv[i] * w[i] + sh[i]);
        ora_fft2(w, n, +1);
        if (abl)
            for (long y = 0; y < n; y++)
                for (long x = 0; x < n; x++) w[y * n + x] *= abl[y] * abl[x];
        double num = 0.0, den = 0.0;
        for (int x = 0; x < n; x++) {
            num += cabs(w[(size_t)row * n + x] - psi[(size_t)row * n + x]);
            den += cabs(psi[(size_t)row * n + x]);
        }
        const double err = num / den;
        if (errs) errs[it - 1] = err;
        memcpy(psi, w, sizeof(cplx) * nn);
        info->iters = it;
        info->error = err;
        if (!isfinite(err)) {
            info->status = 3;
            break;
        }
        if (err < tol) {
            info->status = 0;
            break;
        }
    }
    free(w);
    free(sh);
    return 0;
}

/* Broadband synthesis.  The paper solves one frequency at a time with the
 * e^{-i omega t} convention of the outgoing Green's function (Section 2.2);
 * the time signal of a set of single-frequency fields is the inverse Fourier
 * sum over them:
 *     s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t).
 * psi_k(X): bilinear interpolation between the cell centres x_i = i dx_k of
 * field k (n_k x n_k, row y, column x), each fractional index clamped to
 * [0, n_k - 1].  Receivers X = (x0 + ix sx, y0 + iy sy); t_j = t0 + j dt.
 * out: [n_rhs][ny][nx][n_t]. */
static double ora_clamp_index(double u, int n, int *i0)
{
    if (u < 0.0) u = 0.0;
    if (u > n - 1) u = n - 1;
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    return u - i;
}

int ora_synthesize(int n_freq, const cplx *const *fields, const int *n, const double *dx, const double *f,
                   const double *w, int n_rhs, double x0, double y0, double sx, double sy, int nx, int ny,
                   double t0, double dt, int n_t, cplx *out)
{
    for (int k = 0; k < n_freq; k++)
        if (n[k] < 2 || !(dx[k] > 0.0)) return -1;
    for (int r = 0; r < n_rhs; r++)
        for (int iy = 0; iy < ny; iy++)
            for (int ix = 0; ix < nx; ix++) {
                cplx *o = out + (((size_t)r * ny + iy) * nx + ix) * n_t;
                for (int j = 0; j < n_t; j++) o[j] = 0.0;
                for (int k = 0; k < n_freq; k++) {
                    const int m = n[k];
                    int i0, j0;
                    const double fx = ora_clamp_index((x0 + ix * sx) / dx[k], m, &i0);
                    const double fy = ora_clamp_index((y0 + iy * sy) / dx[k], m, &j0);
                    const cplx *a = fields[k] + (size_t)r * m * m;
                    const cplx val = (1.0 - fy) * ((1.0 - fx) * a[(size_t)j0 * m + i0] + fx * a[(size_t)j0 * m + i0 + 1]) +
                                     fy * ((1.0 - fx) * a[(size_t)(j0 + 1) * m + i0] + fx * a[(size_t)(j0 + 1) * m + i0 + 1]);
                    for (int j = 0; j < n_t; j++) {
                        const double t = t0 + j * dt;
                        o[j] += w[k] * val * cexp(-2.0 * M_PI * I * f[k] * t);
                    }
                }
            }
    return 0;
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
