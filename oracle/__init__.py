"""Complex128 CPU oracle for the traditional Born series (arxiv 2507.13754).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product path (``paper_2507_13754_gb300``) never imports this
package, and this package never imports the product.

The arithmetic lives in ``tbs_oracle.c`` (plain C99, complex double, own
radix-2 FFT).  This module only marshals numpy arrays through ctypes; the few
numpy lines here are bookkeeping (dtype conversion, list assembly), not steps
of the method.  Every function cites the paper passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tbs_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libtbs_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "CONVERGED", 1: "MAX_TERMS", 2: "DIVERGED", 3: "NONFINITE"}
STOP_L2, STOP_L1_ROW = 0, 1


def build(force: bool = False) -> str:
    """Compile tbs_oracle.c with gcc (-O2, OpenMP when available)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _StopParams(C.Structure):
    _fields_ = [("max_terms", C.c_int), ("tol", C.c_double), ("stop_mode", C.c_int),
                ("l1_row", C.c_int), ("div_grace", C.c_int), ("div_window", C.c_int),
                ("div_factor", C.c_double)]


class _SolveInfo(C.Structure):
    _fields_ = [("terms", C.c_int), ("status", C.c_int), ("residual", C.c_double),
                ("term_norm_max", C.c_double), ("psi_norm", C.c_double)]


def _bind(lib):
    """Declare the argument types of the C entry points on a loaded library."""
    P = C.c_void_p
    lib.ora_gauss_legendre.argtypes = [C.c_int, P, P]
    lib.ora_green_point.argtypes = [C.c_double, C.c_double, P, P]
    lib.ora_green_cell.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, P, P]
    lib.ora_green_table.argtypes = [C.c_int, C.c_double, C.c_double, P]
    lib.ora_fft.argtypes = [P, C.c_long, C.c_int]
    lib.ora_fft2.argtypes = [P, C.c_long, C.c_int]
    lib.ora_ghat.argtypes = [C.c_int, C.c_int, C.c_double, P, P]
    lib.ora_apply_g.argtypes = [C.c_int, C.c_int, P, P, P, C.c_int]
    lib.ora_potential.argtypes = [C.c_long, C.c_double, C.c_double, P, P,
                                  C.c_double, C.c_double, P]
    lib.ora_potential.restype = None
    lib.ora_potential_derivs.argtypes = [C.c_long, C.c_double, P, P, C.c_double,
                                         C.c_double, P, P]
    lib.ora_potential_derivs.restype = None
    lib.ora_deposit_points.argtypes = [C.c_int, C.c_double, C.c_int, P, P, P, P]
    lib.ora_harmonic2_source.argtypes = [C.c_long, C.c_double, P, P, P, P, P]
    lib.ora_harmonic2_source.restype = None
    lib.ora_tbs_solve.argtypes = [C.c_int, C.c_int, P, P, P, C.POINTER(_StopParams),
                                  P, C.POINTER(_SolveInfo), P, P]
    lib.ora_tbs_adjoint.argtypes = [C.c_int, C.c_int, P, P, C.c_int, P, P, P]
    lib.ora_harmonic_source.argtypes = [C.c_long, C.c_int, C.c_double, P, P, P, P, P]
    lib.ora_vv_kspace.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_double, P]
    lib.ora_eps_solve_kspace.argtypes = [C.c_int, P, P, P, P, C.c_int, C.c_double, C.c_int, P,
                                         C.POINTER(_EpsInfo), P]
    lib.ora_ghat_eps.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, P]
    lib.ora_abl_profile.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, P]
    lib.ora_abl_profile.restype = None
    lib.ora_eps_solve.argtypes = [C.c_int, P, P, P, P, C.c_int, C.c_double, C.c_int, P,
                                  C.POINTER(_EpsInfo), P]
    lib.ora_eps_solve_cbs.argtypes = [C.c_int, P, P, P, P, C.c_double, C.c_int, C.c_double, C.c_int, P,
                                      C.POINTER(_EpsInfo), P]
    lib.ora_synthesize.argtypes = [C.c_int, P, P, P, P, P, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(C.CDLL(_LIB))
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle uses (all host cores unless OMP_NUM_THREADS)."""
    return int(_load().ora_num_threads())


def padded_size(n: int) -> int:
    """Smallest power of two M >= 2N - 1: cyclic convolution of that size
    equals the linear one on the N x N crop."""
    m = 1
    while m < 2 * n - 1:
        m *= 2
    return m


# --- primitives -----------------------------------------------------------

def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().ora_gauss_legendre(n, _p(x), _p(w)) != 0:
        raise ValueError("n must be >= 1")
    return x, w


def fft(a, sign: int = -1):
    """Unnormalised DFT, X[k] = sum_j a[j] exp(sign 2 pi i j k / n) (own radix-2)."""
    a = _c128(a).copy()
    if _load().ora_fft(_p(a), a.size, sign) != 0:
        raise ValueError("length must be a power of two")
    return a


def fft2(a, sign: int = -1):
    a = _c128(a).copy()
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square 2D array required")
    if _load().ora_fft2(_p(a), a.shape[0], sign) != 0:
        raise ValueError("side must be a power of two")
    return a


def green_point(k0: float, r: float) -> complex:
    """g(r) = (i/4) H0^(1)(k0 r): Eq. 16 of Section 2.2 with epsilon -> 0."""
    re, im = C.c_double(), C.c_double()
    _load().ora_green_point(k0, r, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def green_cell(k0: float, dx: float, a: int, b: int) -> complex:
    """Gc[(a, b)]: mean of g over the cell centred (a dx, b dx)."""
    re, im = C.c_double(), C.c_double()
    _load().ora_green_cell(k0, dx, a, b, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def green_table(n: int, k0: float, dx: float):
    """Quadrant table gc[b, a] = Gc[(a, b)], a, b in [0, n)."""
    gc = np.zeros((n, n), np.complex128)
    _load().ora_green_table(n, k0, dx, _p(gc))
    return gc


def ghat(n: int, m: int, dx: float, gc):
    """M x M spectrum of the wrapped table, scaled by dx^2 / M^2 (G = F^-1 g~ F,
    Section 2.2 below Eq. 17, with the free-space cell-averaged table)."""
    gc = _c128(gc)
    out = np.zeros((m, m), np.complex128)
    if _load().ora_ghat(n, m, dx, _p(gc), _p(out)) != 0:
        raise ValueError("need M a power of two >= 2N - 1")
    return out


def apply_g(n: int, m: int, gh, f, conj_kernel: bool = False):
    """G f (or G^H f) on the N x N grid by zero-padded FFT convolution."""
    gh = _c128(gh)
    f = _c128(f)
    out = np.zeros((n, n), np.complex128)
    if _load().ora_apply_g(n, m, _p(gh), _p(f), _p(out), int(conj_kernel)) != 0:
        raise ValueError("bad sizes")
    return out


def potential(f: float, c0: float, c, alpha=None, ypow: float = 1.0, f_ref: float | None = None):
    """V = p^2 - k0^2 with p = omega/c + alpha (tan(pi y/2) delta + i) (Eqs. 3, 4, 7, 13, 25)."""
    c = _f64(c)
    al = None if alpha is None else _f64(alpha)
    V = np.zeros(c.shape, np.complex128)
    fr = f if f_ref is None else f_ref
    _load().ora_potential(c.size, f, c0, _p(c), _p(al), ypow, fr, _p(V))
    return V


def potential_derivs(f: float, c, alpha=None, ypow: float = 1.0, f_ref: float | None = None):
    c = _f64(c)
    al = None if alpha is None else _f64(alpha)
    dc = np.zeros(c.shape, np.complex128)
    da = np.zeros(c.shape, np.complex128)
    fr = f if f_ref is None else f_ref
    _load().ora_potential_derivs(c.size, f, _p(c), _p(al), ypow, fr, _p(dc), _p(da))
    return dc, da


def deposit_points(n: int, dx: float, ix, iy, amp):
    """Dense source S = sum_j a_j delta_{cell_j} / dx^2 (Section 3.1)."""
    ix = np.ascontiguousarray(ix, np.int32)
    iy = np.ascontiguousarray(iy, np.int32)
    amp = _c128(amp)
    s = np.zeros((n, n), np.complex128)
    if _load().ora_deposit_points(n, dx, ix.size, _p(ix), _p(iy), _p(amp), _p(s)) != 0:
        raise ValueError("source outside the grid")
    return s


def harmonic2_source(omega: float, beta, rho, c, psi1):
    """S2 = -(1/2) xi (2 omega)^2 psi1^2, xi = beta / (rho c^4) (Eqs. 11, 28b)."""
    beta, rho, c = _f64(beta), _f64(rho), _f64(c)
    psi1 = _c128(psi1)
    s2 = np.zeros(psi1.shape, np.complex128)
    _load().ora_harmonic2_source(psi1.size, omega, _p(beta), _p(rho), _p(c), _p(psi1), _p(s2))
    return s2


def harmonic_source(order: int, omega: float, beta, rho, c, lower):
    """Sum-term source of harmonic `order` (2..5) from lower = [psi_1, ...,
    psi_{order-1}]: -xi (order omega)^2 [sum_{i<j, i+j=order} psi_i psi_j +
    psi_{order/2}^2 / 2] (Eqs. 28b-28e)."""
    beta, rho, c = _f64(beta), _f64(rho), _f64(c)
    if len(lower) != order - 1:
        raise ValueError("need psi_1 .. psi_{order-1}")
    psi = _c128(np.stack([np.asarray(p) for p in lower]))
    out = np.zeros(np.asarray(lower[0]).shape, np.complex128)
    if _load().ora_harmonic_source(out.size, order, omega, _p(beta), _p(rho), _p(c), _p(psi), _p(out)) != 0:
        raise ValueError("order must be 2 .. 5")
    return out


def solve(n: int, m: int, gh, V, s, max_terms: int, tol: float, stop_mode: int = STOP_L2,
          l1_row: int | None = None, div_grace: int = 8, div_window: int = 4,
          div_factor: float = 1e6, keep_terms: bool = False):
    """Born series u_0 = G S, u_{n+1} = G V u_n, psi = sum u_n (Eqs. 18-20)
    with the stop rule of Eq. 30 (L1 row) or the full-grid L2 ratio.

    Returns (psi, info dict, per-term norms, terms array or None)."""
    gh, V, s = _c128(gh), _c128(V), _c128(s)
    sp = _StopParams(max_terms, tol, stop_mode, n // 2 if l1_row is None else l1_row,
                     div_grace, div_window, div_factor)
    info = _SolveInfo()
    psi = np.zeros((n, n), np.complex128)
    norms = np.zeros(max_terms)
    u_all = np.zeros((max_terms, n, n), np.complex128) if keep_terms else None
    rc = _load().ora_tbs_solve(n, m, _p(gh), _p(V), _p(s), C.byref(sp), _p(psi),
                               C.byref(info), _p(norms), _p(u_all))
    if rc != 0:
        raise ValueError("oracle solve failed (%d)" % rc)
    d = dict(terms=info.terms, status=info.status, status_name=STATUS[info.status],
             residual=info.residual, term_norm_max=info.term_norm_max,
             psi_norm=info.psi_norm)
    return psi, d, norms[: info.terms].copy(), (u_all[: info.terms] if keep_terms else None)


def adjoint(n: int, m: int, gh, V, u_all, g):
    """Q = sum_j conj(lambda_{j+1}) u_j of the truncated series' adjoint; the
    gradient of a real loss is Re(Q dV/dtheta) (derivation in tbs_oracle.c)."""
    gh, V, g = _c128(gh), _c128(V), _c128(g)
    u_all = _c128(u_all)
    T = u_all.shape[0]
    Q = np.zeros((n, n), np.complex128)
    if _load().ora_tbs_adjoint(n, m, _p(gh), _p(V), T, _p(u_all), _p(g), _p(Q)) != 0:
        raise ValueError("bad sizes")
    return Q


# --- convenience: one full problem ----------------------------------------

def plan(n: int, dx: float, f: float, c0: float):
    """Spectrum of the cell-averaged Green's table for one (N, k0) pair."""
    k0 = 2.0 * np.pi * f / c0
    m = padded_size(n)
    gc = green_table(n, k0, dx)
    return m, ghat(n, m, dx, gc)


# ---------------------------------------------------------------------------
# The paper's own discretisation: periodic grid, epsilon-shifted spectral G,
# absorbing layer, Eq. 30 row stop (Section 3.1, Algorithm 1)
# ---------------------------------------------------------------------------
class _EpsInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("error", C.c_double)]


def ghat_eps(n: int, dx: float, k0: float, eps: float):
    """g~(p) / N^2 = 1 / ((|p|^2 - k0^2 - i eps) N^2) on the DFT wavenumbers
    (row-major [ky][kx]), for unnormalised transforms (Section 2.2)."""
    gh = np.zeros((n, n), np.complex128)
    if _load().ora_ghat_eps(n, dx, k0, eps, _p(gh)) != 0:
        raise ValueError("n must be a power of two")
    return gh


def abl_profile(n: int, dx: float, zeta: float, width: int):
    """Per-axis absorbing-layer profile: 1 / (1 + exp(-zeta (x - mu/2))) at
    distance x from the nearer edge within mu = width cells, 1 elsewhere."""
    prof = np.zeros(n, np.float64)
    _load().ora_abl_profile(n, dx, zeta, width, _p(prof))
    return prof


def eps_solve(n: int, gh, V, S, abl, max_iter: int, tol: float, row: int | None = None):
    """psi^0 = G S, psi^{l+1} = A . G (V psi^l + S) until Eq. 30's row ratio
    < tol (abl: per-axis profile or None).  Returns (psi, info dict, errors)."""
    gh, V, S = _c128(gh), _c128(V), _c128(S)
    ab = None if abl is None else _f64(abl)
    psi = np.zeros((n, n), np.complex128)
    errs = np.zeros(max(1, max_iter))
    info = _EpsInfo()
    if _load().ora_eps_solve(n, _p(gh), _p(V), _p(S), _p(ab), max_iter, tol, n // 2 if row is None else row,
                             _p(psi), C.byref(info), _p(errs)) != 0:
        raise ValueError("bad sizes")
    return psi, dict(iters=info.iters, status=info.status, error=info.error), errs[:info.iters]


def eps_solve_cbs(n: int, gh, V, S, abl, eps: float, max_iter: int, tol: float, row: int | None = None):
    """The paper's periodic iteration with the convergent Born series
    preconditioner gamma = i V / eps (V = U - i eps, eps >= max |U|):
    psi^0 = G S, psi^{l+1} = A . (psi + gamma (G (V psi + S) - psi)), Eq. 30
    stop.  Returns (psi, info dict, errors)."""
    gh, V, S = _c128(gh), _c128(V), _c128(S)
    ab = None if abl is None else _f64(abl)
    psi = np.zeros((n, n), np.complex128)
    errs = np.zeros(max(1, max_iter))
    info = _EpsInfo()
    if _load().ora_eps_solve_cbs(n, _p(gh), _p(V), _p(S), _p(ab), eps, max_iter, tol,
                                 n // 2 if row is None else row, _p(psi), C.byref(info), _p(errs)) != 0:
        raise ValueError("bad sizes or eps")
    return psi, dict(iters=info.iters, status=info.status, error=info.error), errs[:info.iters]


def vv_kspace(n: int, dx: float, omega: float, alpha0: float, nu: float, v: float, eps: float,
              dispersion: bool = True):
    """VV(p) = eta |p|^(nu+1) - i (tau omega |p|^nu + eps) on the DFT
    wavenumbers, tau = -2 alpha0 v^(nu-1), eta = 2 alpha0 v^nu tan(pi nu/2)
    (Eq. 24, Section 3.1, Algorithm 1 case II); dispersion=False drops the
    eta term (the absorbing, non-dispersive case of Table 2)."""
    tau = -2.0 * alpha0 * v ** (nu - 1.0)
    eta = 2.0 * alpha0 * v ** nu * np.tan(np.pi * nu / 2.0) if dispersion else 0.0
    vv = np.zeros((n, n), np.complex128)
    if _load().ora_vv_kspace(n, dx, omega, eta, tau, nu, eps, _p(vv)) != 0:
        raise ValueError("n must be a power of two")
    return vv


def eps_solve_kspace(n: int, gh, vv, S, abl, max_iter: int, tol: float, row: int | None = None):
    """Case II: psi^0 = G S, psi^{l+1} = A . IDFT(g~ (VV DFT(psi^l) + DFT(S)))
    until Eq. 30 < tol.  Returns (psi, info dict, errors)."""
    gh, vv, S = _c128(gh), _c128(vv), _c128(S)
    ab = None if abl is None else _f64(abl)
    psi = np.zeros((n, n), np.complex128)
    errs = np.zeros(max(1, max_iter))
    info = _EpsInfo()
    if _load().ora_eps_solve_kspace(n, _p(gh), _p(vv), _p(S), _p(ab), max_iter, tol, n // 2 if row is None else row,
                                    _p(psi), C.byref(info), _p(errs)) != 0:
        raise ValueError("bad sizes")
    return psi, dict(iters=info.iters, status=info.status, error=info.error), errs[:info.iters]



def synthesize(fields, dxs, freqs, weights, origin, step, counts, t0: float, dt: float, n_t: int):
    """Time signal s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t) at the
    receiver lattice X = origin + (ix, iy) * step, 0 <= (ix, iy) < counts,
    psi_k bilinear between cell centres i dx_k (indices clamped), with the
    e^{-i omega t} convention of Section 2.2.  fields[k]: [n_rhs][n_k][n_k].
    Returns complex128 [n_rhs][ny][nx][n_t]."""
    fs = [_c128(np.asarray(f).reshape((-1,) + np.asarray(f).shape[-2:])) for f in fields]
    n_rhs = fs[0].shape[0]
    nx, ny = counts
    ptrs = (C.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    ns = np.array([f.shape[-1] for f in fs], np.int32)
    d, fr, w = _f64(dxs), _f64(freqs), _f64(weights)
    out = np.zeros((n_rhs, ny, nx, n_t), np.complex128)
    if _load().ora_synthesize(len(fs), ptrs, ns.ctypes.data_as(C.c_void_p), _p(d), _p(fr), _p(w), n_rhs,
                              float(origin[0]), float(origin[1]), float(step[0]), float(step[1]), nx, ny,
                              float(t0), float(dt), n_t, _p(out)) != 0:
        raise ValueError("every field needs n >= 2 and dx > 0")
    return out
