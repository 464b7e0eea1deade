"""Pins of the complex128 oracle against references other than itself.

Each test checks one oracle routine against something the mathematics or the
paper fixes independently: a textbook DFT, SciPy's Hankel function and
adaptive quadrature, closed forms, a direct O(N^4) convolution sum, a dense
linear solve, reciprocity, the paper's dispersion relation (Eq. 7), the
paper's nonlinear wave equation (Eq. 11) and finite differences.  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")
scipy_integrate = pytest.importorskip("scipy.integrate")

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------

def test_gauss_legendre_matches_numpy(oracle_mod):
    for n in (1, 2, 3, 6, 8, 16, 20, 40):
        x, w = oracle_mod.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        assert np.allclose(x[order], xr, atol=1e-14, rtol=0)
        assert np.allclose(w[order], wr, atol=1e-13, rtol=0)


@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_textbook_dft(oracle_mod, sign):
    rng = np.random.default_rng(1)
    for n in (1, 2, 4, 8, 16, 32, 64):
        a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        j = np.arange(n)
        dft = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        assert np.allclose(oracle_mod.fft(a, sign), dft @ a, atol=1e-12 * max(1, n), rtol=0)


def test_fft_large_and_2d_match_library(oracle_mod):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(4096) + 1j * rng.standard_normal(4096)
    assert rel(oracle_mod.fft(a, -1), np.fft.fft(a)) < 1e-14
    b = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    assert rel(oracle_mod.fft2(b, -1), np.fft.fft2(b)) < 1e-14
    # unnormalised inverse: F^+ F = M^2 I, and Parseval
    assert rel(oracle_mod.fft2(oracle_mod.fft2(b, -1), +1) / 64 ** 2, b) < 1e-14
    assert abs(np.sum(np.abs(oracle_mod.fft2(b)) ** 2) / 64 ** 2 / np.sum(np.abs(b) ** 2) - 1) < 1e-13
    with pytest.raises(ValueError):
        oracle_mod.fft(np.ones(12))


# --------------------------------------------------------------------------
# Green's function (Eq. 16 with epsilon -> 0) and its cell averages
# --------------------------------------------------------------------------

def test_green_point_matches_scipy_hankel(oracle_mod):
    for k0, r in [(1.0, 1e-4), (3.0, 0.7), (2 * np.pi / 8, 17.3), (500.0, 3.1)]:
        ref = 0.25j * scipy_special.hankel1(0, k0 * r)
        assert abs(oracle_mod.green_point(k0, r) - ref) < 1e-14 * max(1.0, abs(ref))


def _cell_mean_scipy(k0, a, b):
    g = lambda y, x: 0.25j * scipy_special.hankel1(0, k0 * math.hypot(x, y))
    if a == 0 and b == 0:
        # polar about the centre, 8 symmetric triangles
        def inner(th):
            R = 0.5 / math.cos(th)
            fr = lambda r: g(0.0, r) * r
            re = scipy_integrate.quad(lambda r: fr(r).real, 0, R, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
            im = scipy_integrate.quad(lambda r: fr(r).imag, 0, R, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
            return re, im
        re = scipy_integrate.quad(lambda t: inner(t)[0], 0, np.pi / 4, epsabs=1e-14, epsrel=1e-13)[0]
        im = scipy_integrate.quad(lambda t: inner(t)[1], 0, np.pi / 4, epsabs=1e-14, epsrel=1e-13)[0]
        return 8 * (re + 1j * im)
    kw = dict(epsabs=1e-14, epsrel=1e-12)
    re = scipy_integrate.dblquad(lambda y, x: g(y, x).real, a - 0.5, a + 0.5, b - 0.5, b + 0.5, **kw)[0]
    im = scipy_integrate.dblquad(lambda y, x: g(y, x).imag, a - 0.5, a + 0.5, b - 0.5, b + 0.5, **kw)[0]
    return re + 1j * im


@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (1, 1), (3, 2), (4, 1), (9, 7), (30, 2)])
def test_green_cell_matches_adaptive_quadrature(oracle_mod, ab):
    # dx = 1, lambda = 8 cells (the lambda/8 grids of every workload) and the
    # coarser 4 points per wavelength of the 2nd harmonic
    for k0 in (2 * np.pi / 8, 2 * np.pi / 4):
        got = oracle_mod.green_cell(k0, 1.0, *ab)
        ref = _cell_mean_scipy(k0, *ab)
        assert abs(got - ref) < 1e-10 * abs(ref), (ab, k0, got, ref)


def test_green_cell_scales_with_dx(oracle_mod):
    # the cell average depends on (k0 dx, offset) only
    assert abs(oracle_mod.green_cell(2.0, 0.5, 3, 1) - oracle_mod.green_cell(1.0, 1.0, 3, 1)) < 1e-14


def test_self_cell_small_kh_closed_form(oracle_mod):
    # g(r) ~ i/4 - (ln(k r/2) + gamma)/(2 pi) for small k r, and the mean of
    # ln r over a square of side h is ln(h/2) + (ln 2 - 3 + pi/2)/2.
    k, h = 1e-3, 1.0
    mean_ln = math.log(h / 2) + (math.log(2) - 3 + math.pi / 2) / 2
    ref = 0.25j - (math.log(k / 2) + np.euler_gamma + mean_ln) / (2 * math.pi)
    got = oracle_mod.green_cell(k, h, 0, 0)
    assert abs(got - ref) < 1e-5


def test_green_table_symmetry(oracle_mod):
    gc = oracle_mod.green_table(9, 2 * np.pi / 8, 1.0)
    assert np.allclose(gc, gc.T, atol=1e-15, rtol=0)  # Gc[(a,b)] = Gc[(b,a)]
    assert abs(gc[3, 5] - oracle_mod.green_cell(2 * np.pi / 8, 1.0, -5, 3)) < 1e-15


# --------------------------------------------------------------------------
# G as zero-padded FFT convolution
# --------------------------------------------------------------------------

def _direct_matrix(gc, n, dx):
    yy, xx = np.divmod(np.arange(n * n), n)
    dy = np.abs(yy[:, None] - yy[None, :])
    dxo = np.abs(xx[:, None] - xx[None, :])
    return dx * dx * gc[dy, dxo]


@pytest.mark.parametrize("n,m", [(12, 32), (12, 64), (17, 64)])
def test_convolution_matches_direct_sum(oracle_mod, n, m):
    rng = np.random.default_rng(3)
    k0, dx = 2 * np.pi / (8 * 0.3), 0.3
    gc = oracle_mod.green_table(n, k0, dx)
    gh = oracle_mod.ghat(n, m, dx, gc)
    f = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = _direct_matrix(gc, n, dx)
    assert rel(oracle_mod.apply_g(n, m, gh, f), (A @ f.ravel()).reshape(n, n)) < 1e-12
    # G^H: convolution with conj(Gc)
    assert rel(oracle_mod.apply_g(n, m, gh, f, conj_kernel=True),
               (A.conj() @ f.ravel()).reshape(n, n)) < 1e-12
    with pytest.raises(ValueError):
        oracle_mod.ghat(n, 16, dx, gc)  # M < 2N - 1 would alias


def test_ghat_even_and_transpose_symmetric(oracle_mod):
    n, m = 10, 32
    gc = oracle_mod.green_table(n, 2 * np.pi / 8, 1.0)
    gh = oracle_mod.ghat(n, m, 1.0, gc)
    idx = (-np.arange(m)) % m
    assert np.allclose(gh, gh[idx, :], atol=1e-15)
    assert np.allclose(gh, gh[:, idx], atol=1e-15)
    assert np.allclose(gh, gh.T, atol=1e-15)


@pytest.mark.parametrize("dx", [1.0, 0.25])
def test_homogeneous_field_is_hankel_superposition(oracle_mod, dx):
    # V = 0: psi = u_0 = sum_j a_j Gc[. - n_j] exactly, and the series stops
    # after one term (u_1 = 0).  Away from the sources the cell average
    # approaches the point Hankel field with offset 1 - (k0 dx)^2/24.  The
    # grid is 8 cells per wavelength at either cell size (dx != 1 exposes a
    # lost dx^2 in the source deposit or the spectrum scale).
    n, k0 = 40, 2 * np.pi / (8 * dx)
    m = oracle_mod.padded_size(n)
    gc = oracle_mod.green_table(n, k0, dx)
    gh = oracle_mod.ghat(n, m, dx, gc)
    ix = np.array([5, 17, 30], np.int32)
    iy = np.array([3, 3, 8], np.int32)
    amp = np.array([1.0, 0.5 - 0.25j, -0.8j])
    s = oracle_mod.deposit_points(n, dx, ix, iy, amp)
    psi, info, norms, _ = oracle_mod.solve(n, m, gh, np.zeros((n, n)), s, 10, 1e-12)
    yy, xx = np.mgrid[0:n, 0:n]
    ref = sum(a * gc[np.abs(yy - y), np.abs(xx - x)] for x, y, a in zip(ix, iy, amp))
    assert rel(psi, ref) < 1e-12
    assert info["terms"] == 2 and info["status_name"] == "CONVERGED"
    far = (yy > 25)
    r = [np.hypot(yy - y, xx - x) * dx for x, y in zip(ix, iy)]
    hank = sum(a * 0.25j * scipy_special.hankel1(0, k0 * rr) for a, rr in zip(amp, r))
    assert rel(psi[far], hank[far] * (1 - (k0 * dx) ** 2 / 24)) < 3e-3


# --------------------------------------------------------------------------
# the series (Eqs. 18-20)
# --------------------------------------------------------------------------

def _small_problem(oracle_mod, n=12, seed=4, scale=0.15):
    rng = np.random.default_rng(seed)
    dx, k0 = 1.0, 2 * np.pi / 8
    m = oracle_mod.padded_size(n)
    gc = oracle_mod.green_table(n, k0, dx)
    gh = oracle_mod.ghat(n, m, dx, gc)
    V = scale * k0 ** 2 * (rng.standard_normal((n, n)) + 1j * rng.random((n, n)))
    s = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return n, m, dx, gc, gh, V, s


def test_converged_series_matches_dense_solve(oracle_mod):
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod)
    A = _direct_matrix(gc, n, dx)
    psi_ref = np.linalg.solve(np.eye(n * n) - A * V.ravel()[None, :], A @ s.ravel())
    psi, info, _, _ = oracle_mod.solve(n, m, gh, V, s, 400, 1e-15)
    assert info["status_name"] == "CONVERGED", info
    assert rel(psi.ravel(), psi_ref) < 1e-11


def test_truncated_series_matches_matrix_powers(oracle_mod):
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=10, seed=5, scale=0.4)
    A = _direct_matrix(gc, n, dx)
    AD = A * V.ravel()[None, :]
    u = A @ s.ravel()
    ref = np.zeros_like(u)
    for _ in range(7):
        ref += u
        u = AD @ u
    psi, info, _, _ = oracle_mod.solve(n, m, gh, V, s, 7, 0.0)
    assert info["terms"] == 7 and info["status_name"] == "MAX_TERMS"
    assert rel(psi.ravel(), ref) < 1e-12


def test_lippmann_schwinger_residual_identity(oracle_mod):
    # psi_T - u_0 - G V psi_T = -u_T exactly (Eq. 17 truncated)
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=16, seed=6)
    psi, info, _, u = oracle_mod.solve(n, m, gh, V, s, 7, 0.0, keep_terms=True)
    u_next = oracle_mod.apply_g(n, m, gh, V * u[-1])
    resid = psi - u[0] - oracle_mod.apply_g(n, m, gh, V * psi)
    assert rel(resid, -u_next) < 1e-11


def test_reciprocity_with_complex_potential(oracle_mod):
    # (G V)^n G is symmetric for even Gc and diagonal V: u_p[q] = u_q[p]
    n, m, dx, gc, gh, V, _ = _small_problem(oracle_mod, n=20, seed=7, scale=0.3)
    p, q = (3, 4), (15, 11)
    sp = oracle_mod.deposit_points(n, dx, [p[0]], [p[1]], [1.0])
    sq = oracle_mod.deposit_points(n, dx, [q[0]], [q[1]], [1.0])
    for T in (1, 3, 6):
        up, _, _, _ = oracle_mod.solve(n, m, gh, V, sp, T, 0.0)
        uq, _, _, _ = oracle_mod.solve(n, m, gh, V, sq, T, 0.0)
        a, b = up[q[1], q[0]], uq[p[1], p[0]]
        assert abs(a - b) < 1e-12 * abs(a)


def test_stop_rule_l2(oracle_mod):
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=16, seed=8, scale=0.25)
    psi, info, norms, u = oracle_mod.solve(n, m, gh, V, s, 60, 1e-6, keep_terms=True)
    T = info["terms"]
    assert info["status_name"] == "CONVERGED" and 2 < T < 60
    partial = np.cumsum(u, axis=0)
    r = np.array([np.linalg.norm(u[k]) / np.linalg.norm(partial[k]) for k in range(T)])
    assert np.all(r[:-1] >= 1e-6) and r[-1] < 1e-6
    assert abs(info["residual"] - r[-1]) < 1e-12 * r[-1]
    assert np.allclose(norms, [np.linalg.norm(x) for x in u], rtol=1e-13)
    assert rel(psi, partial[-1]) < 1e-14


def test_stop_rule_l1_row_eq30(oracle_mod):
    # Eq. 30: sum_m |psi_{l+1}(row,m) - psi_l(row,m)| / sum_m |psi_l(row,m)|
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=16, seed=9, scale=0.25)
    row = 7
    psi, info, _, u = oracle_mod.solve(n, m, gh, V, s, 60, 1e-5, stop_mode=oracle_mod.STOP_L1_ROW,
                                       l1_row=row, keep_terms=True)
    partial = np.cumsum(u, axis=0)
    T = info["terms"]
    err = [np.sum(np.abs(partial[l + 1][row] - partial[l][row])) / np.sum(np.abs(partial[l][row]))
           for l in range(T - 1)]
    assert info["status_name"] == "CONVERGED"
    assert all(e >= 1e-5 for e in err[:-1]) and err[-1] < 1e-5


def test_divergence_and_nonfinite_flags(oracle_mod):
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=12, seed=10)
    k0 = 2 * np.pi / 8
    Vbig = np.full((n, n), 8.0 * k0 ** 2 + 0j)
    _, info, norms, _ = oracle_mod.solve(n, m, gh, Vbig, s, 200, 1e-6)
    assert info["status_name"] == "DIVERGED"
    assert norms[-1] > norms[-2] > norms[-3]
    Vnan = V.copy()
    Vnan[3, 4] = np.nan
    _, info, _, _ = oracle_mod.solve(n, m, gh, Vnan, s, 20, 1e-6)
    assert info["status_name"] == "NONFINITE" and info["terms"] == 2


# --------------------------------------------------------------------------
# potential (Eqs. 3, 4, 7, 13, 25) and the nonlinear source (Eqs. 11, 28b)
# --------------------------------------------------------------------------

def test_potential_lossless_closed_form(oracle_mod):
    f, c0 = 1e6, 1500.0
    c = np.array([1500.0, 1530.0, 1350.0, 1800.0])
    w = 2 * np.pi * f
    V = oracle_mod.potential(f, c0, c)
    assert np.allclose(V, (w / c) ** 2 - (w / c0) ** 2, rtol=1e-14, atol=0)
    assert V[0] == 0


def test_potential_satisfies_paper_dispersion_relation(oracle_mod):
    # Eq. 7 for a plane wave exp(i p x): p^2 = w^2/v^2 - i tau w p^y + eta p^(y+1)
    # with tau = -2 a0 v^(y-1), eta = 2 a0 v^y tan(pi y/2) (Eq. 4).  To first
    # order in a0 its root is the oracle's p with no reference frequency.
    for y in (1.1, 1.5, 1.7):
        f, v = 3e6, 1540.0
        w = 2 * np.pi * f
        a0 = 2e-12 * (1.0 / w) ** (y - 1.5)
        alpha = a0 * w ** y
        V = oracle_mod.potential(f, v, np.array([v]), np.array([alpha]), y, f_ref=0.0)[0]
        p = np.sqrt(V + (w / v) ** 2)
        tau, eta = -2 * a0 * v ** (y - 1), 2 * a0 * v ** y * math.tan(math.pi * y / 2)
        res = p ** 2 - ((w / v) ** 2 - 1j * tau * w * p ** y + eta * p ** (y + 1))
        assert abs(res) < 1e-3 * abs(p ** 2 - (w / v) ** 2), (y, res)
        assert abs(p.imag - alpha) < 1e-9 * alpha  # Im p = alpha = a0 w^y (Eq. 3)


def test_potential_reference_frequency(oracle_mod):
    # c is the phase speed at f_ref: at f = f_ref, Re p = w/c exactly
    f = 5e6
    c = np.array([1540.0, 1500.0])
    al = np.array([33.8, 10.0])
    V = oracle_mod.potential(f, 1540.0, c, al, 1.1, f_ref=f)
    p = np.sqrt(V + (2 * np.pi * f / 1540.0) ** 2)
    assert np.allclose(p.real, 2 * np.pi * f / c, rtol=1e-13)
    assert np.allclose(p.imag, al, rtol=1e-12)


def test_paper_parameters_golden(oracle_mod):
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"]
    f = g["bin_multiple"]["value"] * v / (n * dx)
    assert abs(f - g["f_hz"]["value"]) < 0.5
    kf = 2 * np.pi * g["f_hz"]["value"] / v
    assert round(kf * g["scatterer_radius_m"]["value"], g["kfa"]["digits"]) == g["kfa"]["value"]
    # inside the disk the potential is k_s^2 - k_f^2 (Eq. 25, epsilon = 0)
    vs = np.array(g["v_s_values"]["value"])
    V = oracle_mod.potential(g["f_hz"]["value"], v, vs)
    ks = 2 * np.pi * g["f_hz"]["value"] / vs
    assert np.allclose(V, ks ** 2 - kf ** 2, rtol=1e-13)


def test_harmonic2_source_from_nonlinear_wave_equation(oracle_mod):
    # Eq. 11: lap P - P_tt/c^2 + xi (P^2)_tt = -S cos(wt).  With
    # P = Re(psi1 e^{-iwt}), the e^{-2iwt} phasor of -xi (P^2)_tt is the right
    # side R2 of lap psi2 + k2^2 psi2 = R2; in the form lap psi + k^2 psi = -S
    # the second-harmonic source is S2 = -R2 (Eq. 28b).
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    beta = 1.0 + g["ba"]["value"] / 2.0
    rng = np.random.default_rng(11)
    psi1 = (rng.standard_normal(5) + 1j * rng.standard_normal(5)) * 3e5
    c = np.array([1500.0, 1450.0, 1520.0, 1500.0, 1600.0])
    rho = np.full(5, 1000.0)
    w = 2 * np.pi * 2e6
    xi = beta / (rho * c ** 4)
    nt = 64
    t = np.arange(nt) / nt * (2 * np.pi / w)
    P = np.real(psi1[:, None] * np.exp(-1j * w * t[None, :]))
    sq = P ** 2
    coef = np.fft.fft(sq, axis=1) / nt  # sq = sum_q coef_q e^{+i q w t}
    q = np.fft.fftfreq(nt, 1.0 / nt)
    d2 = np.real(np.fft.ifft(coef * nt * (1j * q * w) ** 2, axis=1))  # (P^2)_tt
    rhs = -xi[:, None] * d2
    # phasor of e^{-2iwt}: R2 = (2/T) int rhs e^{+2iwt} dt
    R2 = 2.0 * np.mean(rhs * np.exp(2j * w * t[None, :]), axis=1)
    s2 = oracle_mod.harmonic2_source(w, np.full(5, beta), rho, c, psi1)
    assert np.allclose(s2, -R2, rtol=1e-10, atol=0)


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_harmonic_sum_term_sources_from_nonlinear_wave_equation(oracle_mod, order):
    # With only psi_1 .. psi_{n-1} present, the e^{-inwt} phasor of
    # -xi (P^2)_tt, P = Re sum_k psi_k e^{-ikwt}, holds exactly the sum terms
    # psi_i psi_j, i + j = n (no difference term can reach n): it is -S_n
    rng = np.random.default_rng(20 + order)
    k = order - 1
    lower = [(rng.standard_normal(5) + 1j * rng.standard_normal(5)) * 3e5 / (j + 1) for j in range(k)]
    c = np.array([1500.0, 1450.0, 1520.0, 1500.0, 1600.0])
    rho = np.full(5, 1000.0)
    beta = np.full(5, 3.5)
    w = 2 * np.pi * 1e6
    xi = beta / (rho * c ** 4)
    nt = 64
    t = np.arange(nt) / nt * (2 * np.pi / w)
    P = np.real(sum(lower[j][:, None] * np.exp(-1j * (j + 1) * w * t[None, :]) for j in range(k)))
    coef = np.fft.fft(P ** 2, axis=1) / nt
    q = np.fft.fftfreq(nt, 1.0 / nt)
    rhs = -xi[:, None] * np.real(np.fft.ifft(coef * nt * (1j * q * w) ** 2, axis=1))
    Rn = 2.0 * np.mean(rhs * np.exp(1j * order * w * t[None, :]), axis=1)
    sn = oracle_mod.harmonic_source(order, w, beta, rho, c, lower)
    assert np.allclose(sn, -Rn, rtol=1e-10, atol=0)
    if order == 2:
        assert np.allclose(sn, oracle_mod.harmonic2_source(w, beta, rho, c, lower[0]), rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# adjoint of the truncated series
# --------------------------------------------------------------------------

def test_adjoint_dot_product(oracle_mod):
    # <g, L dV> = sum Q dV for the tangent map L: dV -> d psi (complex-linear)
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=14, seed=12, scale=0.2)
    rng = np.random.default_rng(13)
    T = 6
    dV = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 1e-4 * np.abs(V).max() / np.abs(dV).max()
    pp, _, _, _ = oracle_mod.solve(n, m, gh, V + h * dV, s, T, 0.0)
    pm, _, _, _ = oracle_mod.solve(n, m, gh, V - h * dV, s, T, 0.0)
    LdV = (pp - pm) / (2 * h)
    _, _, _, u = oracle_mod.solve(n, m, gh, V, s, T, 0.0, keep_terms=True)
    Q = oracle_mod.adjoint(n, m, gh, V, u, g)
    lhs = np.vdot(g, LdV)
    rhs = np.sum(Q * dV)
    assert abs(lhs - rhs) < 1e-7 * abs(lhs)


def test_truncated_adjoint_converges_to_dense_adjoint(oracle_mod):
    # For the converged series psi = (I - A V)^-1 A s, d psi = (I - A V)^-1 A
    # (dV psi), so <g, d psi> = sum Q dV with Q = (g^H (I - A V)^-1 A) * psi:
    # the truncated adjoint's Q must reach it once the series has converged
    n, m, dx, gc, gh, V, s = _small_problem(oracle_mod, n=10, seed=15, scale=0.15)
    rng = np.random.default_rng(16)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = _direct_matrix(gc, n, dx)
    K = np.eye(n * n) - A * V.ravel()[None, :]
    psi_ref = np.linalg.solve(K, A @ s.ravel())
    row = np.linalg.solve(K.T, np.conj(g.ravel())) @ A  # g^H K^-1 A
    Q_ref = row * psi_ref
    psi, info, _, u = oracle_mod.solve(n, m, gh, V, s, 300, 0.0, keep_terms=True)
    Q = oracle_mod.adjoint(n, m, gh, V, u, g)
    assert rel(psi.ravel(), psi_ref) < 1e-11
    assert rel(Q.ravel(), Q_ref) < 1e-10


def _cylinder_scattered(k0, k1, a, src, obs, nmax=40):
    """Scattered field of a unit line source (i/4) H0(k0 |r - src|) by a
    penetrable circular cylinder (radius a, centre 0, interior wavenumber
    k1, same density): separation of variables, continuity of u and du/dr
    at r = a (Graf's addition theorem for the incident field)."""
    from scipy import special as sp
    rs, ths = np.hypot(*src), np.arctan2(src[1], src[0])
    r, th = np.hypot(*obs), np.arctan2(obs[1], obs[0])
    out = np.zeros(r.shape, complex)
    for q in range(-nmax, nmax + 1):
        j0, dj0 = sp.jv(q, k0 * a), sp.jvp(q, k0 * a)
        j1, dj1 = sp.jv(q, k1 * a), sp.jvp(q, k1 * a)
        h0, dh0 = sp.hankel1(q, k0 * a), sp.h1vp(q, k0 * a)
        cq = 0.25j * sp.hankel1(q, k0 * rs) * (k1 * j0 * dj1 - k0 * dj0 * j1) / (k0 * dh0 * j1 - k1 * h0 * dj1)
        out += cq * sp.hankel1(q, k0 * r) * np.exp(1j * q * (th - ths))
    return out


def test_penetrable_cylinder_matches_separation_of_variables(oracle_mod):
    # Physics, not parity: a disk of radius 1 wavelength with k1 = 1.1 k0, a
    # unit point source 2.5 wavelengths from its centre, series converged.
    # The grid's scattered field psi - G S approaches the analytic series at
    # second order in dx (staircased boundary, cell-averaged G).
    pytest.importorskip("scipy")
    errs = []
    for ppw in (16, 32):
        dx = 1.0 / ppw
        n = 6 * ppw
        ic = n // 2
        yy, xx = np.mgrid[0:n, 0:n]
        X, Y = (xx - ic) * dx, (yy - ic) * dx
        c = np.where(X ** 2 + Y ** 2 <= 1.0, 1.0 / 1.1, 1.0)
        m, gh = oracle_mod.plan(n, dx, 1.0, 1.0)  # k0 = 2 pi
        V = oracle_mod.potential(1.0, 1.0, c, None, 1.0, 1.0)
        sx = ic + int(round(2.5 / dx))
        S = oracle_mod.deposit_points(n, dx, [sx], [ic], [1.0])
        psi, info, _, _ = oracle_mod.solve(n, m, gh, V, S, 200, 1e-12)
        assert info["status_name"] == "CONVERGED"
        sc = psi - oracle_mod.apply_g(n, m, gh, S)
        obs = (np.hypot(X, Y) > 1.0 + 3 * dx) & (np.hypot(X - (sx - ic) * dx, Y) > 3 * dx)
        ua = _cylinder_scattered(2 * np.pi, 2.2 * np.pi, 1.0, ((sx - ic) * dx, 0.0), (X[obs], Y[obs]))
        errs.append(rel(sc[obs], ua))
    assert errs[0] < 0.04 and errs[1] < 0.012, errs
    assert errs[0] / errs[1] > 2.5, errs


def test_adjoint_gradient_matches_finite_differences(oracle_mod):
    # J = 1/2 sum_s sum_row |psi_s - d_s|^2; dJ/dc and dJ/dalpha at random
    # pixels by central differences through the whole chain c, alpha -> V -> psi
    n, dx_cells = 16, 1.0
    f, c0, y, fref = 1e6, 1500.0, 1.5, 0.6e6
    dx = c0 / f / 8.0
    rng = np.random.default_rng(14)
    c = c0 * (1 + 0.05 * rng.standard_normal((n, n)))
    al = 40.0 * (1 + rng.random((n, n)))
    m = oracle_mod.padded_size(n)
    gh = oracle_mod.ghat(n, m, dx, oracle_mod.green_table(n, 2 * np.pi * f / c0, dx))
    srcs = [oracle_mod.deposit_points(n, dx, [x], [1], [1.0]) for x in (2, 8, 13)]
    row = n - 2
    data = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in srcs]
    T = 6

    def J(cc, aa):
        V = oracle_mod.potential(f, c0, cc, aa, y, fref)
        tot = 0.0
        for s, d in zip(srcs, data):
            psi, _, _, _ = oracle_mod.solve(n, m, gh, V, s, T, 0.0)
            tot += 0.5 * np.sum(np.abs(psi[row] - d) ** 2)
        return tot

    V = oracle_mod.potential(f, c0, c, al, y, fref)
    dVdc, dVda = oracle_mod.potential_derivs(f, c, al, y, fref)
    Q = np.zeros((n, n), complex)
    for s, d in zip(srcs, data):
        psi, _, _, u = oracle_mod.solve(n, m, gh, V, s, T, 0.0, keep_terms=True)
        g = np.zeros((n, n), complex)
        g[row] = psi[row] - d
        Q += oracle_mod.adjoint(n, m, gh, V, u, g)
    gc_, ga_ = np.real(Q * dVdc), np.real(Q * dVda)
    pix = [(int(a), int(b)) for a, b in rng.integers(0, n, (12, 2))]
    for (py, px) in pix:
        e = np.zeros((n, n))
        e[py, px] = 1.0
        hc, ha = 1e-4 * c[py, px], 1e-4 * al[py, px]
        fd_c = (J(c + hc * e, al) - J(c - hc * e, al)) / (2 * hc)
        fd_a = (J(c, al + ha * e) - J(c, al - ha * e)) / (2 * ha)
        assert abs(fd_c - gc_[py, px]) <= 1e-6 * abs(fd_c) + 1e-12 * np.abs(gc_).max()
        assert abs(fd_a - ga_[py, px]) <= 1e-6 * abs(fd_a) + 1e-12 * np.abs(ga_).max()

# --------------------------------------------------------------------------
# the paper's own discretisation: periodic grid, epsilon-shifted spectral G,
# absorbing layer, Eq. 30 row stop (Section 3.1, Algorithm 1)
# --------------------------------------------------------------------------

def test_eps_iteration_without_layer_solves_periodic_helmholtz(oracle_mod):
    # V = U - i eps: the fixed point of psi = G_eps (V psi + S) solves
    # (|p|^2 - k0^2) psi^ - (U psi)^ = S^ on the periodic grid (i eps cancels);
    # dense solve in the Fourier basis, absorbing U so the problem is regular
    n, dx = 16, 0.1
    k0 = 2 * np.pi / (8 * dx)
    eps = 0.8 * k0 * k0
    rng = np.random.default_rng(3)
    U = eps * (0.2 * rng.standard_normal((n, n)) + 1j * (0.3 + 0.1 * rng.random((n, n))))
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    psi, info, _ = oracle_mod.eps_solve(n, oracle_mod.ghat_eps(n, dx, k0, eps), U - 1j * eps, S, None, 3000, 1e-15)
    assert info["status"] == 0
    p = 2 * np.pi * np.fft.fftfreq(n, dx)
    F = np.fft.fft2(np.eye(n * n).reshape(n * n, n, n), axes=(1, 2)).reshape(n * n, n * n).T
    L = np.linalg.inv(F) @ np.diag((p[None, :] ** 2 + p[:, None] ** 2 - k0 ** 2).ravel()) @ F - np.diag(U.ravel())
    ref = np.linalg.solve(L, S.ravel()).reshape(n, n)
    assert rel(psi, ref) < 1e-12


def test_eps_green_impulse_response_is_lossy_hankel(oracle_mod):
    # G_eps applied to a unit point source approaches (i/4) H0(kappa r),
    # kappa = sqrt(k0^2 + i eps), the Green's function of Eq. 16 with finite
    # eps, as the grid is refined (band-limited spectrum)
    sp = pytest.importorskip("scipy.special")
    errs = []
    for ppw, n in ((8, 128), (16, 256), (32, 512)):
        dx = 1.0 / ppw
        k0 = 2 * np.pi
        eps = 0.8 * k0 * k0
        gh = oracle_mod.ghat_eps(n, dx, k0, eps)
        S = np.zeros((n, n), complex)
        S[n // 2, n // 2] = 1.0 / (dx * dx)
        w = np.fft.ifft2(np.fft.fft2(S) * gh * n * n)
        yy, xx = np.mgrid[0:n, 0:n]
        r = np.hypot(xx - n // 2, yy - n // 2) * dx
        m = (r >= 0.5) & (r <= 2.0)
        errs.append(rel(w[m], 0.25j * sp.hankel1(0, np.sqrt(k0 * k0 + 1j * eps) * r[m])))
    assert errs[0] < 0.02 and errs[1] < 3e-3 and errs[2] < 5e-4, errs


def test_abl_profile_is_the_sigmoid(oracle_mod):
    # Eq. 29 within mu of each edge, 1 inside; symmetric
    n, dx, zeta, width = 64, 0.5, 0.7, 10
    prof = oracle_mod.abl_profile(n, dx, zeta, width)
    mu = width * dx
    for e in (0, 3, 5, 9):
        f = 1.0 / (1.0 + np.exp(-zeta * (e * dx - 0.5 * mu)))
        assert abs(prof[e] - f) < 1e-15 and abs(prof[n - 1 - e] - f) < 1e-15
    assert abs(prof[5] - 0.5) < 1e-15
    assert np.all(prof[width:n - width] == 1.0)


def test_paper_homogeneous_case_converges_in_table2_iterations(oracle_mod):
    # The paper's 4096^2 homogeneous lossless run (Section 3.1, Algorithm 1):
    # 501 point sources S = -1e6 i on column 675 around row 2049 (1-based),
    # f = 1.00708 MHz, eps = 0.8 k^2, sigmoid layer zeta = 21.48 Np/cm over
    # 450 cells, Eq. 30 on row 2049 to 1e-5.  Table 2 prints 135 (GPU) and
    # 133 (CPU) iterations.  With the readings here (0-based column 675, the
    # layer's distance counted from each edge's first cell, corners as
    # products) the count is 143: 5.9% and 7.5% above the printed ones.  The
    # same excess appears on the two k-space runs below and on the harmonic
    # runs, and none of the other readings tried (row L2, full-grid L1, layer
    # from the cell centre, min at the corners, layer on psi^0) moves the
    # count, so it is pinned as an excess of 4-8% over every printed count.
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    k0 = 2 * np.pi * f / v
    eps = g["eps_factor"]["value"] * k0 * k0
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    S = np.zeros((n, n), complex)
    S[row - half:row + half + 1, g["source_column"]["value"]] = complex(*g["source_amplitude"]["value"])
    V = np.full((n, n), -1j * eps)
    abl = oracle_mod.abl_profile(n, dx, g["abl_zeta_np_per_m"]["value"], g["abl_width_cells"]["value"])
    _, info, errs = oracle_mod.eps_solve(n, oracle_mod.ghat_eps(n, dx, k0, eps), V, S, abl, 2000,
                                         g["stop_tol"]["value"], row=row)
    it = g["iterations_homogeneous"]["value"]
    assert info["status"] == 0
    assert all(1.04 <= info["iters"] / v <= 1.08 for v in it.values()), (info, it)
    assert np.all(errs[-20:] < 1e-2)  # the last stretch converges, no stall


def test_kspace_potential_matches_paper_tau_eta(oracle_mod):
    # Section 3.1 / Table 3: tau = -2 alpha0 v^(nu-1) = -4.3e-8, eta = 2 alpha0
    # v^nu tan(pi nu / 2) = -6.4e-5 for alpha0 = 5.5e-10, nu = 1.5, v = 1500;
    # VV at a wavenumber p is eta p^(nu+1) - i (tau omega p^nu + eps)
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    a0, nu, v = g["alpha0"]["value"], g["nu"]["value"], g["v_f"]["value"]
    n, dx, w, eps = 16, 1e-4, 2 * np.pi * 1e6, 3.0
    vv = oracle_mod.vv_kspace(n, dx, w, a0, nu, v, eps)
    dp = 2 * np.pi / (n * dx)
    p = dp * np.hypot(3, -5)  # entry (ky, kx) = (-5, 3) sits at row n - 5, column 3
    tau = round(-2 * a0 * v ** (nu - 1), g["tau"]["digits"])
    eta = round(2 * a0 * v ** nu * np.tan(np.pi * nu / 2), g["eta"]["digits"])
    assert tau == g["tau"]["value"] and eta == g["eta"]["value"]
    tau_x = -2 * a0 * v ** (nu - 1)
    eta_x = 2 * a0 * v ** nu * np.tan(np.pi * nu / 2)
    expect = eta_x * p ** (nu + 1) - 1j * (tau_x * w * p ** nu + eps)
    assert abs(vv[n - 5, 3] - expect) < 1e-12 * abs(expect)


def test_kspace_iteration_without_layer_has_closed_form(oracle_mod):
    # Case II without the layer on a homogeneous medium is diagonal in k:
    # psi^ = S^ / (|p|^2 - k^2 - i eps - VV(p)) at the fixed point
    v, f, nu, a0 = 1500.0, 1e6, 1.5, 2e-8
    w = 2 * np.pi * f
    k0 = w / v
    dx = v / f / 8
    eps = 0.8 * k0 * k0
    n = 32
    gh = oracle_mod.ghat_eps(n, dx, k0, eps)
    vv = oracle_mod.vv_kspace(n, dx, w, a0, nu, v, eps)
    rng = np.random.default_rng(7)
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    psi, info, _ = oracle_mod.eps_solve_kspace(n, gh, vv, S, None, 2000, 1e-14)
    assert info["status"] == 0
    p = 2 * np.pi * np.fft.fftfreq(n, dx)
    ref = np.fft.ifft2(np.fft.fft2(S) / (p[None, :] ** 2 + p[:, None] ** 2 - k0 ** 2 - 1j * eps - vv))
    assert rel(psi, ref) < 1e-12


def test_paper_absorbing_dispersive_case_converges_in_table2_iterations(oracle_mod):
    # Section 3.1's absorbing-dispersive run: the homogeneous geometry with
    # the k-space potential (alpha0 = 5.5e-10, nu = 1.5); Table 2 prints 132
    # (GPU) and 131 (CPU) iterations; the readings of the homogeneous pin give
    # 141, the same 4-8% excess
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    k0 = 2 * np.pi * f / v
    eps = g["eps_factor"]["value"] * k0 * k0
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    S = np.zeros((n, n), complex)
    S[row - half:row + half + 1, g["source_column"]["value"]] = complex(*g["source_amplitude"]["value"])
    abl = oracle_mod.abl_profile(n, dx, g["abl_zeta_np_per_m"]["value"], g["abl_width_cells"]["value"])
    vv = oracle_mod.vv_kspace(n, dx, 2 * np.pi * f, g["alpha0"]["value"], g["nu"]["value"], v, eps)
    _, info, errs = oracle_mod.eps_solve_kspace(n, oracle_mod.ghat_eps(n, dx, k0, eps), vv, S, abl, 2000,
                                                g["stop_tol"]["value"], row=row)
    it = g["iterations_absorbing_dispersive"]["value"]
    assert info["status"] == 0
    assert all(1.04 <= info["iters"] / v <= 1.08 for v in it.values()), (info, it)



# ---- broadband synthesis (inverse Fourier sum over single-frequency fields)

def test_synthesis_of_bilinear_fields_is_exact(oracle_mod):
    # fields a + b x + c y (x, y at the cell centres i dx) are reproduced
    # exactly by bilinear interpolation anywhere inside each grid, on grids
    # of different spacing; b != c catches a transposed lookup, the dx of
    # each grid its own scaling
    rng = np.random.default_rng(3)
    grids = [(17, 1.0e-4), (33, 0.5e-4), (24, 0.7e-4)]
    coef = rng.standard_normal((3, 2, 3)) + 1j * rng.standard_normal((3, 2, 3))  # [k][rhs][a, b, c]
    fields = []
    for k, (n, dx) in enumerate(grids):
        y, x = np.mgrid[0:n, 0:n] * dx
        fields.append(np.stack([coef[k, r, 0] + coef[k, r, 1] * x * 1e4 + coef[k, r, 2] * y * 1e4
                                for r in range(2)]))
    freqs = np.array([1.0e6, 1.7e6, 2.3e6])
    w = np.array([0.5, 1.0, 2.0])
    origin, step, counts = (0.13e-3, 0.21e-3), (0.11e-3, 0.09e-3), (9, 7)
    t0, dt, nt = 1e-7, 3.1e-8, 40
    s = oracle_mod.synthesize(fields, [g[1] for g in grids], freqs, w, origin, step, counts, t0, dt, nt)
    X = origin[0] + np.arange(counts[0]) * step[0]
    Y = origin[1] + np.arange(counts[1]) * step[1]
    t = t0 + np.arange(nt) * dt
    for r in range(2):
        ref = np.zeros((counts[1], counts[0], nt), complex)
        for k in range(3):
            v = coef[k, r, 0] + coef[k, r, 1] * X[None, :] * 1e4 + coef[k, r, 2] * Y[:, None] * 1e4
            ref += w[k] * v[:, :, None] * np.exp(-2j * np.pi * freqs[k] * t)[None, None, :]
        assert rel(s[r], ref) < 1e-13


def test_synthesis_on_a_frequency_comb_is_the_dft(oracle_mod):
    # f_k = k df, t_j = j / (K df), one constant field per frequency: the sum
    # is the forward DFT sum_k c_k w_k e^{-2 pi i k j / K} (numpy's fft),
    # which fixes the sign of the e^{-i omega t} convention
    K, df = 16, 0.25e6
    rng = np.random.default_rng(4)
    c = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    w = rng.uniform(0.5, 1.5, K)
    fields = [np.full((1, 4, 4), c[k]) for k in range(K)]
    s = oracle_mod.synthesize(fields, [1e-4] * K, df * np.arange(K), w, (1e-4, 2e-4), (0, 0), (1, 1), 0.0,
                              1.0 / (K * df), K)
    assert rel(s[0, 0, 0], np.fft.fft(c * w)) < 1e-13


def test_synthesis_samples_nodes_and_clamps_outside(oracle_mod):
    # on a cell centre the sample is the stored value; beyond the grid it is
    # the edge value (nearest clamped index)
    rng = np.random.default_rng(5)
    n, dx = 9, 2e-4
    a = rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))
    s = oracle_mod.synthesize([a], [dx], [0.0], [1.0], (3 * dx, 5 * dx), (dx, dx), (2, 2), 0.0, 1.0, 1)
    assert np.allclose(s[0, :, :, 0], a[0, 5:7, 3:5], rtol=1e-14, atol=0)
    s = oracle_mod.synthesize([a], [dx], [0.0], [1.0], (-3 * dx, 20 * dx), (0, 0), (1, 1), 0.0, 1.0, 1)
    assert abs(s[0, 0, 0, 0] - a[0, n - 1, 0]) < 1e-14


def test_paper_absorbing_case_converges_in_table2_iterations(oracle_mod):
    # Table 2's absorbing (non-dispersive) run: the k-space potential
    # without its eta term; 133 (GPU) and 134 (CPU) iterations printed; the
    # readings of the homogeneous pin give the same 4-8% excess
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    k0 = 2 * np.pi * f / v
    eps = g["eps_factor"]["value"] * k0 * k0
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    S = np.zeros((n, n), complex)
    S[row - half:row + half + 1, g["source_column"]["value"]] = complex(*g["source_amplitude"]["value"])
    abl = oracle_mod.abl_profile(n, dx, g["abl_zeta_np_per_m"]["value"], g["abl_width_cells"]["value"])
    vv = oracle_mod.vv_kspace(n, dx, 2 * np.pi * f, g["alpha0"]["value"], g["nu"]["value"], v, eps,
                              dispersion=False)
    assert np.all(vv.real == 0.0)
    _, info, _ = oracle_mod.eps_solve_kspace(n, oracle_mod.ghat_eps(n, dx, k0, eps), vv, S, abl, 2000,
                                             g["stop_tol"]["value"], row=row)
    it = g["iterations_absorbing"]["value"]
    assert info["status"] == 0
    assert all(1.04 <= info["iters"] / v <= 1.08 for v in it.values()), (info, it)


def test_cbs_iteration_converges_where_the_plain_one_diverges(oracle_mod):
    # A strong absorbing random medium (max |U| ~ 3 k0^2): the paper's plain
    # iteration with eps = 0.8 k0^2 diverges, and with eps = max |U| it does
    # not converge in 5000 iterations; the convergent Born series
    # preconditioner (gamma = i V / eps, eps >= max |U|) converges to the
    # dense solution of the periodic Helmholtz problem (Fourier basis)
    n, dx = 32, 0.1
    k0 = 2 * np.pi / (8 * dx)
    rng = np.random.default_rng(9)
    base = 0.8 * k0 * k0
    for _ in range(3):  # skip three draws of the medium and source (the fourth set is used)
        rng.uniform(-1, 1, (n, n)), rng.random((n, n)), rng.standard_normal((n, n)), rng.standard_normal((n, n))
    U = base * (4.0 * rng.uniform(-1, 1, (n, n)) + 1j * 0.8 * rng.random((n, n)))
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    eps = 1.01 * np.abs(U).max()
    gh = oracle_mod.ghat_eps(n, dx, k0, eps)
    psi, info, _ = oracle_mod.eps_solve_cbs(n, gh, U - 1j * eps, S, None, eps, 5000, 1e-13)
    assert info["status"] == 0 and info["iters"] < 1000, info
    p = 2 * np.pi * np.fft.fftfreq(n, dx)
    F = np.fft.fft2(np.eye(n * n).reshape(n * n, n, n), axes=(1, 2)).reshape(n * n, n * n).T
    L = np.linalg.inv(F) @ np.diag((p[None, :] ** 2 + p[:, None] ** 2 - k0 ** 2).ravel()) @ F - np.diag(U.ravel())
    ref = np.linalg.solve(L, S.ravel()).reshape(n, n)
    assert rel(psi, ref) < 1e-10
    _, plain, _ = oracle_mod.eps_solve(n, oracle_mod.ghat_eps(n, dx, k0, base), U - 1j * base, S, None, 5000, 1e-13)
    assert plain["status"] != 0
    _, plain_eps, _ = oracle_mod.eps_solve(n, gh, U - 1j * eps, S, None, 5000, 1e-13)
    assert plain_eps["status"] != 0


def test_cbs_fixed_point_with_layer(oracle_mod):
    # with the absorbing layer the limit satisfies psi = A (psi + gamma
    # (G (V psi + S) - psi)) itself, checked by applying one step by hand
    n, dx = 32, 0.1
    k0 = 2 * np.pi / (8 * dx)
    rng = np.random.default_rng(10)
    U = 0.8 * k0 * k0 * (2.0 * rng.uniform(-1, 1, (n, n)) + 0.4j * rng.random((n, n)))
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    eps = 1.01 * np.abs(U).max()
    gh = oracle_mod.ghat_eps(n, dx, k0, eps)
    abl = oracle_mod.abl_profile(n, dx, 4.0 / (6 * dx), 6)
    psi, info, _ = oracle_mod.eps_solve_cbs(n, gh, U - 1j * eps, S, abl, eps, 5000, 1e-14)
    assert info["status"] == 0
    V = U - 1j * eps
    g = np.fft.ifft2(np.fft.fft2(V * psi + S) * gh * n * n)
    step = np.outer(abl, abl) * (psi + 1j * V / eps * (g - psi))
    assert rel(step, psi) < 1e-12


def test_eps_iteration_fixed_point_with_layer(oracle_mod):
    # with the absorbing layer the plain iteration's limit satisfies
    # psi = A . G (V psi + S) (Algorithm 1's update), checked by applying one
    # step by hand with numpy's FFT; A is the product of the two axes' Eq. 29
    # profiles, so a layer applied along one axis only fails here
    n, dx = 32, 0.1
    k0 = 2 * np.pi / (8 * dx)
    eps = 0.8 * k0 * k0
    rng = np.random.default_rng(13)
    U = eps * (0.2 * rng.standard_normal((n, n)) + 1j * (0.3 + 0.1 * rng.random((n, n))))
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    gh = oracle_mod.ghat_eps(n, dx, k0, eps)
    abl = oracle_mod.abl_profile(n, dx, 4.0 / (6 * dx), 6)
    psi, info, _ = oracle_mod.eps_solve(n, gh, U - 1j * eps, S, abl, 5000, 1e-14)
    assert info["status"] == 0
    g = np.fft.ifft2(np.fft.fft2((U - 1j * eps) * psi + S) * gh * n * n)
    assert rel(np.outer(abl, abl) * g, psi) < 1e-12
