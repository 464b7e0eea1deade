"""The paper's own discretisation on the GPU (TBS_FLAG_PERIODIC): periodic
grid, epsilon-shifted spectral Green's function formed in the column pass,
the sigmoid absorbing layer and the Eq. 30 row stop, against the oracle's
plain iteration (Section 3.1, Algorithm 1)."""
import json
import math
import os

import numpy as np
import pytest

from _helpers import PARITY_RTOL, library, rel_l2

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()


def _gpu_periodic(n, dx, f, c0, V_u, ix, iy, amp, width, zeta, tol, max_terms, row, eps_factor=0.8,
                  want_eps=False, **kw):
    import torch
    from paper_2507_13754_gb300 import tbs
    p = tbs.Plan(n, dx, f, c0, n_rhs=amp.shape[0], max_terms=max_terms, tol=tol, stop_mode=tbs.TBS_STOP_L1_ROW,
                 l1_row=row, periodic=True, eps_factor=eps_factor, abl_width=width, abl_zeta=zeta,
                 div_window=1 << 30, div_factor=math.inf, **kw)
    assert p.m == n
    p.set_potential(torch.from_numpy(V_u.astype(np.complex64)).cuda())
    p.set_sources(ix, iy, amp)
    psi, infos = p.solve()
    out = psi.cpu().numpy(), tbs.Plan.info_dicts(infos)
    if want_eps:
        out = out + (tbs.tbs_plan_eps(p.handle),)
    p.close()
    return out


@pytest.mark.parametrize("width", [0, 16])
def test_periodic_iteration_matches_oracle(width):
    """128^2 smooth random medium with absorption, four point sources, eps =
    0.8 k^2, optional layer, Eq. 30 on row 64 to 1e-5."""
    import oracle
    from paper_2507_13754_gb300 import workloads as W
    n = 128
    w = W.random_medium(n, seed=51, n_rhs=2)
    U = oracle.potential(w.f, w.c0, w.c.astype(np.float64), w.alpha.astype(np.float64), w.ypow, w.f_ref)
    k0 = 2 * math.pi * w.f / w.c0
    eps = 0.8 * k0 * k0
    zeta = 4.0 / (width * w.dx) if width else 0.0
    psi, info = _gpu_periodic(n, w.dx, w.f, w.c0, U, w.src_ix, w.src_iy, w.src_amp, width, zeta, 1e-5, 1000, n // 2)
    gh = oracle.ghat_eps(n, w.dx, k0, eps)
    abl = oracle.abl_profile(n, w.dx, zeta, width) if width else None
    for r in range(2):
        S = oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, w.src_amp[r].astype(np.complex128))
        ref, rinfo, _ = oracle.eps_solve(n, gh, U - 1j * eps, S, abl, 1000, 1e-5, row=n // 2)
        assert rinfo["status"] == 0 and info[r]["status_name"] == "CONVERGED"
        iters = info[r]["terms"] - 1  # psi^0 .. psi^{terms-1}
        if iters != rinfo["iters"]:  # the stop decision sat on the threshold on one side
            assert abs(iters - rinfo["iters"]) == 1
            ref, _, _ = oracle.eps_solve(n, gh, U - 1j * eps, S, abl, iters, 0.0, row=n // 2)
        assert rel_l2(psi[r], ref) < PARITY_RTOL, (r, rel_l2(psi[r], ref))


def test_periodic_plan_rejects_what_it_cannot_do():
    from paper_2507_13754_gb300 import tbs
    with pytest.raises(tbs.TbsError):
        tbs.Plan(100, 1e-4, 1e6, 1500.0, periodic=True)  # not a power of two
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, periodic=True, keep_terms=True)
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, periodic=True, abl_width=8)  # zeta missing
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, kspace_alpha0=1e-9)  # the k-space potential needs the periodic grid
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, periodic=True, kspace_alpha0=1e-9, kspace_nu=3.0)
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, cbs=True)  # the preconditioner needs the periodic grid
    with pytest.raises(tbs.TbsError):
        tbs.Plan(128, 1e-4, 1e6, 1500.0, periodic=True, cbs=True, kspace_alpha0=1e-9)
    p = tbs.Plan(64, 1e-4, 1e6, 1500.0, periodic=True)
    with pytest.raises(tbs.TbsError):
        p.ghat_quadrant()
    p.close()


@pytest.mark.parametrize("width,dispersion", [(0, True), (16, True), (16, False)])
def test_kspace_potential_matches_oracle(width, dispersion):
    """Case II of Algorithm 1 (Eq. 24's power-law absorption and dispersion as
    the k-space potential VV, Section 3.1): 128^2 homogeneous water at 1 MHz,
    alpha0 = 2e-8 (36x the paper's, so that VV moves the field well above
    the tolerance), nu = 1.5, two right-hand sides, optional layer, Eq. 30
    on row 64 to 1e-5; dispersion=False drops the eta term (Table 2's
    absorbing case)."""
    import oracle
    n, f, c0, a0, nu = 128, 1e6, 1500.0, 2e-8, 1.5
    dx = c0 / f / 8.0
    k0 = 2 * math.pi * f / c0
    eps = 0.8 * k0 * k0
    zeta = 4.0 / (width * dx) if width else 0.0
    ix = np.array([20, 90], np.int32)
    iy = np.array([64, 30], np.int32)
    amp = np.array([[1.0 + 0.5j, -0.3j], [0.2, 1.0]], np.complex64)
    psi, info = _gpu_periodic(n, dx, f, c0, np.zeros((n, n)), ix, iy, amp, width, zeta, 1e-5, 1000, n // 2,
                              kspace_alpha0=a0, kspace_nu=nu, kspace_dispersion=dispersion)
    gh = oracle.ghat_eps(n, dx, k0, eps)
    vv = oracle.vv_kspace(n, dx, 2 * math.pi * f, a0, nu, c0, eps, dispersion=dispersion)
    abl = oracle.abl_profile(n, dx, zeta, width) if width else None
    for r in range(2):
        S = oracle.deposit_points(n, dx, ix, iy, amp[r].astype(np.complex128))
        ref, rinfo, _ = oracle.eps_solve_kspace(n, gh, vv, S, abl, 1000, 1e-5, row=n // 2)
        assert rinfo["status"] == 0 and info[r]["status_name"] == "CONVERGED"
        iters = info[r]["terms"] - 1
        if iters != rinfo["iters"]:
            assert abs(iters - rinfo["iters"]) == 1
            ref, _, _ = oracle.eps_solve_kspace(n, gh, vv, S, abl, iters, 0.0, row=n // 2)
        # VV must matter at this tolerance: the same run without it differs
        plain, _, _ = oracle.eps_solve(n, gh, np.full((n, n), -1j * eps), S, abl, iters, 0.0, row=n // 2)
        assert rel_l2(plain, ref) > 100 * PARITY_RTOL
        assert rel_l2(psi[r], ref) < PARITY_RTOL, (r, rel_l2(psi[r], ref))


@pytest.mark.slow
def test_paper_homogeneous_4096_matches_oracle():
    """Section 3.1's run: 4096^2, f = 1.00708 MHz, 501 sources of -1e6 i on
    column 675 around row 2049 (1-based), layer of 450 cells with zeta =
    21.48 Np/cm, Eq. 30 on row 2049 to 1e-5.  The oracle needs 143
    iterations (Table 2 prints 135 GPU / 133 CPU); the GPU must stop at
    the same count (or one off) and match the oracle's field on the row."""
    import oracle
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    k0 = 2 * math.pi * f / v
    eps = g["eps_factor"]["value"] * k0 * k0
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    col = g["source_column"]["value"]
    amp = complex(*g["source_amplitude"]["value"])
    width, zeta = g["abl_width_cells"]["value"], g["abl_zeta_np_per_m"]["value"]
    iy = np.arange(row - half, row + half + 1, dtype=np.int32)
    ix = np.full_like(iy, col)
    a = np.full((1, iy.size), amp * dx * dx, np.complex64)  # the plan deposits a / dx^2 per cell
    psi, info = _gpu_periodic(n, dx, f, v, np.zeros((n, n)), ix, iy, a, width, zeta, g["stop_tol"]["value"],
                              2000, row)
    S = np.zeros((n, n), complex)
    S[row - half:row + half + 1, col] = amp
    abl = oracle.abl_profile(n, dx, zeta, width)
    gh = oracle.ghat_eps(n, dx, k0, eps)
    ref, rinfo, _ = oracle.eps_solve(n, gh, np.full((n, n), -1j * eps), S, abl, 2000, g["stop_tol"]["value"], row=row)
    iters = info[0]["terms"] - 1
    assert info[0]["status_name"] == "CONVERGED" and abs(iters - rinfo["iters"]) <= 1, (iters, rinfo)
    if iters != rinfo["iters"]:
        ref, _, _ = oracle.eps_solve(n, gh, np.full((n, n), -1j * eps), S, abl, iters, 0.0, row=row)
    assert rel_l2(psi[0][row], ref[row]) < PARITY_RTOL
    assert rel_l2(psi[0], ref) < PARITY_RTOL


@pytest.mark.slow
@pytest.mark.parametrize("dispersion", [True, False])
def test_paper_absorbing_4096_matches_oracle(dispersion):
    """Section 3.1's absorbing runs: the homogeneous 4096^2 case with the
    k-space potential of alpha0 = 5.5e-10, nu = 1.5, with the dispersive
    term (Table 2 'absorbing-dispersive': 132 GPU / 131 CPU iterations) and
    without it ('absorbing': 133 / 134).  The GPU stops where the oracle
    does (or one off) and matches its field."""
    import oracle
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    n, dx, v, f = g["grid_n"]["value"], g["dx_m"]["value"], g["v_f"]["value"], g["f_hz"]["value"]
    a0, nu = g["alpha0"]["value"], g["nu"]["value"]
    k0 = 2 * math.pi * f / v
    eps = g["eps_factor"]["value"] * k0 * k0
    row = g["source_row_1based"]["value"] - 1
    half = (g["n_elements"]["value"] - 1) // 2
    col = g["source_column"]["value"]
    amp = complex(*g["source_amplitude"]["value"])
    width, zeta = g["abl_width_cells"]["value"], g["abl_zeta_np_per_m"]["value"]
    tol = g["stop_tol"]["value"]
    iy = np.arange(row - half, row + half + 1, dtype=np.int32)
    ix = np.full_like(iy, col)
    a = np.full((1, iy.size), amp * dx * dx, np.complex64)
    psi, info = _gpu_periodic(n, dx, f, v, np.zeros((n, n)), ix, iy, a, width, zeta, tol, 2000, row,
                              kspace_alpha0=a0, kspace_nu=nu, kspace_dispersion=dispersion)
    S = np.zeros((n, n), complex)
    S[row - half:row + half + 1, col] = amp
    abl = oracle.abl_profile(n, dx, zeta, width)
    gh = oracle.ghat_eps(n, dx, k0, eps)
    vv = oracle.vv_kspace(n, dx, 2 * math.pi * f, a0, nu, v, eps, dispersion=dispersion)
    ref, rinfo, _ = oracle.eps_solve_kspace(n, gh, vv, S, abl, 2000, tol, row=row)
    iters = info[0]["terms"] - 1
    assert info[0]["status_name"] == "CONVERGED" and abs(iters - rinfo["iters"]) <= 1, (iters, rinfo)
    if iters != rinfo["iters"]:
        ref, _, _ = oracle.eps_solve_kspace(n, gh, vv, S, abl, iters, 0.0, row=row)
    assert rel_l2(psi[0], ref) < PARITY_RTOL


@pytest.mark.slow
def test_paper_inhomogeneous_4096_matches_oracle():
    """Section 3.1's inhomogeneous run: the homogeneous geometry plus a
    cylinder of radius 50 dx = 1 mm at 1350 m/s (water 1500 m/s), centred
    40.2 mm from the array along its axis, as a spatial potential on the
    periodic plan.  The GPU stops where the oracle does (or one off) and
    matches its field."""
    import torch
    import oracle
    from paper_2507_13754_gb300 import tbs, workloads as W
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    case = W.paper_periodic_case(g, scatterer_speed=1350.0)
    p = tbs.Plan(case.n, case.dx, case.f, case.c0, max_terms=2000, tol=case.tol, stop_mode=tbs.TBS_STOP_L1_ROW,
                 l1_row=case.l1_row, periodic=True, eps_factor=case.eps_factor, abl_width=case.abl_width,
                 abl_zeta=case.abl_zeta, div_window=1 << 30, div_factor=math.inf)
    p.set_medium(torch.from_numpy(case.c).cuda(), None, 1.0, case.f)
    p.set_sources(case.ix, case.iy, case.amp)
    psi, infos = p.solve()
    psi = psi.cpu().numpy()
    info = tbs.Plan.info_dicts(infos)[0]
    p.close()
    n = case.n
    k0 = 2 * math.pi * case.f / case.c0
    eps = case.eps_factor * k0 * k0
    U = oracle.potential(case.f, case.c0, case.c.astype(np.float64), None, 1.0, case.f)
    S = oracle.deposit_points(n, case.dx, case.ix, case.iy, case.amp[0].astype(np.complex128))
    abl = oracle.abl_profile(n, case.dx, case.abl_zeta, case.abl_width)
    gh = oracle.ghat_eps(n, case.dx, k0, eps)
    ref, rinfo, _ = oracle.eps_solve(n, gh, U - 1j * eps, S, abl, 2000, case.tol, row=case.l1_row)
    iters = info["terms"] - 1
    assert info["status_name"] == "CONVERGED" and abs(iters - rinfo["iters"]) <= 1, (iters, rinfo)
    if iters != rinfo["iters"]:
        ref, _, _ = oracle.eps_solve(n, gh, U - 1j * eps, S, abl, iters, 0.0, row=case.l1_row)
    assert rel_l2(psi[0], ref) < PARITY_RTOL


def _paper_case_plan(case, max_terms, tol, **kw):
    import torch
    from paper_2507_13754_gb300 import tbs
    p = tbs.Plan(case.n, case.dx, case.f, case.c0, max_terms=max_terms, tol=tol, stop_mode=tbs.TBS_STOP_L1_ROW,
                 l1_row=case.l1_row, periodic=True, eps_factor=case.eps_factor, abl_width=case.abl_width,
                 abl_zeta=case.abl_zeta, div_window=1 << 30, div_factor=math.inf, **kw)
    p.set_medium(torch.from_numpy(case.c).cuda(), None, 1.0, case.f)
    p.set_sources(case.ix, case.iy, case.amp)
    return p


@pytest.mark.parametrize("which", ["v_s_high", "nu_max"])
def test_paper_convergence_ranges(which):
    """Table 3's convergence test at its range edges, on the paper's 4096^2
    geometry: the cylinder at 3750 m/s, and the k-space potential at nu =
    1.7 (alpha0 = 5.5e-10).  The series converges (Eq. 30 < 1e-5) within
    2000 iterations and the field is finite."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    v_s = g["convergence_v_s_range"]["value"][1] if which == "v_s_high" else None
    kw = {}
    if which == "nu_max":
        kw = dict(kspace_alpha0=g["alpha0"]["value"], kspace_nu=g["convergence_nu_max"]["value"])
    p = _paper_case_plan(W.paper_periodic_case(g, scatterer_speed=v_s), 2000, g["stop_tol"]["value"], **kw)
    psi, infos = p.solve()
    info = tbs.Plan.info_dicts(infos)[0]
    p.close()
    assert info["status_name"] == "CONVERGED", (which, info)
    assert bool(torch.isfinite(torch.view_as_real(psi)).all())


@pytest.mark.slow
def test_paper_low_speed_cylinder_follows_oracle():
    """Table 3's lower edge, the cylinder at 1100 m/s.  The iteration has an
    unstable mode there: in FP64 the Eq. 30 error falls to 9.6e-6 at
    iteration 189 and then grows about 9% per iteration (0.92 by 400), so
    the oracle meets the tolerance only because its rounding seeds that mode
    at 1e-16; FP32 seeds it at 1e-7 and the GPU run never meets 1e-5.  What
    holds at any precision is checked: the GPU field follows the oracle's
    over the first 30 iterations."""
    import oracle
    from paper_2507_13754_gb300 import tbs, workloads as W
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    case = W.paper_periodic_case(g, scatterer_speed=g["convergence_v_s_range"]["value"][0])
    K = 30
    p = _paper_case_plan(case, K + 1, 0.0)
    psi, infos = p.solve()
    psi = psi.cpu().numpy()
    assert tbs.Plan.info_dicts(infos)[0]["terms"] == K + 1
    p.close()
    n = case.n
    k0 = 2 * math.pi * case.f / case.c0
    eps = case.eps_factor * k0 * k0
    U = oracle.potential(case.f, case.c0, case.c.astype(np.float64), None, 1.0, case.f)
    S = oracle.deposit_points(n, case.dx, case.ix, case.iy, case.amp[0].astype(np.complex128))
    abl = oracle.abl_profile(n, case.dx, case.abl_zeta, case.abl_width)
    ref, _, _ = oracle.eps_solve(n, oracle.ghat_eps(n, case.dx, k0, eps), U - 1j * eps, S, abl, K, 0.0,
                                 row=case.l1_row)
    assert rel_l2(psi[0], ref) < PARITY_RTOL


@pytest.mark.parametrize("width", [0, 16])
def test_cbs_matches_oracle_on_a_strong_medium(width):
    """The convergent Born series preconditioner (TBS_FLAG_CBS) on a strong
    absorbing random potential (max |U| ~ 3.3 k0^2; the plain iteration with
    eps = 0.8 k0^2 ends NONFINITE in the oracle), 128^2, eps chosen by the
    library from the potential (eps_factor = 0: eps = 1.01 max |U|), two
    right-hand sides, optional layer, Eq. 30 on row 64 to 1e-5."""
    import oracle
    n, f, c0 = 128, 1e6, 1500.0
    dx = c0 / f / 8.0
    k0 = 2 * math.pi * f / c0
    rng = np.random.default_rng(12)
    U = 0.8 * k0 * k0 * (4.0 * rng.uniform(-1, 1, (n, n)) + 0.8j * rng.random((n, n)))
    zeta = 4.0 / (width * dx) if width else 0.0
    ix = np.array([30, 100], np.int32)
    iy = np.array([64, 20], np.int32)
    amp = np.array([[1.0, 0.5j], [-0.3, 1.0]], np.complex64)
    psi, info, eps = _gpu_periodic(n, dx, f, c0, U, ix, iy, amp, width, zeta, 1e-5, 3000, n // 2,
                                   eps_factor=0.0, want_eps=True, cbs=True)
    # the library's choice: 1.01 max |U| of the complex64 potential it was given
    U = U.astype(np.complex64).astype(np.complex128)
    assert abs(eps / (1.01 * np.abs(U).max()) - 1) < 1e-12
    gh = oracle.ghat_eps(n, dx, k0, eps)
    abl = oracle.abl_profile(n, dx, zeta, width) if width else None
    for r in range(2):
        S = oracle.deposit_points(n, dx, ix, iy, amp[r].astype(np.complex128))
        ref, rinfo, _ = oracle.eps_solve_cbs(n, gh, U - 1j * eps, S, abl, eps, 3000, 1e-5, row=n // 2)
        assert rinfo["status"] == 0 and info[r]["status_name"] == "CONVERGED", (rinfo, info[r])
        iters = info[r]["terms"] - 1
        if iters != rinfo["iters"]:
            assert abs(iters - rinfo["iters"]) == 1
            ref, _, _ = oracle.eps_solve_cbs(n, gh, U - 1j * eps, S, abl, eps, iters, 0.0, row=n // 2)
        assert rel_l2(psi[r], ref) < PARITY_RTOL, (r, rel_l2(psi[r], ref))


@pytest.mark.slow
def test_cbs_converges_on_the_low_speed_cylinder():
    """Table 3's 1100 m/s cylinder, where the plain iteration has an unstable
    mode: with the convergent Born series preconditioner (eps = 1.01 max |U|)
    the FP32 GPU run meets Eq. 30 < 1e-5 and matches the oracle's
    preconditioned iteration."""
    import oracle
    from paper_2507_13754_gb300 import tbs, workloads as W
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    case = W.paper_periodic_case(g, scatterer_speed=g["convergence_v_s_range"]["value"][0])
    case.eps_factor = 0.0  # the library chooses eps = 1.01 max |U| from the medium
    p = _paper_case_plan(case, 2000, case.tol, cbs=True)
    eps = tbs.tbs_plan_eps(p.handle)
    psi, infos = p.solve()
    psi = psi.cpu().numpy()
    info = tbs.Plan.info_dicts(infos)[0]
    p.close()
    n = case.n
    k0 = 2 * math.pi * case.f / case.c0
    U = oracle.potential(case.f, case.c0, case.c.astype(np.float64), None, 1.0, case.f)
    assert abs(eps / (1.01 * np.abs(U).max()) - 1) < 1e-6  # FP32 V against the FP64 potential
    S = oracle.deposit_points(n, case.dx, case.ix, case.iy, case.amp[0].astype(np.complex128))
    abl = oracle.abl_profile(n, case.dx, case.abl_zeta, case.abl_width)
    gh = oracle.ghat_eps(n, case.dx, k0, eps)
    ref, rinfo, _ = oracle.eps_solve_cbs(n, gh, U - 1j * eps, S, abl, eps, 2000, case.tol, row=case.l1_row)
    iters = info["terms"] - 1
    assert info["status_name"] == "CONVERGED" and abs(iters - rinfo["iters"]) <= 1, (iters, rinfo)
    if iters != rinfo["iters"]:
        ref, _, _ = oracle.eps_solve_cbs(n, gh, U - 1j * eps, S, abl, eps, iters, 0.0, row=case.l1_row)
    assert rel_l2(psi[0], ref) < PARITY_RTOL


@pytest.mark.parametrize("weak", [1.0, 1e-6])
def test_periodic_harmonics_match_oracle(weak):
    """The paper's nonlinear chain on the periodic grid (Section 3.1: each
    harmonic n with eps_n = 0.8 n^2 k^2 and the sum-term source), homogeneous
    water, 128^2, a 16-cell layer, harmonics 1 .. 3, Eq. 30 to 1e-5.  With
    the source 1e-6 times weaker psi_3 peaks near 1e-41, below FP32's normal
    range: the chain's per-harmonic scaling must carry it."""
    import torch
    import oracle
    from paper_2507_13754_gb300.solvers import harmonics
    n, f, c0 = 128, 1e6, 1500.0
    dx = c0 / f / 8.0
    width, zeta = 16, 4.0 / (16 * dx)
    ix = np.array([20], np.int32)
    iy = np.array([64], np.int32)
    amp = np.full((1, 1), -1e6j * dx * dx * weak, np.complex64)
    ones = np.ones((n, n), np.float32)
    bd, rd = (torch.from_numpy(x).cuda() for x in (3.5 * ones, 1000.0 * ones))
    fields, infos = harmonics(3, n, dx, f, c0, None, None, 1.0, bd, rd, ix, iy, amp, max_terms=2000, tol=1e-5,
                              periodic=True, abl_width=width, abl_zeta=zeta, stop_mode=1, l1_row=64,
                              div_window=1 << 30, div_factor=math.inf)
    abl = oracle.abl_profile(n, dx, zeta, width)
    refs = []
    for order in range(1, 4):
        k = 2 * math.pi * order * f / c0
        eps = 0.8 * k * k
        gh = oracle.ghat_eps(n, dx, k, eps)
        if order == 1:
            S = oracle.deposit_points(n, dx, ix, iy, amp[0].astype(np.complex128))
        else:
            S = oracle.harmonic_source(order, 2 * math.pi * f, 3.5 * ones, 1000.0 * ones, c0 * ones, refs)
        iters = infos[order - 1][0]["terms"] - 1
        assert infos[order - 1][0]["status_name"] == "CONVERGED"
        ref, rinfo, _ = oracle.eps_solve(n, gh, np.full((n, n), -1j * eps), S, abl, 2000, 1e-5, row=64)
        assert abs(iters - rinfo["iters"]) <= 1, (order, iters, rinfo)
        if iters != rinfo["iters"]:
            ref, _, _ = oracle.eps_solve(n, gh, np.full((n, n), -1j * eps), S, abl, iters, 0.0, row=64)
        refs.append(ref)
        e = infos[order - 1][0]["log2_scale"]
        got = fields[order - 1][0].cpu().numpy().astype(np.complex128) * 2.0 ** e
        assert rel_l2(got, ref) < PARITY_RTOL, order
        assert 1e-12 < np.abs(fields[order - 1][0].cpu().numpy()).max() < 1e12, (order, e)
