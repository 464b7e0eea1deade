"""Adjoint (gradient with respect to c and alpha) and second harmonic on the
GPU against the oracle, plus a finite-difference check of the autograd path."""
import math

import numpy as np
import pytest

from _helpers import PARITY_RTOL, library, rel_l2

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-4  # gradient: FP32 terms and products, summed over terms and RHS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()


def _gpu_forward(w, keep_terms=True, max_terms=None, tol=None):
    import torch
    from paper_2507_13754_gb300 import tbs
    plan = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs,
                    max_terms=w.max_terms if max_terms is None else max_terms,
                    tol=w.tol if tol is None else tol, keep_terms=keep_terms)
    c = torch.from_numpy(w.c).cuda()
    al = torch.from_numpy(w.alpha).cuda() if w.alpha is not None else None
    plan.set_medium(c, al, w.ypow, w.f_ref)
    plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
    psi, infos = plan.solve()
    return plan, psi, tbs.Plan.info_dicts(infos)


def _oracle_gradient(w, terms, g):
    import oracle
    m, gh = oracle.plan(w.n, w.dx, w.f, w.c0)
    c = w.c.astype(np.float64)
    al = None if w.alpha is None else w.alpha.astype(np.float64)
    V = oracle.potential(w.f, w.c0, c, al, w.ypow, w.f_ref)
    Q = np.zeros((w.n, w.n), complex)
    for r in range(w.n_rhs):
        s = oracle.deposit_points(w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[r].astype(np.complex128))
        _, _, _, u = oracle.solve(w.n, m, gh, V, s, terms[r], 0.0, keep_terms=True)
        Q += oracle.adjoint(w.n, m, gh, V, u, g[r].astype(np.complex128))
    dc, da = oracle.potential_derivs(w.f, c, al, w.ypow, w.f_ref)
    return np.real(Q * dc), np.real(Q * da)


@pytest.mark.parametrize("n,n_rhs,seed", [(48, 3, 31), (130, 2, 32)])
def test_adjoint_matches_oracle_adjoint(n, n_rhs, seed):
    import torch
    from paper_2507_13754_gb300 import workloads as W
    w = W.random_medium(n, seed=seed, n_rhs=n_rhs)
    w.f_ref = 0.6 * w.f  # dispersion on: exercises tan(pi y / 2) delta in dV/dalpha
    plan, psi, info = _gpu_forward(w)
    terms = [i["terms"] for i in info]
    rng = np.random.default_rng(seed + 100)
    g = (rng.standard_normal((n_rhs, n, n)) + 1j * rng.standard_normal((n_rhs, n, n))).astype(np.complex64)
    gc = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ga = torch.empty((n, n), dtype=torch.float32, device="cuda")
    plan.solve_adjoint(torch.from_numpy(g).cuda(), gc, ga)
    torch.cuda.synchronize()
    rc, ra = _oracle_gradient(w, terms, g)
    assert rel_l2(gc.cpu().numpy(), rc) < GRAD_RTOL
    assert rel_l2(ga.cpu().numpy(), ra) < GRAD_RTOL
    plan.close()


def test_adjoint_graph_loop_and_stream_agree():
    """RHS with different term counts (one zero source stops after a single
    term): the graph's device-counted reverse loop gives bitwise the
    stream-unrolled sweep, and both match the oracle."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    n = 96
    w = W.random_medium(n, seed=34, n_rhs=3)
    w.src_amp[1] = 0
    rng = np.random.default_rng(134)
    g = (rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n))).astype(np.complex64)
    out = []
    for use_graph in (True, False):
        plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=3, max_terms=w.max_terms, tol=w.tol, keep_terms=True,
                        use_graph=use_graph)
        al = torch.from_numpy(w.alpha).cuda() if w.alpha is not None else None
        plan.set_medium(torch.from_numpy(w.c).cuda(), al, w.ypow, w.f_ref)
        plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
        _, infos = plan.solve()
        terms = [i["terms"] for i in tbs.Plan.info_dicts(infos)]
        gc = torch.empty((n, n), dtype=torch.float32, device="cuda")
        ga = torch.empty((n, n), dtype=torch.float32, device="cuda")
        for _ in range(2):  # the second call replays the cached graph
            plan.solve_adjoint(torch.from_numpy(g).cuda(), gc, ga)
        torch.cuda.synchronize()
        out.append((terms, gc.cpu().numpy(), ga.cpu().numpy()))
        plan.close()
    (t0, c0, a0), (t1, c1, a1) = out
    assert t0 == t1 and t0[1] == 1 and t0[0] > 2
    assert np.array_equal(c0, c1) and np.array_equal(a0, a1)
    rc, ra = _oracle_gradient(w, t0, g)
    assert rel_l2(c0, rc) < GRAD_RTOL
    assert rel_l2(a0, ra) < GRAD_RTOL


@pytest.mark.parametrize("n,max_terms", [(96, 64), (75, 40)])
def test_checkpointed_adjoint_is_bitwise_the_stored_one(n, max_terms):
    """TBS_FLAG_CHECKPOINT_TERMS keeps every K-th term (K = ceil(sqrt(max_terms)))
    and recomputes the rest segment by segment: the recomputation runs the
    forward arithmetic on the same values, so the gradient is bitwise that of
    the stored-terms adjoint, for RHS with different term counts."""
    import math
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(n, seed=36, n_rhs=3)
    w.src_amp[1] *= 0.5
    w.src_amp[2] = 0
    rng = np.random.default_rng(136)
    g = torch.from_numpy((rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n))).astype(np.complex64)).cuda()
    out = []
    for ck in (False, True):
        # tol 1e-12: ~20 terms, so the sweep crosses several segments
        plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=3, max_terms=max_terms, tol=1e-12, keep_terms=True, checkpoint=ck)
        al = torch.from_numpy(w.alpha).cuda() if w.alpha is not None else None
        plan.set_medium(torch.from_numpy(w.c).cuda(), al, w.ypow, w.f_ref)
        plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
        psi, infos = plan.solve()
        gc = torch.empty((n, n), dtype=torch.float32, device="cuda")
        ga = torch.empty((n, n), dtype=torch.float32, device="cuda")
        plan.solve_adjoint(g, gc, ga)
        torch.cuda.synchronize()
        out.append(([i["terms"] for i in tbs.Plan.info_dicts(infos)], psi.cpu().numpy(), gc.cpu().numpy(),
                    ga.cpu().numpy(), tbs.tbs_plan_device_bytes(plan.desc)))
        plan.close()
    (t0, p0, c0, a0, b0), (t1, p1, c1, a1, b1) = out
    k = math.ceil(math.sqrt(max_terms))
    assert t0 == t1 and t0[2] == 1 and max(t0) > 2 * k  # several segments
    assert np.array_equal(p0, p1)
    assert np.array_equal(c0, c1) and np.array_equal(a0, a1)
    assert b1 < b0  # fewer stored fields


def test_adjoint_of_single_term_series_is_zero():
    """T = 1 for every RHS: psi = G S does not depend on the medium, the
    reverse loop runs no step and the gradient is exactly zero."""
    import torch
    from paper_2507_13754_gb300 import workloads as W
    w = W.random_medium(40, seed=35, n_rhs=2)
    plan, psi, info = _gpu_forward(w, max_terms=1, tol=0.0)
    assert [i["terms"] for i in info] == [1, 1]
    g = torch.ones((2, 40, 40), dtype=torch.complex64, device="cuda")
    gc = torch.full((40, 40), 7.0, dtype=torch.float32, device="cuda")
    ga = torch.full((40, 40), 7.0, dtype=torch.float32, device="cuda")
    plan.solve_adjoint(g, gc, ga)
    torch.cuda.synchronize()
    assert torch.count_nonzero(gc).item() == 0 and torch.count_nonzero(ga).item() == 0
    plan.close()


def test_adjoint_without_kept_terms_is_a_state_error():
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(32, seed=33)
    plan, psi, info = _gpu_forward(w, keep_terms=False)
    g = torch.zeros((1, 32, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(tbs.TbsError) as ei:
        plan.solve_adjoint(g, None, None)
    assert ei.value.code == 5  # TBS_ERR_STATE
    plan.close()


def test_autograd_gradient_matches_directional_finite_differences():
    """J = 1/2 sum_s |P psi_s - d_s|^2 (receivers on one row), fixed 10 terms."""
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    from paper_2507_13754_gb300.solvers import TBSField
    n, T = 96, 10
    w = W.cfg5(n=n, n_src=3, terms=T, true_model=True)
    row = w.extras["receiver_row"]
    plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=T, tol=0.0, keep_terms=True)
    rng = np.random.default_rng(34)
    d = torch.from_numpy((rng.standard_normal((w.n_rhs, n)) + 1j * rng.standard_normal((w.n_rhs, n)))
                         .astype(np.complex64) * 0.05).cuda()
    c0 = torch.from_numpy(w.c).cuda()
    a0 = torch.from_numpy(w.alpha).cuda()

    def J(c, a):
        psi = TBSField.apply(c, a, plan, w.src_ix, w.src_iy, w.src_amp, w.ypow, w.f_ref)
        r = psi[:, row, :].to(torch.complex128) - d.to(torch.complex128)
        return 0.5 * (r.abs() ** 2).sum()

    c = c0.clone().requires_grad_(True)
    a = a0.clone().requires_grad_(True)
    L = J(c, a)
    L.backward()
    yy, xx = np.mgrid[0:n, 0:n]
    phi = torch.from_numpy(np.exp(-((yy - 0.45 * n) ** 2 + (xx - 0.5 * n) ** 2) / (2 * (0.12 * n) ** 2))
                           .astype(np.float32)).cuda()
    with torch.no_grad():
        hc = 1e-4 * 1540.0
        fd_c = (J(c0 + hc * phi, a0) - J(c0 - hc * phi, a0)).item() / (2 * hc)
        # alpha moves J far less than c does: a 1% step keeps the difference
        # well above the complex64 field's rounding noise, and the central
        # difference's O(h^2) error stays near 1e-5 of the derivative
        ha = 1e-2 * float(a0.mean())
        fd_a = (J(c0, a0 + ha * phi) - J(c0, a0 - ha * phi)).item() / (2 * ha)
    ad_c = float((c.grad.double() * phi.double()).sum())
    ad_a = float((a.grad.double() * phi.double()).sum())
    assert abs(ad_c - fd_c) < 1e-3 * abs(fd_c), (ad_c, fd_c)
    assert abs(ad_a - fd_a) < 1e-3 * abs(fd_a), (ad_a, fd_a)
    plan.close()


@pytest.mark.parametrize("n", [256, pytest.param(2048, marks=pytest.mark.slow)])
def test_second_harmonic_matches_oracle(n):
    import torch
    import oracle
    from paper_2507_13754_gb300 import workloads as W
    from paper_2507_13754_gb300.solvers import second_harmonic
    w = W.cfg3(n=n)
    amp = (w.src_amp * 2e5).astype(np.complex64)  # O(0.5 MPa) fields: S2 ~ psi1^2 is then O(1)
    cd = torch.from_numpy(w.c).cuda()
    ad = torch.from_numpy(w.alpha).cuda()
    bd = torch.from_numpy(w.extras["beta"]).cuda()
    rd = torch.from_numpy(w.extras["rho"]).cuda()
    # the 4 MHz series contracts by ~0.86 per term at 2048^2 (the fat ellipse is
    # twice as strong in phase at 2 k0): it reaches 1e-6 in ~95 terms
    psi1, i1, psi2, i2 = second_harmonic(n, w.dx, w.f, w.c0, cd, ad, w.ypow, bd, rd, w.src_ix, w.src_iy,
                                         amp, max_terms=64, tol=1e-6, max_terms_harmonic=128)
    psi1, psi2 = psi1.cpu().numpy()[0], psi2.cpu().numpy()[0]
    # oracle chain at the GPU's term counts
    c = w.c.astype(np.float64)
    m, gh1 = oracle.plan(n, w.dx, w.f, w.c0)
    V1 = oracle.potential(w.f, w.c0, c, w.alpha.astype(np.float64), w.ypow, w.f)
    s1 = oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, amp[0].astype(np.complex128))
    r1, _, _, _ = oracle.solve(n, m, gh1, V1, s1, i1[0]["terms"], 0.0)
    assert rel_l2(psi1, r1) < PARITY_RTOL
    s2 = oracle.harmonic2_source(2 * math.pi * w.f, w.extras["beta"].astype(np.float64),
                                 w.extras["rho"].astype(np.float64), c, r1)
    _, gh2 = oracle.plan(n, w.dx, 2 * w.f, w.c0)
    V2 = oracle.potential(2 * w.f, w.c0, c, w.alpha.astype(np.float64) * 2 ** w.ypow, w.ypow, 2 * w.f)
    r2, _, _, _ = oracle.solve(n, m, gh2, V2, s2, i2[0]["terms"], 0.0)
    assert i1[0]["status_name"] == "CONVERGED" and i2[0]["status_name"] == "CONVERGED", (i1, i2)
    assert rel_l2(psi2, r2) < PARITY_RTOL


def test_cfg5_gradient_matches_central_differences_on_50_pixels():
    """The gradient workload at 1/8 scale (128^2, 3 MHz, four of the 16
    sources, receivers on row 125): the GPU adjoint gradient of
    J = 1/2 sum_s sum_row |psi_s - d_s|^2 at the homogeneous start model,
    against FP64 central differences (h = 1e-3 relative) of the same J through
    the oracle at 50 seeded random pixels, each series truncated at the
    forward solve's term count."""
    import oracle
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    n, srcs = 128, [0, 5, 10, 15]
    w = W.cfg5(n=n)
    wt = W.cfg5(n=n, true_model=True)
    row = w.extras["receiver_row"]
    m, gh = oracle.plan(n, w.dx, w.f, w.c0)
    S = [oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, w.src_amp[k].astype(np.complex128)) for k in srcs]
    Vt = oracle.potential(w.f, w.c0, wt.c.astype(np.float64), wt.alpha.astype(np.float64), w.ypow, w.f_ref)
    data = [oracle.solve(n, m, gh, Vt, s, 64, 1e-6)[0][row] for s in S]
    # GPU forward + adjoint at the start model
    plan = tbs.Plan(n, w.dx, w.f, w.c0, n_rhs=len(srcs), max_terms=64, tol=1e-6, keep_terms=True)
    plan.set_medium(torch.from_numpy(w.c).cuda(), torch.from_numpy(w.alpha).cuda(), w.ypow, w.f_ref)
    plan.set_sources(w.src_ix, w.src_iy, w.src_amp[srcs])
    psi, infos = plan.solve()
    terms = [i["terms"] for i in tbs.Plan.info_dicts(infos)]
    g = torch.zeros((len(srcs), n, n), dtype=torch.complex64, device="cuda")
    for r, d in enumerate(data):
        g[r, row] = torch.from_numpy((psi[r, row].cpu().numpy() - d).astype(np.complex64)).cuda()
    gc = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ga = torch.empty((n, n), dtype=torch.float32, device="cuda")
    plan.solve_adjoint(g, gc, ga)
    torch.cuda.synchronize()
    gc, ga = gc.cpu().numpy(), ga.cpu().numpy()
    plan.close()

    def J(c, al):
        V = oracle.potential(w.f, w.c0, c, al, w.ypow, w.f_ref)
        return sum(0.5 * np.sum(np.abs(oracle.solve(n, m, gh, V, s, T, 0.0)[0][row] - d) ** 2)
                   for s, d, T in zip(S, data, terms))

    rng = np.random.default_rng(5)
    pix = rng.choice(n * n, 50, replace=False)
    c0 = w.c.astype(np.float64)
    a0 = w.alpha.astype(np.float64)
    fd_c, fd_a = [], []
    for q in pix:
        iy, ix = divmod(int(q), n)
        for base, other, out in ((c0, a0, fd_c), (a0, c0, fd_a)):
            h = 1e-3 * base[iy, ix]
            plus, minus = base.copy(), base.copy()
            plus[iy, ix] += h
            minus[iy, ix] -= h
            if base is c0:
                out.append((J(plus, other) - J(minus, other)) / (2 * h))
            else:
                out.append((J(other, plus) - J(other, minus)) / (2 * h))
    iy, ix = np.divmod(pix, n)
    assert rel_l2(gc[iy, ix], np.array(fd_c)) < 1e-3
    assert rel_l2(ga[iy, ix], np.array(fd_a)) < 1e-3


@pytest.mark.slow
def test_cfg5_adjoint_full_size_two_sources():
    """1024^2, 3 MHz, two of the 16 sources, receivers on row 1000."""
    import torch
    from paper_2507_13754_gb300 import workloads as W
    w = W.cfg5(n=1024, n_src=16)
    w.src_amp = w.src_amp[[0, 9]]
    plan, psi, info = _gpu_forward(w)
    terms = [i["terms"] for i in info]
    row = w.extras["receiver_row"]
    rng = np.random.default_rng(35)
    g = np.zeros((2, 1024, 1024), np.complex64)  # P^H r: seeded residuals on the receiver row
    g[:, row, :] = (rng.standard_normal((2, 1024)) + 1j * rng.standard_normal((2, 1024))).astype(np.complex64)
    gc = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    ga = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    plan.solve_adjoint(torch.from_numpy(g).cuda(), gc, ga)
    torch.cuda.synchronize()
    rc, ra = _oracle_gradient(w, terms, g)
    assert rel_l2(gc.cpu().numpy(), rc) < GRAD_RTOL
    assert rel_l2(ga.cpu().numpy(), ra) < GRAD_RTOL
    plan.close()


def test_harmonics_to_fifth_match_oracle():
    """Sum-term harmonics 1 .. 5 (Eqs. 28a-28e) on the padded
    grid: 128^2, c0 + 0.2% smooth field, weak power-law absorption (alpha_n =
    n^y alpha), beta = 3.5; each harmonic against the oracle's own chain at
    the GPU's term count."""
    import torch
    import oracle
    from paper_2507_13754_gb300 import workloads as W
    from paper_2507_13754_gb300.solvers import harmonics
    n = 128
    w = W.random_medium(n, seed=61)
    wc = W.random_medium(n, seed=61, contrast=0.002)
    c = wc.c
    alpha = (0.1 * w.alpha).astype(np.float32)
    beta = np.full((n, n), 3.5, np.float32)
    rho = np.full((n, n), 1000.0, np.float32)
    amp = (w.src_amp[:1] * 2e5).astype(np.complex64)
    cd, ad, bd, rd = (torch.from_numpy(x).cuda() for x in (c, alpha, beta, rho))
    fields, infos = harmonics(5, n, w.dx, w.f, w.c0, cd, ad, w.ypow, bd, rd, w.src_ix, w.src_iy, amp)
    ref_fields = []
    for order in range(1, 6):
        f = order * w.f
        m, gh = oracle.plan(n, w.dx, f, w.c0)
        V = oracle.potential(f, w.c0, c.astype(np.float64), alpha.astype(np.float64) * order ** w.ypow, w.ypow, f)
        if order == 1:
            S = oracle.deposit_points(n, w.dx, w.src_ix, w.src_iy, amp[0].astype(np.complex128))
        else:
            S = oracle.harmonic_source(order, 2 * math.pi * w.f, beta, rho, c, ref_fields)
        T = infos[order - 1][0]["terms"]
        assert infos[order - 1][0]["status_name"] == "CONVERGED", (order, infos[order - 1])
        ref, _, _, _ = oracle.solve(n, m, gh, V, S, T, 0.0)
        ref_fields.append(ref)
        got = fields[order - 1][0].cpu().numpy().astype(np.complex128) * 2.0 ** infos[order - 1][0]["log2_scale"]
        assert rel_l2(got, ref) < PARITY_RTOL, order
