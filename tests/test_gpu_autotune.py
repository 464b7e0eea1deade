"""Column- and row-pass kernel variants: identical results, autotuned choice."""
import numpy as np
import pytest

from _helpers import gpu_solve, library, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()


# M = 1024, 2048, 4096: the pipelined kernel (one and two columns per thread,
# the latter also staggered; at 4096 also with the radix split 8 x 8 x 8 x 8),
# then col_kernel's tile shapes (3, 2 and 1 of them); M = 256: one shape.  Row pass: persistent and one block per row for
# M >= 512 and even N, one variant otherwise (odd N = 1001).
@pytest.mark.parametrize("n,expect,rows", [(400, 6, 2), (1000, 5, 2), (1001, 5, 1), (2048, 5, 2), (100, 1, 1)])
def test_variants_agree_bitwise_and_autotune_picks_one(tmp_path, n, expect, rows):
    from paper_2507_13754_gb300 import autotune, tbs, workloads as W
    w = W.random_medium(n, seed=51, n_rhs=2)
    w.max_terms, w.tol = 4, 0.0
    psi0, info0, plan = gpu_solve(w)
    nv = tbs.tbs_col_variants(plan.handle)
    nr = tbs.tbs_row_variants(plan.handle)
    assert nv == expect and nr == rows
    for v in range(1, nv):
        tbs.tbs_set_col_variant(plan.handle, v)
        psi_v, _ = plan.solve()
        if "radix 8x8x8x8" in tbs.tbs_col_variant_name(plan.handle):
            # another radix split rounds differently: agreement to FP32 rounding
            assert rel_l2(psi_v.cpu().numpy(), psi0) < 1e-6, (n, v)
        else:  # the same arithmetic in every other shape
            assert np.array_equal(psi_v.cpu().numpy(), psi0), (n, v)
    tbs.tbs_set_col_variant(plan.handle, 0)
    for v in range(1, nr):
        tbs.tbs_set_row_variant(plan.handle, v)
        assert tbs.tbs_row_variant_name(plan.handle) == "one block per row"
        psi_v, _ = plan.solve()
        assert np.array_equal(psi_v.cpu().numpy(), psi0), (n, "row", v)
    cache = str(tmp_path / "tune.json")
    (best, rbest), times = autotune.tune(plan, cache_path=cache, reps=3)
    assert 0 <= best < nv and 0 <= rbest < nr
    if nv > 1 or nr > 1:
        if nv > 1:
            assert len(times["col"]) == nv and min(times["col"]) == times["col"][best]
        if nr > 1:
            assert len(times["row"]) == nr and min(times["row"]) == times["row"][rbest]
        again, times2 = autotune.tune(plan, cache_path=cache)  # cached: no timing
        assert again == (best, rbest) and times2 is None
    # the row timing wrote a scratch field, not the plan's result
    psi_t, _ = plan.solve()
    assert np.array_equal(psi_t.cpu().numpy(), psi0)
    with pytest.raises(tbs.TbsError):
        tbs.tbs_set_col_variant(plan.handle, nv)
    with pytest.raises(tbs.TbsError):
        tbs.tbs_set_row_variant(plan.handle, nr)
    plan.close()


@pytest.mark.parametrize("n,rows,cols,ks", [(128, 1, 2, False), (512, 2, 2, False), (1024, 2, 4, False),
                                             (1024, 2, 4, True), (2048, 2, 4, False), (4096, 2, 4, True)])
def test_periodic_variants_agree_bitwise(n, rows, cols, ks):
    """Periodic plans: every column-pass variant (lockstep with one or two
    columns per thread; from M = 1024 the pipelined kernel, plain and
    staggered) and the row pass's variants give the same field, with and
    without the k-space potential."""
    import math
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(n, seed=52, n_rhs=2)
    k0 = 2 * math.pi * w.f / w.c0
    kw = dict(kspace_alpha0=2e-8, kspace_nu=1.5) if ks else {}
    p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=2, max_terms=6, tol=0.0, periodic=True, eps_factor=0.8,
                 abl_width=16, abl_zeta=4.0 / (16 * w.dx), div_window=1 << 30, div_factor=math.inf, **kw)
    # k-space potential: the medium is homogeneous (U = 0), VV acts in k-space
    u = 0.0 if ks else 0.05 * k0 * k0
    p.set_potential(torch.full((n, n), u, dtype=torch.complex64, device="cuda"))
    p.set_sources(w.src_ix, w.src_iy, w.src_amp)
    assert tbs.tbs_col_variants(p.handle) == cols
    assert tbs.tbs_row_variants(p.handle) == rows
    psi0, _ = p.solve()
    psi0 = psi0.cpu().numpy()
    assert np.isfinite(psi0).all() and np.abs(psi0).max() > 0
    assert tbs.tbs_col_variant_name(p.handle) == "periodic, lockstep, 2 columns/thread"
    for v in range(1, cols):
        tbs.tbs_set_col_variant(p.handle, v)
        name = tbs.tbs_col_variant_name(p.handle)
        assert ("pipelined" in name) == (v >= 2) and (("1 column" in name) == (v == 1)), name
        psi1, _ = p.solve()
        assert np.array_equal(psi1.cpu().numpy(), psi0), (n, ks, v)
    if rows > 1:
        tbs.tbs_set_row_variant(p.handle, 1)
        psi2, _ = p.solve()
        assert np.array_equal(psi2.cpu().numpy(), psi0)
        best, times = tbs.tbs_autotune_rows(p.handle, 2)
        assert 0 <= best < rows and len(times) == rows
        psi3, _ = p.solve()
        assert np.array_equal(psi3.cpu().numpy(), psi0)
    p.close()
