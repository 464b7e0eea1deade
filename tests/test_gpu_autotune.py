"""Column-pass tile-shape variants: identical results, autotuned choice."""
import numpy as np
import pytest

from _helpers import gpu_solve, library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()


# M = 1024, 2048, 4096: the pipelined kernel (one and two columns per thread,
# the latter also staggered), then col_kernel's tile shapes (3, 2 and 1 of
# them); M = 256: one shape
@pytest.mark.parametrize("n,expect", [(400, 6), (1000, 5), (2048, 4), (100, 1)])
def test_variants_agree_bitwise_and_autotune_picks_one(tmp_path, n, expect):
    from paper_2507_13754_gb300 import autotune, tbs, workloads as W
    w = W.random_medium(n, seed=51, n_rhs=2)
    w.max_terms, w.tol = 4, 0.0
    psi0, info0, plan = gpu_solve(w)
    nv = tbs.tbs_col_variants(plan.handle)
    assert nv == expect
    for v in range(1, nv):
        tbs.tbs_set_col_variant(plan.handle, v)
        psi_v, _ = plan.solve()
        assert np.array_equal(psi_v.cpu().numpy(), psi0), (n, v)
    cache = str(tmp_path / "tune.json")
    best, times = autotune.tune(plan, cache_path=cache, reps=3)
    assert 0 <= best < nv
    if nv > 1:
        assert len(times) == nv and min(times) == times[best]
        best2, times2 = autotune.tune(plan, cache_path=cache)  # cached: no timing
        assert best2 == best and times2 is None
    with pytest.raises(tbs.TbsError):
        tbs.tbs_set_col_variant(plan.handle, nv)
    plan.close()


def test_periodic_variants_agree_bitwise():
    """Periodic plans: one and two columns per thread give the same field."""
    import math
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(128, seed=52, n_rhs=2)
    k0 = 2 * math.pi * w.f / w.c0
    p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=2, max_terms=6, tol=0.0, periodic=True, eps_factor=0.8,
                 abl_width=16, abl_zeta=4.0 / (16 * w.dx), div_window=1 << 30, div_factor=math.inf)
    p.set_potential(torch.full((128, 128), 0.05 * k0 * k0, dtype=torch.complex64, device="cuda"))
    p.set_sources(w.src_ix, w.src_iy, w.src_amp)
    assert tbs.tbs_col_variants(p.handle) == 2
    psi0, _ = p.solve()
    psi0 = psi0.cpu().numpy()
    tbs.tbs_set_col_variant(p.handle, 1)
    assert "2 columns" in tbs.tbs_col_variant_name(p.handle)
    psi1, _ = p.solve()
    assert np.array_equal(psi1.cpu().numpy(), psi0)
    p.close()
