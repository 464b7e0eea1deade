"""The allocation-free G application against the plan-based one.

tbs_apply_green_noalloc serves callers that may not call cudaMalloc (graph
capture, allocator internals, real-time loops with memory fixed at start-up):
its scratch is a fixed array inside the library.  This file is collected last
so that a run stopping at the first failure has already run everything else;
it passes alone in a fresh process (the first call then sets the device up)
and after the other tests.
"""
import numpy as np
import pytest

from _helpers import library, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,conj", [(200, 0), (256, 1), (37, 0)])
def test_noalloc_matches_plan_entry_point_twice(n, conj):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(n, seed=21)
    plan = tbs.Plan(w.n, w.dx, w.f, w.c0)
    ghat = torch.from_numpy(plan.ghat_quadrant()).cuda()
    rng = np.random.default_rng(22)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the scratch array
        f = (rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))).astype(np.complex64)
        fd = torch.from_numpy(f).cuda()
        ref = plan.apply_green(fd, conj_kernel=bool(conj)).cpu().numpy()[0]
        out = torch.empty((n, n), dtype=torch.complex64, device="cuda")
        tbs.tbs_apply_green_noalloc(n, ghat.data_ptr(), fd.data_ptr(), out.data_ptr(), conj, stream)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) < 2e-6, (n, conj, call)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    library()
    from paper_2507_13754_gb300 import tbs
    x = torch.zeros((2, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(tbs.TbsError) as ei:
        tbs.tbs_apply_green_noalloc(tbs.TBS_NOALLOC_MAX_N + 1, x.data_ptr(), x.data_ptr(),
                                    x.data_ptr() + 8, 0)
    assert "TBS_NOALLOC_MAX_N" in str(ei.value)
