"""The allocation-free G application against the plan-based one and the oracle.

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


@pytest.mark.parametrize("n,conj", [(200, 0), (256, 1), (37, 0), (2, 0), (9, 1)])
def test_noalloc_matches_plan_entry_point_twice(n, conj):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()
    import oracle
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(n, seed=21)
    plan = tbs.Plan(w.n, w.dx, w.f, w.c0)
    ghat = torch.from_numpy(plan.ghat_quadrant()).cuda()
    m, gh = oracle.plan(w.n, w.dx, w.f, w.c0)
    rng = np.random.default_rng(22)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the scratch array
        f = (rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))).astype(np.complex64)
        fd = torch.from_numpy(f).cuda()
        ref = plan.apply_green(fd, conj_kernel=bool(conj)).cpu().numpy()[0]
        out = torch.empty((n, n), dtype=torch.complex64, device="cuda")
        tbs.tbs_apply_green_noalloc(n, ghat.data_ptr(), fd.data_ptr(), out.data_ptr(), conj, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert rel_l2(got, ref) < 2e-6, (n, conj, call)
        # and against the oracle's zero-padded convolution itself
        ora = oracle.apply_g(n, m, gh, f[0].astype(np.complex128), conj_kernel=bool(conj))
        assert rel_l2(got, ora) < 2e-6, (n, conj, call)
    plan.close()


def test_noalloc_call_changes_no_device_memory_use():
    """After its set-up, a call leaves the device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    library()
    from paper_2507_13754_gb300 import tbs, workloads as W
    n = 128
    w = W.random_medium(n, seed=23)
    plan = tbs.Plan(w.n, w.dx, w.f, w.c0)
    ghat = torch.from_numpy(plan.ghat_quadrant()).cuda()
    f = torch.ones((n, n), dtype=torch.complex64, device="cuda")
    out = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    tbs.tbs_apply_green_noalloc(n, ghat.data_ptr(), f.data_ptr(), out.data_ptr(), 0, stream)  # set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        tbs.tbs_apply_green_noalloc(n, ghat.data_ptr(), f.data_ptr(), out.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
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
