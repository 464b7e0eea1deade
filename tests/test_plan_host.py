"""Host-side plan logic through the C ABI, no GPU: tbs_plan_device_bytes
runs the same validation as tbs_plan and returns the size of the plan's
buffer block, so the argument rules and the memory layout are checked here
without touching a device."""
import pytest


def _lib():
    import shutil
    import os
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build the library")
    from paper_2507_13754_gb300 import build, tbs
    build.build()
    return tbs


def _desc(tbs, n=2048, n_rhs=1, **kw):
    d = tbs.tbs_plan_desc_init()
    d.n, d.n_rhs, d.dx, d.freq_hz, d.c0 = n, n_rhs, 3.85e-5, 5e6, 1540.0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_plan_bytes_follow_the_layout():
    tbs = _lib()
    n, m = 2048, 4096
    base = tbs.tbs_plan_device_bytes(_desc(tbs))
    # X and W (N x M each), psi, V and S (N x N complex64), c and alpha
    # (N x N float32 each), the Ghat quadrant
    floor = 2 * n * m * 8 + 3 * n * n * 8 + 2 * n * n * 4 + (m // 2 + 1) * (m // 2 + 2) * 8
    assert floor <= base < floor + (1 << 20)
    # a second RHS adds its own X, W, psi and S, not another V or Ghat
    two = tbs.tbs_plan_device_bytes(_desc(tbs, n_rhs=2))
    assert 2 * n * m * 8 + 2 * n * n * 8 <= two - base < 2 * n * m * 8 + 2 * n * n * 8 + (1 << 20)
    # stored terms scale with max_terms; checkpoints keep about sqrt of them
    kept = tbs.tbs_plan_device_bytes(_desc(tbs, max_terms=64, flags=tbs.TBS_FLAG_KEEP_TERMS))
    assert kept - base >= 64 * n * n * 8
    ck = tbs.tbs_plan_device_bytes(_desc(tbs, max_terms=64,
                                         flags=tbs.TBS_FLAG_KEEP_TERMS | tbs.TBS_FLAG_CHECKPOINT_TERMS))
    assert base < ck < kept
    # the periodic grid has no padding and no Ghat table; the k-space
    # potential adds psi^0 per RHS
    per = tbs.tbs_plan_device_bytes(_desc(tbs, n=4096, flags=tbs.TBS_FLAG_PERIODIC))
    assert 6 * 4096 * 4096 * 8 <= per < 6 * 4096 * 4096 * 8 + (1 << 20)
    ks = tbs.tbs_plan_device_bytes(_desc(tbs, n=4096, flags=tbs.TBS_FLAG_PERIODIC | tbs.TBS_FLAG_KSPACE_ABSORPTION,
                                         kspace_alpha0=5.5e-10, kspace_nu=1.5))
    assert ks - per >= 4096 * 4096 * 8


@pytest.mark.parametrize("kw,code", [
    (dict(n=1), "TBS_ERR_UNSUPPORTED_SIZE"),
    (dict(n=2049), "TBS_ERR_UNSUPPORTED_SIZE"),
    (dict(n=100, flags=8), "TBS_ERR_UNSUPPORTED_SIZE"),                 # periodic: power of two only
    (dict(n_rhs=0), "TBS_ERR_INVALID_ARG"),
    (dict(max_terms=0), "TBS_ERR_INVALID_ARG"),
    (dict(tol=-1.0), "TBS_ERR_INVALID_ARG"),
    (dict(stop_mode=7), "TBS_ERR_INVALID_ARG"),
    (dict(l1_row=2048), "TBS_ERR_INVALID_ARG"),
    (dict(flags=4), "TBS_ERR_INVALID_ARG"),                              # checkpoint without kept terms
    (dict(n=128, flags=8 | 1), "TBS_ERR_INVALID_ARG"),                  # periodic with kept terms
    (dict(n=128, flags=8, abl_width=65, abl_zeta=1.0), "TBS_ERR_INVALID_ARG"),
    (dict(n=128, flags=8, abl_width=8), "TBS_ERR_INVALID_ARG"),         # layer without zeta
    (dict(n=128, flags=16, kspace_alpha0=1e-9, kspace_nu=1.5), "TBS_ERR_INVALID_ARG"),   # k-space, not periodic
    (dict(n=128, flags=8 | 16, kspace_alpha0=1e-9, kspace_nu=3.0), "TBS_ERR_INVALID_ARG"),
    (dict(n=128, flags=32), "TBS_ERR_INVALID_ARG"),                     # CBS, not periodic
    (dict(n=128, flags=8 | 16 | 32, kspace_alpha0=1e-9, kspace_nu=1.5), "TBS_ERR_INVALID_ARG"),
])
def test_plan_rejects_what_it_cannot_do(kw, code):
    tbs = _lib()
    with pytest.raises(tbs.TbsError) as e:
        tbs.tbs_plan_device_bytes(_desc(tbs, **kw))
    assert code in str(e.value)


def test_flag_values_match_the_header():
    tbs = _lib()
    assert (tbs.TBS_FLAG_KEEP_TERMS, tbs.TBS_FLAG_NO_GRAPH, tbs.TBS_FLAG_CHECKPOINT_TERMS, tbs.TBS_FLAG_PERIODIC,
            tbs.TBS_FLAG_KSPACE_ABSORPTION, tbs.TBS_FLAG_CBS) == (1, 2, 4, 8, 16, 32)


def test_synthesize_rejects_bad_arguments_before_any_launch():
    # argument checks run on the host before the kernel is launched; the
    # "device" pointers here are never dereferenced
    tbs = _lib()
    f1, out = 0x10000, 0x20000
    good = (f1, 8, 1e-4, 1e6, 1.0)
    cases = [
        ([(0, 8, 1e-4, 1e6, 1.0)], dict()),                     # NULL field
        ([(f1, 1, 1e-4, 1e6, 1.0)], dict()),                    # a one-cell grid
        ([(f1, 8, 0.0, 1e6, 1.0)], dict()),                     # dx = 0
        ([(f1, 8, 1e-4, float("nan"), 1.0)], dict()),           # frequency not finite
        ([(out, 8, 1e-4, 1e6, 1.0)], dict()),                   # out aliases a field
        ([good], dict(n_rhs=0)),
        ([good], dict(nx=0)),
        ([good], dict(n_t=0)),
        ([good], dict(dt=float("inf"))),
    ]
    for entries, kw in cases:
        a = dict(n_rhs=1, x0=0.0, y0=0.0, sx=1e-4, sy=1e-4, nx=4, ny=4, t0=0.0, dt=1e-8, n_t=16)
        a.update(kw)
        with pytest.raises(tbs.TbsError) as e:
            tbs.tbs_synthesize(entries, a["n_rhs"], a["x0"], a["y0"], a["sx"], a["sy"], a["nx"], a["ny"], a["t0"],
                               a["dt"], a["n_t"], out)
        assert "TBS_ERR_INVALID_ARG" in str(e.value), (entries, kw)


def test_noalloc_rejects_sizes_and_null_pointers_on_the_host():
    tbs = _lib()
    for n in (1, tbs.TBS_NOALLOC_MAX_N + 1):
        with pytest.raises(tbs.TbsError) as e:
            tbs.tbs_apply_green_noalloc(n, 0x10000, 0x20000, 0x30000)
        assert "TBS_ERR_UNSUPPORTED_SIZE" in str(e.value)
    with pytest.raises(tbs.TbsError) as e:
        tbs.tbs_apply_green_noalloc(64, 0, 0x20000, 0x30000)
    assert "TBS_ERR_INVALID_ARG" in str(e.value)
