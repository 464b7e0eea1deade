"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function include/tbs.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tbs_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    from paper_2507_13754_gb300 import tbs
    assert sorted(tbs.EXPORTED) == _declared()


def test_library_builds_and_exports_every_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2507_13754_gb300 import build, tbs
    lib_path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(tbs_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    lib = tbs.load_library()
    for name in _declared():
        assert hasattr(lib, name)
    # no compute call here; only the host-only helpers
    d = tbs.tbs_plan_desc_init()
    assert (d.n_rhs, d.max_terms, d.tol, d.div_grace, d.div_window) == (1, 64, 1e-6, 8, 4)
    assert tbs.load_library().tbs_status_string(2) == b"TBS_ERR_UNSUPPORTED_SIZE"


def test_library_is_built_for_sm_103a_only():
    from paper_2507_13754_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_workloads_are_seeded_and_shaped():
    import numpy as np
    from paper_2507_13754_gb300 import workloads as W
    a, b = W.cfg2(n=256), W.cfg2(n=256)
    assert np.array_equal(a.c, b.c) and a.c.dtype == np.float32
    assert abs(np.abs(a.c / 1540.0 - 1).max() - 0.02) < 1e-6
    assert a.src_amp.shape == (1, 16) and np.allclose(np.abs(a.src_amp), 1)
    w1 = W.cfg1()
    assert w1.n == 256 and w1.max_terms == 24 and w1.tol == 0.0
    assert w1.src_amp.shape == (1, 32) and set(w1.src_iy.tolist()) == {16}
    assert (w1.c == 1530.0).sum() > 0
    lst = W.cfg4_list(scale=0.25, n_freq=4, n_ang=8)
    assert len(lst) == 4 and all(x.n_rhs == 8 for x in lst)
    assert lst[0].n < lst[-1].n
