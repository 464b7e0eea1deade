"""GB300-native traditional Born series (TBS) solver for the 2D Helmholtz
equation (arxiv 2507.13754): a C-ABI CUDA library (include/tbs.h,
``_lib/libtbs.so``) with a thin Python binding.

    from paper_2507_13754_gb300 import build, tbs
    build.build()                       # nvcc, sm_103a
    plan = tbs.Plan(n, dx, f, c0, ...)  # Ghat plan on the device
"""
__all__ = ["build", "tbs", "workloads"]
