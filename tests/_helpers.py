"""Shared test plumbing: run one workload through the CUDA path or the oracle.

Inputs come from ``paper_2507_13754_gb300.workloads`` (seeded, no method
arithmetic); the oracle side upcasts the very same float32/complex64 inputs
to float64/complex128.
"""
import functools

import numpy as np

PARITY_RTOL = 2e-5  # relative L2 bar for a complex64 field against the FP64 oracle


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_solve(w, max_terms=None, tol=None, stop_mode=0, l1_row=None, keep_terms=False,
                 rhs=None, V=None, src=None):
    """Oracle solve of workload w for each RHS: list of (psi, info, norms, terms)."""
    import oracle
    m, gh = oracle.plan(w.n, w.dx, w.f, w.c0)
    if V is None:
        V = oracle.potential(w.f, w.c0, w.c.astype(np.float64),
                             None if w.alpha is None else w.alpha.astype(np.float64),
                             w.ypow, w.f_ref)
    out = []
    rlist = range(w.n_rhs) if rhs is None else rhs
    for r in rlist:
        s = src[r] if src is not None else oracle.deposit_points(
            w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[r].astype(np.complex128))
        out.append(oracle.solve(w.n, m, gh, V, s, w.max_terms if max_terms is None else max_terms,
                                w.tol if tol is None else tol, stop_mode=stop_mode,
                                l1_row=l1_row, keep_terms=keep_terms))
    return out


def gpu_plan(w, keep_terms=False, max_terms=None, tol=None, stop_mode=0, l1_row=-1, **kw):
    from paper_2507_13754_gb300 import tbs
    return tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs,
                    max_terms=w.max_terms if max_terms is None else max_terms,
                    tol=w.tol if tol is None else tol, stop_mode=stop_mode, l1_row=l1_row,
                    keep_terms=keep_terms, **kw)


def gpu_solve(w, **kw):
    """(psi numpy [n_rhs, N, N], info dicts, plan)"""
    import torch
    from paper_2507_13754_gb300 import tbs
    plan = gpu_plan(w, **kw)
    c = torch.from_numpy(w.c).cuda()
    al = torch.from_numpy(w.alpha).cuda() if w.alpha is not None else None
    plan.set_medium(c, al, w.ypow, w.f_ref)
    plan.set_sources(w.src_ix, w.src_iy, w.src_amp)
    psi, infos = plan.solve()
    return psi.cpu().numpy(), tbs.Plan.info_dicts(infos), plan


@functools.lru_cache(maxsize=None)
def library():
    from paper_2507_13754_gb300 import build, tbs
    build.build()
    return tbs.load_library()
