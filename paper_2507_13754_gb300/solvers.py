"""Drivers over the C ABI: the differentiable field, the second harmonic and the
surface-pressure calibration.  Every arithmetic step runs in libtbs.so; these
functions only sequence the calls and move tensors.

TBSField          psi(c, alpha) as a torch.autograd.Function whose backward is
                  tbs_solve_adjoint (adjoint of the truncated series, Eqs. 18-20).
second_harmonic   fundamental series at f, source S2 = -(1/2) xi (2 omega)^2 psi1^2
                  (Eqs. 11, 28b), second series at 2f (Section 2.3.4).
surface_scale     the amplitude factor that brings the mean |u_0| over the element
                  cells to a target pressure.
"""
from __future__ import annotations

import math

import numpy as np

from . import tbs


def _torch():
    import torch
    return torch


class TBSField:
    """psi = TBSField.apply(c, alpha, plan, ix, iy, amp, y_pow, f_ref).

    The plan must carry TBS_FLAG_KEEP_TERMS (``Plan(..., keep_terms=True)``).
    Forward runs tbs_set_medium, tbs_set_sources and tbs_solve; backward runs
    tbs_solve_adjoint with PyTorch's complex gradient g = dL/dRe(psi) +
    i dL/dIm(psi) and returns dL/dc and dL/dalpha.  The plan keeps the terms of
    its last solve only: call backward before the next forward on the same
    plan."""

    @staticmethod
    def apply(c, alpha, plan, ix, iy, amp, y_pow=1.0, f_ref=None):
        return _tbs_field_fn().apply(c, alpha, plan, ix, iy, amp, y_pow, f_ref)


_fn_cache = None


def _tbs_field_fn():
    global _fn_cache
    if _fn_cache is not None:
        return _fn_cache
    torch = _torch()

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, c, alpha, plan, ix, iy, amp, y_pow, f_ref):
            plan.set_medium(c, alpha, y_pow, f_ref)
            plan.set_sources(ix, iy, amp)
            psi, infos = plan.solve()
            ctx.plan = plan
            ctx.infos = tbs.Plan.info_dicts(infos)
            ctx.shapes = (c.shape, None if alpha is None else alpha.shape)
            ctx.has_alpha = alpha is not None
            return psi

        @staticmethod
        def backward(ctx, grad_psi):
            plan = ctx.plan
            gc = torch.empty(ctx.shapes[0], dtype=torch.float32, device=grad_psi.device)
            ga = torch.empty(ctx.shapes[1], dtype=torch.float32, device=grad_psi.device) \
                if ctx.has_alpha else None
            plan.solve_adjoint(grad_psi.contiguous().to(torch.complex64), gc, ga)
            return gc, ga, None, None, None, None, None, None

    _fn_cache = _Fn
    return _Fn


def surface_scale(plan, ix, iy, target, c, alpha=None, y_pow=1.0, f_ref=None):
    """Factor s such that the elements driven with amplitude s produce a mean
    |u_0| of `target` over their own cells (u_0 = G S, Eq. 20), evaluated with
    the plan's own first term.  The plan is left with unit sources set."""
    torch = _torch()
    n = plan.n
    one = tbs.Plan(n, plan.desc.dx, plan.freq_hz, plan.desc.c0, n_rhs=1, max_terms=1, tol=0.0)
    one.set_medium(c, alpha, y_pow, f_ref)
    one.set_sources(ix, iy, np.ones((1, len(ix)), np.complex64))
    u0, _ = one.solve()
    one.close()
    vals = u0[0, torch.as_tensor(np.asarray(iy), device=u0.device).long(),
              torch.as_tensor(np.asarray(ix), device=u0.device).long()]
    return float(target / vals.abs().mean().item())


def second_harmonic(n, dx, f0, c0, c, alpha, y_pow, beta, rho, ix, iy, amp,
                    max_terms=64, tol=1e-6, n_rhs=1, max_terms_harmonic=None):
    """Fundamental field psi1 at f0 and second-harmonic field psi2 at 2 f0.

    c, beta, rho: float32 [N, N] CUDA tensors; alpha: absorption [Np/m] at f0
    (the harmonic uses alpha * 2**y_pow, the power law of Eq. 3) or None.
    max_terms_harmonic: the second series' cap (default max_terms); at twice
    the frequency the same scatterer is twice as strong in phase, so that
    series contracts more slowly and may need more terms.
    Returns (psi1, info1, psi2, info2)."""
    p1 = tbs.Plan(n, dx, f0, c0, n_rhs=n_rhs, max_terms=max_terms, tol=tol)
    p1.set_medium(c, alpha, y_pow, f0)
    p1.set_sources(ix, iy, amp)
    psi1, i1 = p1.solve()
    p2 = tbs.Plan(n, dx, 2.0 * f0, c0, n_rhs=n_rhs, max_terms=max_terms_harmonic or max_terms, tol=tol)
    p2.set_medium(c, None if alpha is None else alpha * (2.0 ** y_pow), y_pow, 2.0 * f0)
    p2.set_harmonic2_source(psi1, beta, rho, c, 2.0 * math.pi * f0)
    psi2, i2 = p2.solve()
    out = (psi1, tbs.Plan.info_dicts(i1), psi2, tbs.Plan.info_dicts(i2))
    p1.close()
    p2.close()
    return out


def harmonics(n_max, n, dx, f0, c0, c, alpha, y_pow, beta, rho, ix, iy, amp, max_terms=64, tol=1e-6,
              n_rhs=1, **plan_kw):
    """Fields of the fundamental and harmonics 2 .. n_max (<= 5) of the
    sum-term series (Eqs. 28a-28e): harmonic
    n solves the same series at n f0 with the source formed from psi_1 ..
    psi_{n-1}.  alpha: absorption [Np/m] at f0 (harmonic n uses
    alpha n^y_pow) or None.  plan_kw go to every Plan (e.g. periodic=True,
    abl_width, abl_zeta, stop_mode, l1_row: the paper's periodic run, where
    eps_factor k0^2 at n f0 is the paper's eps_n = 0.8 n^2 k^2).
    Returns ([psi_1, ..., psi_nmax], [info dicts per harmonic]).

    Harmonic n is returned as psi_n / 2^e_n, e_n = the "log2_scale" entry of
    its info dicts (e_1 = 0): the harmonics fall off geometrically (about
    1e-9 per order in the paper's run, psi_5 near 1e-36) and would leave
    FP32's range; the series is linear in its source, so each harmonic is
    solved for a source scaled to order one and the scale is carried."""
    if not 1 <= n_max <= 5:
        raise ValueError("n_max must be in 1 .. 5")
    fields, infos, exps, mags = [], [], [], []
    for order in range(1, n_max + 1):
        p = tbs.Plan(n, dx, order * f0, c0, n_rhs=n_rhs, max_terms=max_terms, tol=tol, **plan_kw)
        a_n = None if alpha is None else alpha * (float(order) ** y_pow)
        if plan_kw.get("periodic") and c is None:
            p.set_potential(_torch().zeros((n, n), dtype=_torch().complex64, device="cuda"))
        else:
            p.set_medium(c, a_n, y_pow, order * f0)
        if order == 1:
            e = 0
            p.set_sources(ix, iy, amp)
        else:
            e = _harmonic_exponent(order, exps, mags)
            cc = c if c is not None else _torch().full((n, n), c0, dtype=_torch().float32, device="cuda")
            p.set_harmonic_source(order, fields, beta, rho, cc, 2.0 * math.pi * f0,
                                  psi_scale=[2.0 ** x for x in exps], source_scale=2.0 ** -e)
        psi, info = p.solve()
        recs = tbs.Plan.info_dicts(info)
        for r in recs:
            r["log2_scale"] = e
        rms = max(r["psi_norm"] for r in recs) / n
        fields.append(psi)
        infos.append(recs)
        exps.append(e)
        mags.append(e + math.log2(rms) if rms > 0 and math.isfinite(rms) else -math.inf)
        p.close()
    return fields, infos


def _harmonic_exponent(order, exps, mags):
    """e_n for harmonic `order`: the largest log2 magnitude of its source's
    products psi_a psi_b (a + b = order), from the RMS of the stored fields,
    so that the scaled source is of order one; 0 when every field is zero."""
    best = max(mags[a - 1] + mags[order - a - 1] for a in range(1, order // 2 + 1))
    return int(round(best)) if math.isfinite(best) else 0

