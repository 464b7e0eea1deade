"""Plain cuFFT + elementwise build of the same Born recurrence (comparison only).

One term u_{n+1} = G (V u_n) (Eq. 19) the straightforward way: embed V u_n in
a zero M x M array, a full 2D forward FFT (cuFFT through torch.fft), a
pointwise product with the full M x M spectrum, a full 2D inverse FFT, a
crop, the accumulation psi += u and the norms as separate elementwise ops.
It shares the plan's spectrum (tbs_get_ghat) so that both paths compute the
same G; it is the baseline the fused kernels are measured against, not a
fallback of the library.
"""
from __future__ import annotations

import math

import numpy as np


def full_spectrum(ghat_quadrant, m):
    """Full M x M spectrum from the stored quadrant (even in both axes)."""
    import torch
    q = torch.as_tensor(ghat_quadrant)
    idx = torch.arange(m)
    idx = torch.minimum(idx, m - idx)
    return q[idx][:, idx].contiguous()


def potential(f, c0, c, alpha=None, ypow=1.0, f_ref=None):
    """V = p^2 - k0^2, p = omega/c + alpha (tan(pi y/2) delta + i), as torch ops."""
    import torch
    w = 2 * math.pi * f
    k0 = w / c0
    p = (w / c.double()).to(torch.complex128)
    if alpha is not None:
        fr = f if f_ref is None else f_ref
        delta = 1.0 - (fr / f) ** (ypow - 1.0) if fr > 0 else 1.0
        p = p + alpha.double() * complex(math.tan(math.pi * ypow / 2) * delta, 1.0)
    return (p * p - k0 * k0).to(torch.complex64)


class CufftBornSeries:
    def __init__(self, n, m, ghat_full, device="cuda"):
        import torch
        self.n, self.m = n, m
        self.G = ghat_full.to(device=device, dtype=torch.complex64)
        self.buf = torch.zeros((m, m), dtype=torch.complex64, device=device)

    def apply_g(self, f):
        import torch
        n = self.n
        self.buf.zero_()
        self.buf[:n, :n] = f
        spec = torch.fft.fft2(self.buf)
        spec *= self.G
        return torch.fft.ifft2(spec, norm="forward")[:n, :n]

    def solve_fixed(self, V, S, terms):
        """psi = sum_{n < terms} u_n with per-term FP64 norms (no early stop)."""
        import torch
        u = self.apply_g(S)
        psi = u.clone()
        norms = [torch.linalg.vector_norm(u.to(torch.complex128))]
        for _ in range(terms - 1):
            u = self.apply_g(V * u)
            psi += u
            norms.append(torch.linalg.vector_norm(u.to(torch.complex128)) /
                         torch.linalg.vector_norm(psi.to(torch.complex128)))
        return psi, norms


def dense_source(n, dx, ix, iy, amp, device="cuda"):
    import torch
    s = np.zeros((n, n), np.complex64)
    np.add.at(s, (np.asarray(iy), np.asarray(ix)), np.asarray(amp, np.complex64) / (dx * dx))
    return torch.from_numpy(s).to(device)
