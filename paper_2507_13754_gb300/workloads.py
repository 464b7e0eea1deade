"""Seeded synthetic inputs for the five workloads (media, sources, stop rules).

This module holds no step of the Born-series method: it only produces the
inputs both the CUDA path and the CPU oracle consume -- sound speed c(x),
absorption alpha(x), nonlinearity beta(x), density rho(x), source cells and
complex source amplitudes.  Values are rounded to the precision the library's
C ABI takes (float32 media, complex64 amplitudes), so both sides see the same
numbers.

Geometry follows the paper's setups (Section 3.1: a line array of point
emitters on one grid row, a disk scatterer, power-law absorbing tissue, a
nonlinear medium) at the sizes of the five benchmark workloads:

  cfg1  256^2 lossless, disk r = 40 cells at 1530 m/s, 32 unit emitters, 24 terms
  cfg2  2048^2 absorbing/dispersive tissue, +-2% Gaussian random c, 128-element
        focused array, residual 1e-6 (<= 64 terms)
  cfg3  2048^2 water + fat ellipse, fundamental at 2 MHz then 2nd harmonic
  cfg4  64 frequencies x 8 steering angles on the cfg1 medium at fixed size
  cfg5  1024^2 gradient workload: 16 sources, receivers on row 1000
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NP_PER_DB = 1.0 / (20.0 * math.log10(math.e))  # 1 dB = 0.1151 Np


@dataclasses.dataclass
class Workload:
    name: str
    n: int                      # unpadded grid side N
    dx: float                   # cell size [m]
    f: float                    # solve frequency [Hz]
    c0: float                   # background speed [m/s]; k0 = 2 pi f / c0
    c: np.ndarray               # float32 [N, N] sound speed
    alpha: np.ndarray | None    # float32 [N, N] absorption [Np/m] at f, or None
    ypow: float                 # power-law exponent y
    f_ref: float                # frequency at which c is the phase speed
    src_ix: np.ndarray          # int32 [P]
    src_iy: np.ndarray          # int32 [P]
    src_amp: np.ndarray         # complex64 [n_rhs, P]
    max_terms: int
    tol: float                  # 0 => fixed number of terms (= max_terms)
    extras: dict = dataclasses.field(default_factory=dict)

    @property
    def n_rhs(self) -> int:
        return int(self.src_amp.shape[0])


def db_cm_mhz_to_np_m(a_db: float, f_hz: float, ypow: float) -> float:
    """alpha [Np/m] at f from a power law given in dB/(cm MHz^y)."""
    return a_db * (f_hz / 1e6) ** ypow * NP_PER_DB * 100.0


def line_array(n: int, n_el: int, pitch: int, row: int):
    """Element cells of a line array centred on column N/2, one row."""
    first = n // 2 - (n_el * pitch) // 2 + pitch // 2
    ix = first + pitch * np.arange(n_el)
    iy = np.full(n_el, row)
    return ix.astype(np.int32), iy.astype(np.int32)


def focus_amplitudes(ix, dx, k0, focus_m, centre_col):
    """Delay law that brings every element in phase at depth focus_m on axis."""
    xj = (ix - centre_col) * dx
    return np.exp(-1j * k0 * (np.sqrt(xj * xj + focus_m ** 2) - focus_m))


def steer_amplitudes(ix, dx, k0, theta, centre_col):
    xj = (ix - centre_col) * dx
    return np.exp(-1j * k0 * xj * math.sin(theta))


def gaussian_random_field(n: int, corr_cells: float, amp: float, seed: int) -> np.ndarray:
    """White N(0,1) noise (PCG64 seed) convolved periodically with
    exp(-r^2/(2 s^2)), s = corr/2 (correlation ~ exp(-r^2/corr^2)), scaled to
    max |delta| = amp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n))
    s = corr_cells / 2.0
    k = np.fft.fftfreq(n) * n
    d2 = np.minimum(np.abs(k), n - np.abs(k)) ** 2
    ker = np.exp(-(d2[:, None] + d2[None, :]) / (2.0 * s * s))
    fld = np.real(np.fft.ifft2(np.fft.fft2(w) * np.fft.fft2(ker)))
    return fld * (amp / np.max(np.abs(fld)))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def cfg1(n: int = 256, terms: int = 24) -> Workload:
    """256^2 (512^2 padded), 1 MHz, c0 1500, dx = lambda/8, disk r = 40 cells
    at 1530 m/s centred, 32 unit emitters one cell apart on row 16."""
    f, c0 = 1e6, 1500.0
    dx = c0 / f / 8.0
    cy = cx = n // 2
    radius = 40 * n / 256.0
    yy, xx = np.mgrid[0:n, 0:n]
    inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= radius ** 2
    c = np.where(inside, 1530.0, c0)
    n_el = max(1, 32 * n // 256)
    ix, iy = line_array(n, n_el, 1, max(1, 16 * n // 256))
    amp = np.ones((1, n_el), np.complex64)
    return Workload("cfg1_disk_%d" % n, n, dx, f, c0, _f32(c), None, 1.0, f,
                    ix, iy, amp, terms, 0.0)


def cfg2(n: int = 2048, max_terms: int = 64, tol: float = 1e-6, seed: int = 20250713) -> Workload:
    """Absorbing/dispersive tissue at 5 MHz: c = 1540 (1 + delta), delta a
    +-2% Gaussian random field with 1 mm correlation; alpha = 0.5 dB/cm/MHz^1.1;
    128-element array (pitch lambda/2) focused at 40 mm; residual 1e-6."""
    f, c0, ypow = 5e6, 1540.0, 1.1
    dx = c0 / f / 8.0
    delta = gaussian_random_field(n, 1e-3 / dx, 0.02, seed)
    c = c0 * (1.0 + delta)
    alpha = np.full((n, n), db_cm_mhz_to_np_m(0.5, f, ypow))
    n_el = min(128, max(4, n // 16))
    ix, iy = line_array(n, n_el, 4, 16)
    k0 = 2 * math.pi * f / c0
    amp = focus_amplitudes(ix, dx, k0, min(40e-3, 0.5 * n * dx), n // 2)[None, :]
    return Workload("cfg2_tissue_%d" % n, n, dx, f, c0, _f32(c), _f32(alpha), ypow, f,
                    ix, iy, amp.astype(np.complex64), max_terms, tol)


def cfg3(n: int = 2048, max_terms: int = 64, tol: float = 1e-6) -> Workload:
    """Nonlinear medium, fundamental at 2 MHz: water (1500 m/s, 1000 kg/m^3,
    beta 3.5, 0.0022 dB/cm/MHz^2) with a fat-like ellipse (1450 m/s, beta 5.0,
    semi-axes 4 mm axial x 2 mm lateral, 40 mm from the array); 64 elements,
    pitch lambda/2, scaled afterwards to 0.5 MPa at the element cells
    (``extras['surface_pressure']``)."""
    f, c0, ypow = 2e6, 1500.0, 2.0
    dx = c0 / f / 8.0
    yy, xx = np.mgrid[0:n, 0:n]
    row = 16
    depth = min(40e-3 / dx, 0.5 * n)
    ay, ax = min(4e-3 / dx, n / 8), min(2e-3 / dx, n / 16)
    inside = ((yy - (row + depth)) / ay) ** 2 + ((xx - n // 2) / ax) ** 2 <= 1.0
    c = np.where(inside, 1450.0, 1500.0)
    beta = np.where(inside, 5.0, 3.5)
    rho = np.full((n, n), 1000.0)
    alpha = np.full((n, n), db_cm_mhz_to_np_m(0.0022, f, ypow))
    n_el = min(64, max(4, n // 32))
    ix, iy = line_array(n, n_el, 4, row)
    amp = np.ones((1, n_el), np.complex64)
    return Workload("cfg3_nonlinear_%d" % n, n, dx, f, c0, _f32(c), _f32(alpha), ypow, f,
                    ix, iy, amp, max_terms, tol,
                    extras=dict(beta=_f32(beta), rho=_f32(rho), a_db=0.0022,
                                surface_pressure=5e5))


def cfg3_harmonic_alpha(w: Workload) -> np.ndarray:
    """Absorption at the second harmonic: alpha(2f) = 2^y alpha(f)."""
    return _f32(w.alpha.astype(np.float64) * 2.0 ** w.ypow)


def cfg4_frequencies(n_freq: int = 64):
    """The sweep's frequencies f_k = 2 + 6k/(n_freq-1) MHz."""
    return [2e6 + 6e6 * k / max(1, n_freq - 1) for k in range(n_freq)]


def cfg4_grid_sizes(scale: float = 1.0, n_freq: int = 64):
    """N of each frequency's grid (lambda/8 over the fixed 48 mm domain),
    without building the media: the same N as cfg4_list."""
    c0 = 1500.0
    return [int(round(48e-3 * scale / (c0 / f / 8.0))) for f in cfg4_frequencies(n_freq)]


def cfg4_list(scale: float = 1.0, n_freq: int = 64, n_ang: int = 8):
    """Broadband sweep: f_k = 2 + 6k/(n_freq-1) MHz, 8 steering angles in
    [-30, 30] deg, Gaussian spectral weight exp(-((f-5 MHz)/1.5 MHz)^2), the
    cfg1 medium at a fixed 48 mm x 48 mm (disk r 7.5 mm, 1530 m/s) on a
    lambda/8 grid per frequency (N = round(256 f/MHz) * scale); 24 terms.
    Returns one Workload per frequency with n_rhs = n_ang."""
    out = []
    c0 = 1500.0
    side = 48e-3 * scale
    thetas = np.deg2rad(np.linspace(-30.0, 30.0, n_ang))
    for k, f in enumerate(cfg4_frequencies(n_freq)):
        dx = c0 / f / 8.0
        n = int(round(side / dx))
        yy, xx = np.mgrid[0:n, 0:n]
        x = xx * dx
        y = yy * dx
        inside = (x - 24e-3 * scale) ** 2 + (y - 24e-3 * scale) ** 2 <= (7.5e-3 * scale) ** 2
        c = np.where(inside, 1530.0, c0)
        xel = (112 + np.arange(32)) * (0.1875e-3) * scale
        ix = np.round(xel / dx).astype(np.int32)
        iy = np.full(32, int(round(3e-3 * scale / dx)), np.int32)
        ix = np.clip(ix, 0, n - 1)
        iy = np.clip(iy, 0, n - 1)
        k0 = 2 * math.pi * f / c0
        wgt = math.exp(-(((f - 5e6) / 1.5e6) ** 2))
        centre = (xel[0] + xel[-1]) / 2.0 / dx
        amp = np.stack([wgt * steer_amplitudes(ix, dx, k0, th, centre) for th in thetas])
        out.append(Workload("cfg4_f%02d_%d" % (k, n), n, dx, f, c0, _f32(c), None, 1.0, f,
                            ix, iy, amp.astype(np.complex64), 24, 0.0,
                            extras=dict(thetas=thetas, weight=wgt)))
    return out


@dataclasses.dataclass
class PeriodicCase:
    """The paper's own periodic-grid run (Section 3.1, Algorithm 1)."""
    n: int
    dx: float
    f: float
    c0: float
    c: np.ndarray               # float32 [N, N] sound speed
    ix: np.ndarray              # int32 [P] source columns
    iy: np.ndarray              # int32 [P] source rows
    amp: np.ndarray             # complex64 [1, P]: a dx^2 (the plans deposit a / dx^2 per cell)
    tol: float                  # Eq. 30 threshold
    l1_row: int                 # Eq. 30 row (0-based)
    eps_factor: float
    abl_width: int
    abl_zeta: float


def paper_periodic_case(params: dict, scatterer_speed: float | None = None) -> PeriodicCase:
    """Section 3.1's geometry from its printed parameters (``params``: the
    name -> {"value": ...} table of the paper's numbers): an N x N periodic
    grid, the 501-element line source on one column around the centre row
    with amplitude a per element, the sigmoid layer and Eq. 30 on the
    centre row; with ``scatterer_speed`` the cylinder of the inhomogeneous
    case (radius a, centred on the array's axis at the printed offset)."""
    v = lambda k: params[k]["value"]
    n, dx, c0 = v("grid_n"), v("dx_m"), v("v_f")
    row = v("source_row_1based") - 1
    half = (v("n_elements") - 1) // 2
    iy = np.arange(row - half, row + half + 1, dtype=np.int32)
    ix = np.full_like(iy, v("source_column"))
    amp = np.full((1, iy.size), complex(*v("source_amplitude")) * dx * dx, np.complex64)
    c = np.full((n, n), c0, np.float32)
    if scatterer_speed is not None:
        r = v("scatterer_radius_m") / dx
        cx = v("source_column") + v("scatterer_offset_m") / dx
        yy, xx = np.mgrid[0:n, 0:n]
        c[(xx - cx) ** 2 + (yy - row) ** 2 <= r * r] = scatterer_speed
    return PeriodicCase(n, dx, v("f_hz"), c0, c, ix, iy, amp, v("stop_tol"), row, v("eps_factor"),
                        v("abl_width_cells"), v("abl_zeta_np_per_m"))


def cfg5(n: int = 1024, n_src: int = 16, terms: int | None = None, true_model: bool = False) -> Workload:
    """Gradient workload at 3 MHz, N = 1024, c0 = 1540, alpha as cfg2:
    16 point sources on row 24 at columns 32 + 64 j, receivers on row 1000.
    The true model adds two +-3% Gaussian blobs (sigma 3 mm); the start model
    is homogeneous.  ``terms`` fixes the number of terms (None: to 1e-6)."""
    f, c0, ypow = 3e6, 1540.0, 1.1
    dx = c0 / f / 8.0
    s = n / 1024.0
    c = np.full((n, n), c0)
    if true_model:
        sig = 3e-3 / dx * s
        yy, xx = np.mgrid[0:n, 0:n]
        b1 = np.exp(-((yy - 400 * s) ** 2 + (xx - 400 * s) ** 2) / (2 * sig * sig))
        b2 = np.exp(-((yy - 600 * s) ** 2 + (xx - 620 * s) ** 2) / (2 * sig * sig))
        c = c0 * (1.0 + 0.03 * b1 - 0.03 * b2)
    alpha = np.full((n, n), db_cm_mhz_to_np_m(0.5, f, ypow))
    ix = np.round((32 + 64 * np.arange(n_src)) * s).astype(np.int32)
    iy = np.full(n_src, int(round(24 * s)), np.int32)
    # one source configuration per right-hand side: element j only in rhs j
    amp = np.eye(n_src, dtype=np.complex64)
    rrow = min(n - 1, int(round(1000 * s)))
    return Workload("cfg5_gradient_%d" % n, n, dx, f, c0, _f32(c), _f32(alpha), ypow, f,
                    ix, iy, amp, terms if terms else 64, 0.0 if terms else 1e-6,
                    extras=dict(receiver_row=rrow))


def random_medium(n: int, seed: int, f: float = 1e6, c0: float = 1500.0, contrast: float = 0.02,
                  absorbing: bool = True, n_rhs: int = 1, n_pts: int = 4):
    """Small generic case for tests: smooth random c, optional absorption,
    a few random point sources with random complex amplitudes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = c0 / f / 8.0
    delta = gaussian_random_field(n, max(2.0, n / 8.0), contrast, seed + 1)
    c = c0 * (1.0 + delta)
    alpha = np.full((n, n), 20.0) * (1.0 + 0.5 * rng.random((n, n))) if absorbing else None
    ix = rng.integers(0, n, n_pts).astype(np.int32)
    iy = rng.integers(0, n, n_pts).astype(np.int32)
    amp = (rng.standard_normal((n_rhs, n_pts)) + 1j * rng.standard_normal((n_rhs, n_pts)))
    return Workload("random_%d_s%d" % (n, seed), n, dx, f, c0, _f32(c),
                    None if alpha is None else _f32(alpha), 1.5, f, ix, iy,
                    amp.astype(np.complex64), 64, 1e-6)
