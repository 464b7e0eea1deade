"""The oracle's pins must catch plausible mistakes: each case below plants
one in a copy of the C oracle (on the CPU, in a temporary directory), loads
that copy in place of the real one and checks that at least one of the
pins it names fails.  The real oracle is restored afterwards."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

import test_oracle_pins as pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "tbs_oracle.c")

# (name, original text, planted text, pins that must notice)
MUTATIONS = [
    ("Y0 sign in the Green's function", "*re = -0.25 * y;", "*re = 0.25 * y;",
     [pins.test_green_point_matches_scipy_hankel]),
    ("dropped dx^2 in the spectrum scale", "double s = dx * dx / ((double)m * (double)m);",
     "double s = 1.0 / ((double)m * (double)m);",
     [lambda o: pins.test_convolution_matches_direct_sum(o, 12, 32)]),
    ("conjugated V in the series", "vu[i] = V[i] * u[i];", "vu[i] = conj(V[i]) * u[i];",
     [pins.test_converged_series_matches_dense_solve, pins.test_truncated_series_matches_matrix_powers]),
    ("sign of the dispersion term", "return tan(M_PI * ypow / 2.0) * delta;",
     "return -tan(M_PI * ypow / 2.0) * delta;",
     [pins.test_potential_satisfies_paper_dispersion_relation]),
    ("unconjugated V in the adjoint", "ubar[i] = g[i] + conj(V[i]) * lam[i];",
     "ubar[i] = g[i] + V[i] * lam[i];",
     [pins.test_adjoint_dot_product, pins.test_truncated_adjoint_converges_to_dense_adjoint]),
    ("no one-half on the squared harmonic", "acc += (a == b ? 0.5 : 1.0) * pa * pb;",
     "acc += pa * pb;",
     [lambda o: pins.test_harmonic_sum_term_sources_from_nonlinear_wave_equation(o, 2),
      lambda o: pins.test_harmonic_sum_term_sources_from_nonlinear_wave_equation(o, 4)]),
    ("source not divided by dx^2", "s[(size_t)iy[j] * n + ix[j]] += amp[j] / (dx * dx);",
     "s[(size_t)iy[j] * n + ix[j]] += amp[j];",
     [lambda o: pins.test_homogeneous_field_is_hankel_superposition(o, 0.25)]),
    ("layer on one axis only", "for (long x = 0; x < n; x++) w[y * n + x] *= abl[y] * abl[x];\n        double num",
     "for (long x = 0; x < n; x++) w[y * n + x] *= abl[x];\n        double num",
     [pins.test_eps_iteration_fixed_point_with_layer]),
    ("sign of the preconditioner", "const cplx gamma = I * V[i] / eps;", "const cplx gamma = -I * V[i] / eps;",
     [pins.test_cbs_iteration_converges_where_the_plain_one_diverges]),
    ("sign of i eps in the shifted spectrum", "inv / (px * px + py * py - k0 * k0 - I * eps);",
     "inv / (px * px + py * py - k0 * k0 + I * eps);",
     [pins.test_eps_green_impulse_response_is_lossy_hankel,
      pins.test_eps_iteration_without_layer_solves_periodic_helmholtz]),
    ("sign of the layer's sigmoid", "exp(-zeta * (e * dx - 0.5 * mu))", "exp(zeta * (e * dx - 0.5 * mu))",
     [pins.test_abl_profile_is_the_sigmoid]),
    ("sign of eta in the k-space potential", "vv[(size_t)j * n + i] = eta * pow(p, nu + 1.0) - I *",
     "vv[(size_t)j * n + i] = -eta * pow(p, nu + 1.0) - I *",
     [pins.test_kspace_potential_matches_paper_tau_eta, pins.test_kspace_iteration_without_layer_has_closed_form]),
    ("source dropped from the k-space update", "w[i] = gh[i] * (vv[i] * w[i] + sh[i]);",
     "w[i] = gh[i] * (vv[i] * w[i]);",
     [pins.test_kspace_iteration_without_layer_has_closed_form]),
    ("harmonic frequency omega instead of n omega", "const double wn = order * omega;",
     "const double wn = omega;",
     [lambda o: pins.test_harmonic_sum_term_sources_from_nonlinear_wave_equation(o, 3)]),
    ("time convention of the synthesis", "o[j] += w[k] * val * cexp(-2.0 * M_PI * I * f[k] * t);",
     "o[j] += w[k] * val * cexp(2.0 * M_PI * I * f[k] * t);",
     [pins.test_synthesis_on_a_frequency_comb_is_the_dft]),
]


def _build_variant(text, tmp):
    src = os.path.join(tmp, "mutant.c")
    lib = os.path.join(tmp, "libmutant.so")
    with open(src, "w") as f:
        f.write(text)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", lib, "-lm"]
    if subprocess.run(base[:4] + ["-fopenmp"] + base[4:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return lib


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed to build the planted copies")
@pytest.mark.parametrize("name,orig,planted,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(oracle_mod, tmp_path, name, orig, planted, checks):
    text = open(SRC).read()
    assert text.count(orig) >= 1, "the planted site moved: %s" % name
    mutant = text.replace(orig, planted, 1)
    lib = oracle_mod._bind(C.CDLL(_build_variant(mutant, str(tmp_path))))
    saved = oracle_mod._load()
    failed = []
    try:
        oracle_mod._lib = lib
        for check in checks:
            try:
                check(oracle_mod)
            except (AssertionError, ValueError, FloatingPointError):
                failed.append(check)
    finally:
        oracle_mod._lib = saved
    assert failed, "no pin noticed: %s" % name
    # and the real oracle still passes them
    for check in checks:
        check(oracle_mod)
