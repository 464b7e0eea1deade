"""The FFT engine's R-point butterflies on the host, against the DFT definition.

The engine (csrc/tbs_fft.cuh) writes each Stockham butterfly as layers of
two-point butterflies in FMA form with the stage twiddle W^r folded in.  Its
butterfly functions are host-callable, so this test compiles a small host
program with nvcc (no GPU needed) that runs every radix (2, 4, 8, 16), both
directions, the first-stage form (W = 1, optionally with the upper half of
the inputs zero) and the twiddled form, and compares each output with
X[k] = sum_r x[r] W^r exp(DIR 2 pi i r k / R) evaluated in complex128 here.
A wrong twiddle index, a swapped output or a wrong sign fails it.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_13754_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include "tbs_fft.cuh"
using namespace tbs;
static const int M = 4096;
static float2 tab[M];
template <int R, int DIR, bool TW, bool ZIN>
static void run(int e, const float2 *x) {
    TwSet<R> s{};
    if (TW) {
        // the table entries the engine's loader reads for stage twiddle tw[e]
        if (R == 2) s.p[0] = tab[e];
        if (R == 4) { s.u1 = tab[e]; s.u2 = tab[2 * e]; }
        if (R == 8) { s.u1 = tab[2 * e]; s.u2 = tab[4 * e]; s.p[0] = tab[e]; s.p[1] = tab[e + M / 8]; }
        if (R == 16) {
            s.u1 = tab[4 * e]; s.u2 = tab[8 * e];
            for (int k = 0; k < 4; k++) s.p[k] = tab[e + k * (M / 16)];
            s.q[0] = tab[2 * e]; s.q[1] = tab[2 * e + M / 8];
        }
    }
    float2 v[R];
    for (int r = 0; r < R; r++) v[r] = (ZIN && r >= R / 2) ? make_float2(NAN, NAN) : x[r];
    butterfly<R, DIR, TW, ZIN>(v, s);
    printf("%d %d %d %d %d", R, DIR, (int)TW, (int)ZIN, e);
    for (int r = 0; r < R; r++) printf(" %.9e %.9e", v[r].x, v[r].y);
    printf("\n");
}
template <int R>
static void all(int e, const float2 *x) {
    run<R, -1, false, false>(0, x); run<R, +1, false, false>(0, x);
    run<R, -1, false, true>(0, x);  run<R, +1, false, true>(0, x);
    run<R, -1, true, false>(e, x);  run<R, +1, true, false>(e, x);
}
int main() {
    for (int k = 0; k < M; k++)
        tab[k] = make_float2((float)cos(-2.0 * M_PI * k / M), (float)sin(-2.0 * M_PI * k / M));
    float2 x[16];
    unsigned st = 12345u;
    for (int i = 0; i < 16; i++) {
        st = st * 1664525u + 1013904223u; float a = (st >> 8) / 16777216.0f - 0.5f;
        st = st * 1664525u + 1013904223u; float b = (st >> 8) / 16777216.0f - 0.5f;
        x[i] = make_float2(a, b);
    }
    // stage twiddle exponents e < M / R, as the engine's stages produce them
    const int es[3] = {1, 77, 255};
    for (int i = 0; i < 3; i++) {
        all<2>(es[i] * 8, x); all<4>(es[i] * 4, x); all<8>(es[i] * 2, x); all<16>(es[i], x);
    }
    // the harness's inputs, for the reference
    printf("X");
    for (int i = 0; i < 16; i++) printf(" %.9e %.9e", x[i].x, x[i].y);
    printf("\n");
    return 0;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_butterflies_match_the_dft_definition(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "harness.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    xs = [ln for ln in out if ln.startswith("X")][0].split()[1:]
    x = np.array([float(xs[2 * i]) + 1j * float(xs[2 * i + 1]) for i in range(16)])
    M = 4096
    n_checked = 0
    for ln in out:
        if ln.startswith("X"):
            continue
        f = ln.split()
        R, DIR, TW, ZIN, e = (int(v) for v in f[:5])
        got = np.array([float(f[5 + 2 * k]) + 1j * float(f[6 + 2 * k]) for k in range(R)])
        xr = x[:R].copy()
        if ZIN:
            xr[R // 2:] = 0
        W = np.exp(-2j * np.pi * e / M) if TW else 1.0
        if DIR > 0:
            W = np.conj(W)
        r = np.arange(R)
        ref = np.array([np.sum(xr * W ** r * np.exp(DIR * 2j * np.pi * r * k / R)) for k in range(R)])
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 3e-6, (R, DIR, TW, ZIN, e, err)
        n_checked += 1
    assert n_checked == 3 * 4 * 6
