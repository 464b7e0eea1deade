"""Broadband synthesis on the GPU (tbs_synthesize): the time signal
s(X, t) = sum_k w_k psi_k(X) exp(-2 pi i f_k t) at receiver lattices, from
fields on different grids, against the oracle's plain sum."""
import numpy as np
import pytest

from _helpers import PARITY_RTOL, library, oracle_solve, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    library()


def test_synthesis_matches_oracle_on_random_fields():
    """70 frequencies (two launches of the 64-frequency chunk), grids of 2 to
    40 cells over the same 6 mm, three right-hand sides, a 13 x 5 receiver
    lattice that reaches outside every grid (clamped samples), 300 time
    samples starting 2.5 ms in (f t up to 2e4 cycles)."""
    import torch
    import oracle
    from paper_2507_13754_gb300 import tbs
    rng = np.random.default_rng(11)
    K, n_rhs, L = 70, 3, 6e-3
    ns = rng.integers(2, 41, K)
    dxs = L / ns
    freqs = rng.uniform(1e6, 8e6, K)
    w = rng.uniform(0.2, 1.0, K)
    fields = [(rng.standard_normal((n_rhs, n, n)) + 1j * rng.standard_normal((n_rhs, n, n))).astype(np.complex64)
              for n in ns]
    origin, step, counts = (-0.4e-3, 0.3e-3), (0.55e-3, 1.45e-3), (13, 5)
    t0, dt, nt = 2.5e-3, 1.3e-8, 300
    dev = [torch.from_numpy(f).cuda() for f in fields]
    s = tbs.synthesize(dev, dxs, freqs, w, origin, step, counts, t0, dt, nt).cpu().numpy()
    ref = oracle.synthesize([f.astype(np.complex128) for f in fields], dxs, freqs, w, origin, step, counts,
                            t0, dt, nt)
    assert s.shape == ref.shape == (n_rhs, 5, 13, nt)
    assert rel_l2(s, ref) < PARITY_RTOL, rel_l2(s, ref)
    # one receiver, one sample: a single launch of a one-block grid
    s1 = tbs.synthesize(dev[:3], dxs[:3], freqs[:3], w[:3], (1e-3, 2e-3), (0, 0), (1, 1), 0.0, 1e-8, 1)
    r1 = oracle.synthesize([f.astype(np.complex128) for f in fields[:3]], dxs[:3], freqs[:3], w[:3], (1e-3, 2e-3),
                           (0, 0), (1, 1), 0.0, 1e-8, 1)
    assert rel_l2(s1.cpu().numpy(), r1) < PARITY_RTOL


def test_synthesis_rejects_bad_arguments():
    import torch
    from paper_2507_13754_gb300 import tbs
    f = torch.zeros((1, 4, 4), dtype=torch.complex64, device="cuda")
    one = torch.zeros((1, 1, 1), dtype=torch.complex64, device="cuda")
    with pytest.raises(tbs.TbsError):  # a grid of one cell has no neighbour to interpolate with
        tbs.synthesize([one], [1e-4], [1e6], [1.0], (0, 0), (0, 0), (1, 1), 0.0, 1e-8, 4)
    with pytest.raises(tbs.TbsError):
        tbs.synthesize([f], [0.0], [1e6], [1.0], (0, 0), (0, 0), (1, 1), 0.0, 1e-8, 4)
    with pytest.raises(tbs.TbsError):
        tbs.synthesize([f], [1e-4], [float("nan")], [1.0], (0, 0), (0, 0), (1, 1), 0.0, 1e-8, 4)
    out = torch.zeros((1, 1, 1, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(tbs.TbsError):  # out aliasing a field
        tbs.tbs_synthesize([(out.data_ptr(), 2, 1e-4, 1e6, 1.0)], 1, 0, 0, 0, 0, 1, 1, 0.0, 1e-8, 4,
                           out.data_ptr())


def test_broadband_sweep_time_signal_matches_oracle():
    """The sweep end to end at quarter scale: 4 frequencies of the broadband
    workload (2, 4, 6, 8 MHz; N 128 .. 512 over the same 12 mm), 2 steering
    angles, solved as one batch, then the time signal on a 64-receiver line
    at 9 mm depth, 128 samples over one period of the comb; the oracle
    solves each field itself and sums."""
    import torch
    import oracle
    from paper_2507_13754_gb300 import tbs, workloads as W
    ws = W.cfg4_list(scale=0.25, n_freq=4, n_ang=2)
    plans = []
    for w in ws:
        p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=w.max_terms, tol=w.tol)
        p.set_medium(torch.from_numpy(w.c).cuda(), None, w.ypow, w.f_ref)
        p.set_sources(w.src_ix, w.src_iy, w.src_amp)
        plans.append(p)
    batch = tbs.Batch(plans)
    batch.solve()
    side = ws[0].n * ws[0].dx
    df = ws[1].f - ws[0].f
    origin, step, counts = (0.0, 0.75 * side), (side / 63, 0.0), (64, 1)
    nt = 128
    dt = 1.0 / df / nt
    dxs = [w.dx for w in ws]
    freqs = [w.f for w in ws]
    wts = [df] * len(ws)
    s = tbs.synthesize(batch.psi, dxs, freqs, wts, origin, step, counts, 0.0, dt, nt).cpu().numpy()
    refs = [np.stack([o[0] for o in oracle_solve(w)]) for w in ws]
    ref = oracle.synthesize(refs, dxs, freqs, wts, origin, step, counts, 0.0, dt, nt)
    assert rel_l2(s, ref) < PARITY_RTOL, rel_l2(s, ref)
    # the signal is the sweep's, not noise: the angles differ
    assert rel_l2(ref[0], ref[1]) > 0.1
    batch.close()
    for p in plans:
        p.close()
