"""Batched graph solves (broadband sweep) and the plain cuFFT baseline."""
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


def _plan_for(w):
    import torch
    from paper_2507_13754_gb300 import tbs
    p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=w.max_terms, tol=w.tol)
    p.set_medium(torch.from_numpy(w.c).cuda(), None, w.ypow, w.f_ref)
    p.set_sources(w.src_ix, w.src_iy, w.src_amp)
    return p


def test_batch_equals_individual_solves_and_oracle():
    """Broadband sweep at quarter scale: 6 frequencies (N 128..512, three
    padded sizes) x 8 steering angles in one graph launch."""
    from paper_2507_13754_gb300 import tbs, workloads as W
    ws = W.cfg4_list(scale=0.25, n_freq=6, n_ang=8)
    plans = [_plan_for(w) for w in ws]
    assert len({p.m for p in plans}) >= 2
    batch = tbs.Batch(plans)
    batch.solve()
    import torch
    torch.cuda.synchronize()
    binfo = batch.infos()
    for w, p, psi_b, inf_b in zip(ws, plans, batch.psi, binfo):
        psi_i, inf_i = p.solve()
        assert np.array_equal(psi_b.cpu().numpy(), psi_i.cpu().numpy()), w.name
        assert [i["terms"] for i in inf_b] == [i["terms"] for i in p.info_dicts(inf_i)] == [24] * 8
    # oracle on a subset: lowest and highest frequency, two angles each
    for k, r in [(0, 0), (0, 7), (len(ws) - 1, 3), (len(ws) - 1, 4)]:
        w = ws[k]
        (ref, _, _, _), = oracle_solve(w, rhs=[r])
        assert rel_l2(batch.psi[k][r].cpu().numpy(), ref) < PARITY_RTOL, (w.name, r)
    batch.close()
    for p in plans:
        p.close()


def test_sharded_sweep_matches_the_single_batch():
    """Independent solves split over ranks (shard.rank_solves, cost M^2 x
    terms), each rank's share run as its own batch of plans holding only the
    angles it owns: every field equals, bit for bit, the same field of the
    whole sweep in one batch.  The three ranks run one after the other on this
    GPU (they exchange nothing while solving)."""
    import math
    import torch
    from paper_2507_13754_gb300 import shard, tbs, workloads as W
    ws = W.cfg4_list(scale=0.25, n_freq=6, n_ang=8)
    fixed = dict(max_terms=24, tol=0.0, div_window=1 << 30, div_factor=math.inf)

    def plans_for(parts):
        out = []
        for k, rhs in parts:
            w = ws[k]
            p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=len(rhs), **fixed)
            p.set_medium(torch.from_numpy(w.c).cuda(), None, w.ypow, w.f_ref)
            p.set_sources(w.src_ix, w.src_iy, w.src_amp[rhs])
            out.append(p)
        return out

    full = plans_for([(k, list(range(w.n_rhs))) for k, w in enumerate(ws)])
    whole = tbs.Batch(full)
    whole.solve()
    torch.cuda.synchronize()
    world, seen = 3, []
    for rank in range(world):
        mine = sorted(shard.rank_solves(ws, world, rank, terms=24).items())
        if not mine:
            continue
        plans = plans_for(mine)
        batch = tbs.Batch(plans)
        batch.solve()
        torch.cuda.synchronize()
        for (k, rhs), psi in zip(mine, batch.psi):
            for j, r in enumerate(rhs):
                assert np.array_equal(psi[j].cpu().numpy(), whole.psi[k][r].cpu().numpy()), (rank, k, r)
                seen.append((k, r))
        batch.close()
        for p in plans:
            p.close()
    # every solve ran on exactly one rank
    assert sorted(seen) == [(k, r) for k, w in enumerate(ws) for r in range(w.n_rhs)]
    whole.close()
    for p in full:
        p.close()


@pytest.mark.slow
def test_cfg4_full_scale_subset_in_one_batch():
    """Full-scale broadband sweep, a seeded subset of 16 solves: 7 of the 64
    frequencies (2 .. 8 MHz; N 512 .. 2048; all three padded sizes M = 1024,
    2048, 4096), each of the 8 steering angles twice, the 7 plans (all 8
    angles each) in one batch graph, divergence rule off, every field at the
    sweep's 24 terms.  Above ~4 MHz the fixed disk makes the terms grow
    before they decay, so the FP32 partial sum carries a cancellation error
    that scales with kappa = max_n |u_n| / |psi|: each field's kappa and
    relative L2 error are printed, and the 2e-5 bar is asserted wherever
    kappa <= 10 (the range where FP32 can hold it)."""
    import math
    import oracle
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    ws = W.cfg4_list()
    picks = [(0, 24, [0, 3, 7]), (3, 24, [2, 5]), (21, 24, [1, 6]), (30, 24, [0, 4]), (42, 24, [2, 5]),
             (52, 24, [3, 7]), (63, 24, [1, 4, 6])]
    assert sum(len(r) for _, _, r in picks) == 16
    assert sorted(a for _, _, r in picks for a in r) == sorted(list(range(8)) * 2)
    nodiv = dict(div_window=1 << 30, div_factor=math.inf)
    plans = []
    for k, terms, _ in picks:
        w = ws[k]
        p = tbs.Plan(w.n, w.dx, w.f, w.c0, n_rhs=w.n_rhs, max_terms=terms, tol=0.0, **nodiv)
        p.set_medium(torch.from_numpy(w.c).cuda(), None, w.ypow, w.f_ref)
        p.set_sources(w.src_ix, w.src_iy, w.src_amp)
        plans.append(p)
    assert sorted({p.m for p in plans}) == [1024, 2048, 4096]
    batch = tbs.Batch(plans)
    batch.solve()
    torch.cuda.synchronize()
    infos = batch.infos()
    for (k, terms, rhs), psi_b, inf_b in zip(picks, batch.psi, infos):
        w = ws[k]
        assert [i["terms"] for i in inf_b] == [terms] * w.n_rhs
        assert all(i["status_name"] == "MAX_TERMS" for i in inf_b)
        m, gh = oracle.plan(w.n, w.dx, w.f, w.c0)
        V = oracle.potential(w.f, w.c0, w.c.astype(np.float64), None, w.ypow, w.f_ref)
        for r in rhs:
            s = oracle.deposit_points(w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[r].astype(np.complex128))
            ref, rinfo, norms, _ = oracle.solve(w.n, m, gh, V, s, terms, 0.0, **nodiv)
            kappa = max(norms) / rinfo["psi_norm"]
            err = rel_l2(psi_b[r].cpu().numpy(), ref)
            print("cfg4 %s M=%d angle %d: kappa %.2f rel L2 %.2e" % (w.name, m, r, kappa, err))
            if kappa <= 10.0:
                assert err < PARITY_RTOL, (w.name, r, kappa, err)
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_host_info_and_repeats():
    import ctypes as C
    import torch
    from paper_2507_13754_gb300 import tbs, workloads as W
    w = W.random_medium(32, seed=41)
    p = _plan_for(w)
    psi = torch.empty((1, 32, 32), dtype=torch.complex64, device="cuda")
    host_info = (tbs.tbs_solve_info * 1)()
    with pytest.raises(tbs.TbsError):
        tbs.tbs_batch_create([p.handle], [psi.data_ptr()], [C.addressof(host_info)])
    dinfo = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(tbs.TbsError):
        tbs.tbs_batch_create([p.handle, p.handle], [psi.data_ptr()] * 2, [dinfo.data_ptr()] * 2)
    p.close()


def test_cufft_baseline_computes_the_same_series():
    import torch
    from paper_2507_13754_gb300 import baseline_cufft as B, workloads as W
    w = W.cfg1()
    p = _plan_for(w)
    psi, _ = p.solve()
    base = B.CufftBornSeries(w.n, p.m, B.full_spectrum(p.ghat_quadrant(), p.m))
    V = B.potential(w.f, w.c0, torch.from_numpy(w.c).cuda())
    S = B.dense_source(w.n, w.dx, w.src_ix, w.src_iy, w.src_amp[0])
    psi_b, _ = base.solve_fixed(V, S, 24)
    assert rel_l2(psi_b.cpu().numpy(), psi[0].cpu().numpy()) < PARITY_RTOL
    p.close()
