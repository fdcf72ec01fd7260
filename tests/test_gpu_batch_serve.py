"""Batched solves, the serving loop and the work-tile autotuner on the GPU.

A job's result must be the same whether it runs alone or among others
(within 1e-6 in the subspace angle wherever the stopping criterion fixes
the subspace to that), and the
host-side failure paths (over-budget submission, cancellation, a bad job
among good ones) must not disturb the rest."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _bk():
    import paper_2012_07595_gb300 as bk
    from paper_2012_07595_gb300 import _build
    _build.build()
    return bk


def _jobs(count, seed=4):
    jobs = synth.batch_jobs(seed=seed, count=count, scale=0.02)
    return [(j, synth.job_tensor(j)) for j in jobs]


def _params(bk, r, prec):
    return bk.BksParams(r1=r, r3=r, stages=2, block_p=4, tol=1e-9, tol_scale_free=1,
                        precision=prec, mixed_tol=1e-6, refine_sweeps=50, max_outer=300)


def _sin(a, b):
    return O.sin_theta_max(np.asarray(a), np.asarray(b))


def _angle_bound(F, mode, tol=1e-9):
    """How far the stopping criterion fixes a factor's subspace.  Turning
    the mode's last column by an angle t changes ||F||^2 by about
    sigma^2 t^2, sigma the mode's last S-value (Section 2.6), so a point
    whose gradient is at most tol ||F||^2 (Section 2.5) lies within an
    angle of about tol ||F||^2 / sigma^2 of the maximiser.  With a zero or
    tiny S-value the subspace is not fixed and two correct runs may differ
    there."""
    sv = O.s_values(np.asarray(F))[mode]
    return tol * float((sv ** 2).sum()) / max(float(sv[-1]) ** 2, 1e-300)


def _oracle_check(c, U, W, F, normF, tol):
    """Properties the oracle evaluates at a returned point (Algorithm 5's
    result): orthonormal U and W, F = A.(U,U,W) (eq. (Rayleigh)) and
    ||F|| as reported, F symmetric in its first two modes, ||F|| <= ||A||,
    and the scale-free G-gradient (Section 2.5) within twice the
    tolerance."""
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    U, W, F = np.asarray(U), np.asarray(W), np.asarray(F)
    r1, r3 = U.shape[1], W.shape[1]
    assert np.abs(U.T @ U - np.eye(r1)).max() < 1e-12
    assert np.abs(W.T @ W - np.eye(r3)).max() < 1e-12
    gg, nf, Fo = O.gradient_global(A, U, W)
    assert abs(nf - normF) <= 1e-10 * nf
    assert np.allclose(F, Fo, rtol=0, atol=1e-10 * nf)
    assert np.allclose(Fo, Fo.transpose(1, 0, 2), rtol=0, atol=1e-12 * nf)
    assert nf ** 2 <= A.fro2() * (1 + 1e-12)
    assert gg / nf ** 2 <= 2 * tol, (gg / nf ** 2, tol)


def _same_solution(a, b, Fa):
    assert abs(a["normF"] - b["normF"]) <= 1e-9 * a["normF"]
    for key, mode in (("U", 0), ("W", 2)):
        bound = _angle_bound(Fa, mode)
        if bound <= 1e-4:
            assert _sin(a[key], b[key]) < max(1e-6, 10 * bound), (key, bound)


def test_autotune_keeps_results():
    import torch
    bk = _bk()
    c = synth.zipf_tensor(8, 30_000, 40, 400_000, 1.1)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    g = synth.rng(1)
    X = torch.tensor(g.standard_normal((c.m, 4)), device="cuda")
    Y = torch.tensor(g.standard_normal((c.n, 3)), device="cuda")
    before = bk.bks_contract_mode1(T, X, Y).cpu().numpy()
    tile, split = bk.bks_tensor_autotune(T)
    assert (tile, split) in {(8, 512), (16, 512), (64, 1024), (128, 2048), (32, 512)}
    after = bk.bks_contract_mode1(T, X, Y).cpu().numpy()
    assert np.abs(after - before).max() <= 1e-12 * max(1.0, np.abs(before).max())
    # every row on a warp; long rows cut into many pieces; all but the
    # longest rows on single lanes
    for tl, sp in [(1, 128), (16, 128), (64, 4096), (128, 2048)]:
        bk.bks_tensor_set_tiles(T, tl, sp)
        got = bk.bks_contract_mode1(T, X, Y).cpu().numpy()
        assert np.abs(got - before).max() <= 1e-12 * max(1.0, np.abs(before).max())
        tri = bk.bks_contract_mode3(T, X).cpu().numpy()
        A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
        ref = O.mode3(A, X.cpu().numpy())
        assert np.abs(tri - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    with pytest.raises(bk.BksError):
        bk.bks_tensor_set_tiles(T, 8, 8)
    with pytest.raises(bk.BksError):
        bk.bks_tensor_set_tiles(T, 129, 1024)


def test_batch_matches_solo():
    bk = _bk()
    jobs = _jobs(10)
    tens, params = [], []
    for j, c in jobs:
        tens.append(bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v))
        params.append(_params(bk, j["r"], bk.BKS_PREC_MIXED))
    res = bk.bks_batch_solve(tens, params, nstreams=4, autotune=True)
    for q, (T, p) in enumerate(zip(tens, params)):
        U, W, F, info, st = res[q]
        assert st in (bk.BKS_OK,), (q, st)
        _oracle_check(jobs[q][1], U.cpu().numpy(), W.cpu().numpy(), F.cpu().numpy(),
                      info["normF"], p.tol)
        Us, Ws, Fs, infos = bk.bks_solve(T, p)
        _same_solution({"U": Us.cpu().numpy(), "W": Ws.cpu().numpy(), "normF": infos["normF"]},
                       {"U": U.cpu().numpy(), "W": W.cpu().numpy(), "normF": info["normF"]},
                       Fs.cpu().numpy())


def test_server_alone_equals_in_mix_and_failure_paths():
    bk = _bk()
    jobs = _jobs(12, seed=7)
    budget = 8 << 30
    # alone: one slot, one job at a time
    alone = []
    with bk.Server(budget, max_slots=1) as srv:
        for j, c in jobs[:4]:
            t = srv.submit(c.m, c.n, c.i, c.j, c.k, c.v, _params(bk, j["r"], bk.BKS_PREC_MIXED))
            alone.append(srv.poll(t, wait=True))
    with bk.Server(budget, max_slots=4) as srv:
        tickets = [srv.submit(c.m, c.n, c.i, c.j, c.k, c.v,
                              _params(bk, j["r"], bk.BKS_PREC_MIXED)) for j, c in jobs]
        # a bad job (index out of range) in the middle of the stream
        bad = srv.submit(10, 3, np.array([11]), np.array([0]), np.array([0]), np.array([1.0]),
                         _params(bk, 2, bk.BKS_PREC_MIXED))
        # an over-budget job is refused at submission
        with pytest.raises(bk.BksError) as e:
            srv.submit(10_000_000, 100, np.zeros(1), np.zeros(1), np.zeros(1), np.ones(1),
                       _params(bk, 2, bk.BKS_PREC_MIXED))
        assert e.value.code == bk.BKS_EBUDGET
        out = [srv.poll(t, wait=True) for t in tickets]
        rb = srv.poll(bad, wait=True)
        assert rb["status"] == bk.BKS_EINVAL
        for (j, c), r in zip(jobs, out):
            assert r["status"] == bk.BKS_OK, r["error"]
            assert r["latency_s"] > 0
            _oracle_check(c, r["U"], r["W"], r["F"], r["normF"], 1e-9)
        for a, b in zip(alone, out[:4]):
            _same_solution(a, b, a["F"])
        assert srv.stats()["running"] == 0


def test_server_cancel_queued_job():
    bk = _bk()
    jobs = _jobs(6, seed=9)
    with bk.Server(8 << 30, max_slots=1) as srv:
        t = [srv.submit(c.m, c.n, c.i, c.j, c.k, c.v, _params(bk, j["r"], bk.BKS_PREC_FP64))
             for j, c in jobs]
        srv.cancel(t[-1])           # still queued behind the others: removed
        last = srv.poll(t[-1], wait=True)
        assert last["status"] == bk.BKS_ECANCELED
        for x in t[:-1]:
            assert srv.poll(x, wait=True)["status"] == bk.BKS_OK
