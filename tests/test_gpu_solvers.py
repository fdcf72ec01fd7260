"""BKS (Algorithm 5) and HOOI on the GPU vs the oracle and closed forms."""
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


def _dense(bk, T):
    c = synth.dense_to_coo(T)
    A = O.symmetrise(T.shape[0], T.shape[2], c.i, c.j, c.k, c.v, mirror=False)
    return A, bk.bks_tensor_create_coo(A.m, A.n, A.i, A.j, A.k, A.v, mirror=False)


def _t(x):
    import torch
    return torch.tensor(np.asarray(x), device="cuda")


@pytest.mark.parametrize("solver", ["bks", "hooi"])
def test_closed_form_rank_one_slices(solver):
    bk = _bk()
    g = synth.rng(32)
    m = 20
    lam = np.concatenate([[9.0, -7.0], g.uniform(-1, 1, m - 2)])
    Q = np.linalg.qr(g.standard_normal((m, m)))[0]
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    c = np.array([1.0, -2.0, 0.5, 3.0])
    T = M[:, :, None] * c[None, None, :]
    A, TT = _dense(bk, T)
    U0 = synth.orthonormal(g, m, 2); W0 = synth.orthonormal(g, 4, 1)
    if solver == "bks":
        U, W, F, info = bk.bks_solve(TT, bk.BksParams(r1=2, r3=1, stages=2, block_p=2), _t(U0), _t(W0))
    else:
        U, W, F, info = bk.hooi_solve(TT, bk.HooiParams(r1=2, r3=1), _t(U0), _t(W0))
    assert info["converged"]
    want = np.sum(c ** 2) * (81.0 + 49.0)
    assert abs(info["normF"] ** 2 - want) < 1e-10 * want
    assert O.sin_theta_max(Q[:, :2], U.cpu().numpy()) < 1e-8
    assert O.sin_theta_max((c / np.linalg.norm(c))[:, None], W.cpu().numpy()) < 1e-8


def test_planted_exact_rank_recovered():
    bk = _bk()
    T, U0t, W0t, F0 = synth.dense_planted(41, m=40, n=12, r1=2, r3=2)
    A, TT = _dense(bk, T)
    g = synth.rng(7)
    U0 = synth.orthonormal(g, 40, 2); W0 = synth.orthonormal(g, 12, 2)
    U, W, F, info = bk.bks_solve(TT, bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-11), _t(U0), _t(W0))
    assert info["converged"]
    nA = np.sqrt(A.fro2())
    assert abs(info["normF"] - nA) < 1e-12 * nA
    assert O.sin_theta_max(U0t, U.cpu().numpy()) < 1e-10
    assert O.sin_theta_max(W0t, W.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("seed", [101, 102])
def test_small_planted_workload_parity(seed):
    """300x300x100, 10,000 draws + planted term, rank (2,2,2), BK(2,2),
    tol 1e-10, FP64: same start on both sides; ||F|| within 1e-10 relative
    and largest principal angles within 1e-8."""
    bk = _bk()
    coo, _ = synth.small_planted(1)
    A = O.symmetrise(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    g = synth.rng(seed)
    U0 = synth.orthonormal(g, A.m, 2); W0 = synth.orthonormal(g, A.n, 2)
    ro = O.bks(A, U0, W0, s=2, p=2, tol=1e-10)
    U, W, F, info = bk.bks_solve(T, bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-10), _t(U0), _t(W0))
    assert ro.converged and info["converged"]
    assert abs(info["normF"] - ro.normF) <= 1e-10 * ro.normF
    assert O.sin_theta_max(ro.U, U.cpu().numpy()) < 1e-8
    assert O.sin_theta_max(ro.W, W.cpu().numpy()) < 1e-8
    Fn = F.cpu().numpy()
    assert np.allclose(Fn, Fn.transpose(1, 0, 2), atol=1e-12 * np.linalg.norm(Fn))
    assert np.sum(Fn ** 2) <= A.fro2() * (1 + 1e-12)
    # the returned F is A.(U,U,W) at the returned point
    assert np.allclose(Fn, O.core(A, U.cpu().numpy(), W.cpu().numpy()), atol=1e-10 * np.linalg.norm(Fn))
    norms = [h[1] for h in info["history"]]
    assert all(b >= a * (1 - 1e-12) for a, b in zip(norms, norms[1:]))


@pytest.mark.parametrize("variant,s,p", [("min", 3, 2), ("max", 2, 2), ("bk", 3, 2)])
def test_schedule_variants_parity(variant, s, p):
    """min-BK (Algorithm 4, Table 1), max-BK (Table 2) and a 3-stage BK on
    the 300x300x100 planted workload, FP64, tol 1e-10: same start on both
    sides; same basis sizes, ||F|| within 1e-10 relative, subspaces within
    1e-8."""
    bk = _bk()
    coo, _ = synth.small_planted(1)
    A = O.symmetrise(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    g = synth.rng(103)
    U0 = synth.orthonormal(g, A.m, 2); W0 = synth.orthonormal(g, A.n, 2)
    ro = O.bks(A, U0, W0, s=s, p=p, tol=1e-10, variant=variant)
    code = {"bk": bk.BKS_VARIANT_BK, "min": bk.BKS_VARIANT_MIN, "max": bk.BKS_VARIANT_MAX}[variant]
    U, W, F, info = bk.bks_solve(T, bk.BksParams(r1=2, r3=2, stages=s, block_p=p, tol=1e-10,
                                                 variant=code), _t(U0), _t(W0))
    assert ro.converged and info["converged"]
    # basis sizes of the last expansion: the schedule's counts less the
    # columns dropped as dependent (max-BK drops some near convergence)
    want = O.schedule_counts(2, 2, s, p, variant, m=A.m, n=A.n)[-1]
    assert 2 < info["k1"] <= want[0] and 2 < info["k3"] <= want[1]
    assert abs(info["normF"] - ro.normF) <= 1e-10 * ro.normF
    assert O.sin_theta_max(ro.U, U.cpu().numpy()) < 1e-8
    assert O.sin_theta_max(ro.W, W.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("rho", [1e-2, 1e-3])
def test_example1_bks_hooi_agree_with_oracle(rho):
    bk = _bk()
    T = synth.example1(61, 30, 10, 2, 2, rho)
    A, TT = _dense(bk, T)
    g = synth.rng(62)
    U0 = synth.orthonormal(g, 30, 2); W0 = synth.orthonormal(g, 10, 2)
    rb = O.bks(A, U0, W0, s=2, p=2, tol=1e-11)
    Ub, Wb, Fb, ib = bk.bks_solve(TT, bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-11), _t(U0), _t(W0))
    Uh, Wh, Fh, ih = bk.hooi_solve(TT, bk.HooiParams(r1=2, r3=2, tol=1e-11), _t(U0), _t(W0))
    rh = O.hooi(A, U0, W0, tol=1e-11)
    assert ib["converged"] and ih["converged"]
    for nf in (ib["normF"], ih["normF"], rh.normF):
        assert abs(nf - rb.normF) < 1e-10 * rb.normF
    for U in (Ub, Uh):
        assert O.sin_theta_max(rb.U, U.cpu().numpy()) < 1e-8
    for W in (Wb, Wh):
        assert O.sin_theta_max(rb.W, W.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("seed", [101])
def test_fast_inner_schedule_reaches_the_oracle_optimum(seed):
    """BKS_INNER_FAST (no HOOI sweeps after the HOSVD start, HOOI sweeps to
    an inexact inner tolerance) reaches the same point as the Section 6.2
    schedule (HOSVD, 5 HOOI sweeps, Newton-Grassmann to the outer
    tolerance): on the 300x300x100 planted workload it ends where the
    oracle ends, ||F|| within 1e-10 relative and subspaces within 1e-8."""
    bk = _bk()
    coo, _ = synth.small_planted(1)
    A = O.symmetrise(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    g = synth.rng(seed)
    U0 = synth.orthonormal(g, A.m, 2); W0 = synth.orthonormal(g, A.n, 2)
    ro = O.bks(A, U0, W0, s=2, p=2, tol=1e-10)
    prm = bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-10,
                       inner_schedule=bk.BKS_INNER_FAST)
    U, W, F, info = bk.bks_solve(T, prm, _t(U0), _t(W0))
    _, _, _, paper = bk.bks_solve(T, bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-10),
                                  _t(U0), _t(W0))
    assert ro.converged and info["converged"] and paper["converged"]
    assert abs(info["normF"] - ro.normF) <= 1e-10 * ro.normF
    assert O.sin_theta_max(ro.U, U.cpu().numpy()) < 1e-8
    assert O.sin_theta_max(ro.W, W.cpu().numpy()) < 1e-8
    # paper mode follows the oracle's outer iteration
    assert abs(paper["iters"] - ro.iters) <= 1


_ZIPF5K = {}


def _zipf5k():
    """The 5000 x 5000 x 20 Zipf(1.1) tensor (60,000 one-sided draws, 86,990
    stored), a seeded rank-3 start and the oracle's BKS(2,4) solution at
    ||grad||/||F|| <= 1e-11 (computed once per session)."""
    if not _ZIPF5K:
        c = synth.zipf_tensor(21, 5000, 20, 60_000, 1.1)
        A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
        g = synth.rng(22)
        U0 = synth.orthonormal(g, c.m, 3); W0 = synth.orthonormal(g, c.n, 3)
        ro = O.bks(A, U0, W0, s=2, p=4, tol=1e-11)
        assert ro.converged
        _ZIPF5K.update(c=c, A=A, U0=U0, W0=W0, ro=ro)
    return _ZIPF5K


def test_mixed_precision_matches_the_oracle_at_1e6():
    """The FP32-contraction form at tol 1e-9 reaches the oracle's optimum
    (FP64, tol 1e-11, same start) within 1e-6 in the subspace angle on a
    power-law tensor, and its point is stationary by the oracle's own
    gradient."""
    bk = _bk()
    z = _zipf5k()
    c, A, ro = z["c"], z["A"], z["ro"]
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    pm = bk.BksParams(r1=3, r3=3, stages=2, block_p=4, tol=1e-9, precision=bk.BKS_PREC_MIXED,
                      refine_sweeps=20, mixed_tol=1e-6)
    Um, Wm, Fm, im = bk.bks_solve(T, pm, _t(z["U0"]), _t(z["W0"]))
    assert im["converged"] and im["fp32_iters"] > 0
    Uh, Wh = Um.cpu().numpy(), Wm.cpu().numpy()
    assert O.sin_theta_max(ro.U, Uh) < 1e-6
    assert O.sin_theta_max(ro.W, Wh) < 1e-6
    gg, nf, Fo = O.gradient_global(A, Uh, Wh)
    assert gg / nf < 1e-8
    assert abs(nf - ro.normF) <= 1e-9 * ro.normF
    assert np.allclose(Fm.cpu().numpy(), Fo, rtol=0, atol=1e-10 * nf)


def test_mixed_refinement_reaches_fp64_accuracy():
    """After the FP32 phase the mixed form refines with FP64 stage-1
    contractions and an FP32 core whose first-order blocks are FP64: it must
    still converge to FP64 accuracy (well below the FP32 noise floor), to the
    optimum of the oracle's FP64 solve from the same start."""
    bk = _bk()
    z = _zipf5k()
    c, A, ro = z["c"], z["A"], z["ro"]
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    tol = 1e-11  # the FP64 floor of ||grad||/||F|| here is about 3e-12
    pm = bk.BksParams(r1=3, r3=3, stages=2, block_p=4, tol=tol, precision=bk.BKS_PREC_MIXED,
                      refine_sweeps=50, mixed_tol=1e-6)
    Um, Wm, Fm, im = bk.bks_solve(T, pm, _t(z["U0"]), _t(z["W0"]))
    assert im["converged"]
    assert im["fp32_iters"] > 0 and im["iters"] > im["fp32_iters"]
    assert im["iters"] <= ro.iters + 10
    assert O.sin_theta_max(ro.U, Um.cpu().numpy()) < 1e-9
    assert O.sin_theta_max(ro.W, Wm.cpu().numpy()) < 1e-9
    gg, nf, _ = O.gradient_global(A, Um.cpu().numpy(), Wm.cpu().numpy())
    assert gg / nf < 2e-11
    assert abs(im["normF"] - ro.normF) <= 1e-12 * ro.normF


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hooi_parity_with_the_oracle(prec):
    """HOOI (Section 6.1) on the power-law tensor, FP64 and mixed (FP32
    contractions, then FP64 to the end), against the oracle's HOOI from the
    same start: ||F|| within 1e-10 relative, subspaces within 1e-8."""
    bk = _bk()
    z = _zipf5k()
    c, A = z["c"], z["A"]
    rh = O.hooi(A, z["U0"], z["W0"], tol=1e-10)
    assert rh.converged
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    hp = bk.HooiParams(r1=3, r3=3, tol=1e-10, max_iter=2000,
                       precision=bk.BKS_PREC_MIXED if prec == "mixed" else bk.BKS_PREC_FP64)
    U, W, F, info = bk.hooi_solve(T, hp, _t(z["U0"]), _t(z["W0"]))
    assert info["converged"]
    if prec == "mixed":
        assert 0 < info["fp32_iters"] < info["iters"]
    else:
        assert info["iters"] == rh.iters
    assert abs(info["normF"] - rh.normF) <= 1e-10 * rh.normF
    assert O.sin_theta_max(rh.U, U.cpu().numpy()) < 1e-8
    assert O.sin_theta_max(rh.W, W.cpu().numpy()) < 1e-8
    assert np.allclose(F.cpu().numpy(), O.core(A, U.cpu().numpy(), W.cpu().numpy()), rtol=0,
                       atol=1e-10 * rh.normF)


def test_newton_inner_solve_on_a_near_degenerate_job():
    """A very sparse batched job (4,400 x 4,400 x 65, 2,462 stored entries,
    rank 2) whose projected problems are nearly degenerate (nearly equal
    S-values): HOOI inner solves stall at their sweep cap, while the
    Section 6.2 schedule with Newton-Grassmann converges, on the GPU as in
    the oracle, to the same optimum from the same start."""
    bk = _bk()
    job = synth.batch_jobs(seed=4, count=256, scale=0.25)[96]
    c = synth.job_tensor(job)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    g = synth.rng(1096)
    U0 = synth.orthonormal(g, c.m, 2); W0 = synth.orthonormal(g, c.n, 2)
    ro = O.bks(A, U0, W0, s=2, p=4, tol=1e-9, scale_free=True, max_outer=100)
    prm = bk.BksParams(r1=2, r3=2, stages=2, block_p=4, tol=1e-9, tol_scale_free=1,
                       max_outer=100)
    U, W, F, info = bk.bks_solve(T, prm, _t(U0), _t(W0))
    assert ro.converged and info["converged"]
    assert abs(info["normF"] - ro.normF) <= 1e-10 * ro.normF
    gg, nf, _ = O.gradient_global(A, U.cpu().numpy(), W.cpu().numpy())
    assert gg / nf ** 2 <= 2e-9
