"""The general (l x m x n, three-basis) path on the GPU against the oracle:
ingest, the three block contractions, the core C = A.(X,Y,Z) and the solve
(Section 5, Algorithm 5, Proposition 2 with three terms)."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import fp32_bound

pytestmark = pytest.mark.gpu


def _bk():
    import paper_2012_07595_gb300 as bk
    from paper_2012_07595_gb300 import _build
    _build.build()
    return bk


def _t(x, dtype=None):
    import torch
    t = torch.tensor(np.asarray(x), device="cuda")
    return t if dtype is None else t.to(dtype)


def _pair(bk, c, vdtype=np.float64):
    A = O.gen_tensor(c.l, c.m, c.n, c.i, c.j, c.k, c.v.astype(vdtype))
    T = bk.bks_gen_tensor_create_coo(c.l, c.m, c.n, c.i, c.j, c.k, c.v.astype(vdtype))
    return A, T


# power-law rows in modes 1 and 2 (long rows cut into pieces, short rows in
# the lane-interleaved copy), ragged dimensions
CASES = {
    "uniform": lambda: synth.general_random_coo(3, 57, 43, 11, 3000),
    "zipf": lambda: synth.general_zipf_tensor(4, 3001, 2203, 37, 60000, 1.2),
    "tiny": lambda: synth.general_random_coo(5, 3, 2, 1, 7),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("vdtype", [np.float64, np.float32])
def test_ingest_bitwise(case, vdtype):
    bk = _bk()
    c = CASES[case]()
    A, T = _pair(bk, c, vdtype)
    assert T.general and (T.l, T.m, T.n) == (c.l, c.m, c.n) and T.nnz == A.nnz
    i, j, k, v = (x.cpu().numpy() for x in bk.bks_tensor_export_coo(T))
    assert np.array_equal(i, A.i) and np.array_equal(j, A.j) and np.array_equal(k, A.k)
    assert v.dtype == A.v.dtype and v.tobytes() == A.v.tobytes()
    assert abs(T.fro2 - A.fro2()) <= 1e-12 * A.fro2()


def test_errors_and_handle_kinds():
    bk = _bk()
    import torch
    with pytest.raises(bk.BksError):                     # j >= m
        bk.bks_gen_tensor_create_coo(4, 3, 2, [0], [3], [0], np.array([1.0]))
    T = bk.bks_gen_tensor_create_coo(4, 3, 2, [3], [2], [1], np.array([1.0]))
    X = torch.ones((3, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(bk.BksError, match="general"):    # symmetric calls refuse it
        bk.bks_contract_mode1(T, X, torch.ones((2, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(bk.BksError, match="general"):
        bk.bks_solve(T, bk.BksParams(r1=1, r3=1))
    S = bk.bks_tensor_create_coo(3, 2, [0], [1], [0], np.array([1.0]))
    assert not S.general and S.l == S.m
    with pytest.raises(bk.BksError, match="symmetric"):  # general calls refuse a symmetric one
        bk.bks_gen_contract(S, 1, X, X)
    with pytest.raises(bk.BksError):
        bk.bks_gen_contract(T, 4, X, X)
    with pytest.raises(bk.BksError):                     # rank above the dimension
        bk.bks_gen_solve(T, bk.BksGenParams(r1=1, r2=1, r3=3))
    # empty tensor: contractions give zeros
    E = bk.bks_gen_tensor_create_coo(5, 4, 3, np.zeros(0, np.int32), np.zeros(0, np.int32),
                                     np.zeros(0, np.int32), np.zeros(0))
    out = bk.bks_gen_contract(E, 2, torch.ones((5, 2), dtype=torch.float64, device="cuda"),
                              torch.ones((3, 3), dtype=torch.float64, device="cuda"))
    assert out.shape == (4, 6) and float(out.abs().max()) == 0.0


def _abs_terms(A, md, L, R):
    Aa = O.GenTensor(A.l, A.m, A.n, A.i, A.j, A.k, np.abs(A.vf()))
    f = (O.gmode1, O.gmode2, O.gmode3)[md - 1]
    return f(Aa, np.abs(L), np.abs(R))


@pytest.mark.parametrize("case", ["uniform", "zipf"])
@pytest.mark.parametrize("p,q", [(1, 1), (3, 4), (5, 5), (8, 3), (2, 8)])
def test_contractions_fp64_and_fp32(case, p, q):
    bk = _bk()
    import torch
    c = CASES[case]()
    A, T = _pair(bk, c)
    g = synth.rng(100 + p * 10 + q)
    rows = {1: (A.m, A.n), 2: (A.l, A.n), 3: (A.l, A.m)}
    f = {1: O.gmode1, 2: O.gmode2, 3: O.gmode3}
    A32, T32 = _pair(bk, c, np.float32)
    for md in (1, 2, 3):
        L = g.standard_normal((rows[md][0], p)); R = g.standard_normal((rows[md][1], q))
        ref = f[md](A, L, R)
        bound = _abs_terms(A, md, L, R)
        got = bk.bks_gen_contract(T, md, _t(L), _t(R)).cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-13 * bound + 1e-300), (md, "fp64")
        # FP32 operands and values: the FP64 oracle on the rounded inputs,
        # within the blocked-sum bound
        L32, R32 = L.astype(np.float32), R.astype(np.float32)
        ref32 = f[md](A32, L32.astype(np.float64), R32.astype(np.float64))
        got32 = bk.bks_gen_contract(T32, md, _t(L32), _t(R32)).cpu().numpy()
        assert np.all(np.abs(got32 - ref32) <= fp32_bound(_abs_terms(A32, md, L32, R32))), (md, "fp32")


@pytest.mark.parametrize("k", [(14, 9, 6), (36, 30, 21), (70, 57, 40), (100, 128, 30), (1, 1, 1)])
def test_core_fp64(k):
    bk = _bk()
    c = CASES["zipf"]()
    A, T = _pair(bk, c)
    g = synth.rng(sum(k))
    k1, k2, k3 = k
    X = g.standard_normal((A.l, k1)); Y = g.standard_normal((A.m, k2)); Z = g.standard_normal((A.n, k3))
    ref = O.gcore(A, X, Y, Z)
    Aa = O.GenTensor(A.l, A.m, A.n, A.i, A.j, A.k, np.abs(A.vf()))
    bound = O.gcore(Aa, np.abs(X), np.abs(Y), np.abs(Z))
    got = bk.bks_gen_core(T, _t(X), _t(Y), _t(Z)).cpu().numpy()
    assert got.shape == (k1, k2, k3)
    assert np.all(np.abs(got - ref) <= 1e-12 * bound + 1e-300)


def _starts(seed, dims, r):
    g = synth.rng(seed)
    return [synth.orthonormal(g, d, rr) for d, rr in zip(dims, r)]


def _check_at_point(A, U, V, W, F, tol):
    """The oracle at the returned point: orthonormal factors, F = A.(U,V,W)
    and a gradient within the tolerance."""
    for Q in (U, V, W):
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-12
    Fo = O.gcore(A, U, V, W)
    assert np.abs(F - Fo).max() <= 1e-10 * np.abs(Fo).max()
    g, nf, _ = O.gen_gradient_global(A, U, V, W)
    assert g / nf <= 2 * tol


@pytest.mark.parametrize("variant", ["bk", "min", "max"])
def test_solve_parity_planted_sparse(variant):
    """Same start and schedule as the oracle: the same optimum (||F|| within
    1e-10, subspaces within 1e-8) and the oracle's checks at the returned
    point."""
    bk = _bk()
    c = synth.general_noisy_planted(31, (40, 30, 12), (2, 2, 2), 0.3)
    A, T = _pair(bk, c)
    r = (2, 2, 2)
    U0, V0, W0 = _starts(22, (A.l, A.m, A.n), r)
    vcode = {"bk": bk.BKS_VARIANT_BK, "min": bk.BKS_VARIANT_MIN, "max": bk.BKS_VARIANT_MAX}[variant]
    U, V, W, F, info = bk.bks_gen_solve(
        T, bk.BksGenParams(r1=2, r2=2, r3=2, stages=2, block_p=2, tol=1e-10, variant=vcode),
        _t(U0), _t(V0), _t(W0))
    ref = O.gen_bks(A, U0, V0, W0, s=2, p=2, tol=1e-10, variant=variant)
    assert info["converged"] and ref.converged
    assert abs(info["normF"] - ref.normF) <= 1e-10 * ref.normF
    Ug, Vg, Wg, Fg = (x.cpu().numpy() for x in (U, V, W, F))
    for X, Y in ((ref.U, Ug), (ref.V, Vg), (ref.W, Wg)):
        assert O.sin_theta_max(X, Y) < 1e-8
    _check_at_point(A, Ug, Vg, Wg, Fg, 1e-10)
    assert info["iters"] == ref.iters


def test_fast_inner_schedule_reaches_the_oracle_optimum():
    """BKS_INNER_FAST (no start sweeps, inexact inner tolerance) against the
    oracle on the Section 6.2 schedule: the same optimum."""
    bk = _bk()
    c = synth.general_noisy_planted(32, (50, 40, 15), (3, 2, 2), 0.5)
    A, T = _pair(bk, c)
    U0, V0, W0 = _starts(33, (50, 40, 15), (3, 2, 2))
    ref = O.gen_bks(A, U0, V0, W0, s=2, p=2, tol=1e-10)
    U, V, W, F, info = bk.bks_gen_solve(
        T, bk.BksGenParams(r1=3, r2=2, r3=2, block_p=2, tol=1e-10,
                           inner_schedule=bk.BKS_INNER_FAST), _t(U0), _t(V0), _t(W0))
    assert ref.converged and info["converged"]
    assert abs(info["normF"] - ref.normF) <= 1e-10 * ref.normF
    for X, Y in ((ref.U, U), (ref.V, V), (ref.W, W)):
        assert O.sin_theta_max(X, Y.cpu().numpy()) < 1e-8


def test_hooi_parity_and_agreement_with_bks():
    """General HOOI on the GPU against the oracle's (same start, same
    iteration count at the 10-iteration gradient cadence, same optimum),
    and the BKS optimum on the same tensor."""
    bk = _bk()
    c = synth.general_noisy_planted(34, (45, 35, 14), (2, 3, 2), 0.4)
    A, T = _pair(bk, c)
    U0, V0, W0 = _starts(35, (45, 35, 14), (2, 3, 2))
    U, V, W, F, info = bk.bks_gen_hooi_solve(T, bk.BksGenHooiParams(r1=2, r2=3, r3=2, tol=1e-10),
                                             _t(U0), _t(V0), _t(W0))
    ref = O.gen_hooi(A, U0, V0, W0, tol=1e-10)
    assert info["converged"] and ref.converged
    assert info["iters"] == ref.iters
    assert abs(info["normF"] - ref.normF) <= 1e-10 * ref.normF
    Ug, Vg, Wg, Fg = (x.cpu().numpy() for x in (U, V, W, F))
    for X, Y in ((ref.U, Ug), (ref.V, Vg), (ref.W, Wg)):
        assert O.sin_theta_max(X, Y) < 1e-8
    _check_at_point(A, Ug, Vg, Wg, Fg, 1e-10)
    Ub, Vb, Wb, Fb, ib = bk.bks_gen_solve(T, bk.BksGenParams(r1=2, r2=3, r3=2, block_p=2, tol=1e-10),
                                          _t(U0), _t(V0), _t(W0))
    assert ib["converged"] and abs(ib["normF"] - info["normF"]) <= 1e-10 * info["normF"]
    for X, Y in ((Ub, U), (Vb, V), (Wb, W)):
        assert O.sin_theta_max(X.cpu().numpy(), Y.cpu().numpy()) < 1e-7


def test_planted_exact_rank_and_matrix_case():
    bk = _bk()
    T0, Ut, Vt, Wt, F0 = synth.general_dense_planted(23, 26, 19, 9, (2, 3, 2))
    A, T = _pair(bk, synth.general_dense_to_coo(T0))
    U0, V0, W0 = _starts(24, (26, 19, 9), (2, 3, 2))
    U, V, W, F, info = bk.bks_gen_solve(T, bk.BksGenParams(r1=2, r2=3, r3=2, block_p=2, tol=1e-11),
                                        _t(U0), _t(V0), _t(W0))
    assert info["converged"]
    assert abs(info["normF"] - np.sqrt(A.fro2())) <= 1e-10 * info["normF"]
    for X, Y in ((Ut, U), (Vt, V), (Wt, W)):
        assert O.sin_theta_max(X, Y.cpu().numpy()) < 1e-8
    # n = 1: Eckart-Young
    g = synth.rng(25)
    Mx = g.standard_normal((30, 22)) @ np.diag(np.linspace(3, 0.1, 22)) @ g.standard_normal((22, 22))
    A, T = _pair(bk, synth.general_dense_to_coo(Mx[:, :, None]))
    U0, V0 = synth.orthonormal(g, 30, 3), synth.orthonormal(g, 22, 3)
    U, V, W, F, info = bk.bks_gen_solve(T, bk.BksGenParams(r1=3, r2=3, r3=1, block_p=3, tol=1e-11),
                                        _t(U0), _t(V0), _t(np.ones((1, 1))))
    s = np.linalg.svd(Mx, compute_uv=False)
    assert info["converged"]
    assert abs(info["normF"] - np.sqrt(np.sum(s[:3] ** 2))) <= 1e-10 * info["normF"]


def test_symmetric_tensor_through_the_general_path():
    """A (1,2)-symmetric tensor stored as a general one, solved from
    (U0, U0, W0): the symmetric solver's optimum, with span(U) = span(V)."""
    bk = _bk()
    c, meta = synth.small_planted(seed=26, m=80, n=24, draws=2500)
    S = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    TS = bk.bks_tensor_create_coo(S.m, S.n, S.i, S.j, S.k, S.v, mirror=False)
    TG = bk.bks_gen_tensor_create_coo(S.m, S.m, S.n, S.i, S.j, S.k, S.v)
    g = synth.rng(27)
    U0 = synth.orthonormal(g, 80, 2); W0 = synth.orthonormal(g, 24, 2)
    Us, Ws, Fs, infs = bk.bks_solve(TS, bk.BksParams(r1=2, r3=2, stages=2, block_p=2, tol=1e-10),
                                    _t(U0), _t(W0))
    U, V, W, F, info = bk.bks_gen_solve(TG, bk.BksGenParams(r1=2, r2=2, r3=2, block_p=2, tol=1e-10),
                                        _t(U0), _t(U0), _t(W0))
    assert infs["converged"] and info["converged"]
    assert abs(info["normF"] - infs["normF"]) <= 1e-9 * infs["normF"]
    assert O.sin_theta_max(U.cpu().numpy(), V.cpu().numpy()) < 1e-7
    assert O.sin_theta_max(Us.cpu().numpy(), U.cpu().numpy()) < 1e-7
    assert O.sin_theta_max(Ws.cpu().numpy(), W.cpu().numpy()) < 1e-7


def test_zipf_workload_solve_checked_by_the_oracle():
    """A power-law general tensor (several thousand rows per mode) solved
    to 1e-9: the oracle's gradient and core at the returned point."""
    bk = _bk()
    c = synth.general_zipf_tensor(28, 4000, 3000, 40, 80000, 1.1)
    A, T = _pair(bk, c)
    U, V, W, F, info = bk.bks_gen_solve(T, bk.BksGenParams(r1=3, r2=3, r3=3, tol=1e-9, seed=5))
    assert info["converged"]
    _check_at_point(A, *(x.cpu().numpy() for x in (U, V, W, F)), 1e-9)


def test_bench_size_general_solve_checked_by_the_oracle():
    """The benchmark's general workload (100,000 x 80,000 x 50, 5M draws,
    rank (3,3,3), BK(2,4), ||grad||/||F||^2 <= 1e-9) from the benchmark's
    start: the oracle's gradient and core at the returned point."""
    bk = _bk()
    c = synth.general_zipf_tensor(6, 100_000, 80_000, 50, 5_000_000, 1.1)
    A, T = _pair(bk, c)
    U0, V0, W0 = _starts(23, (A.l, A.m, A.n), (3, 3, 3))
    U, V, W, F, info = bk.bks_gen_solve(
        T, bk.BksGenParams(r1=3, r2=3, r3=3, tol=1e-9, tol_scale_free=1, max_outer=300),
        _t(U0), _t(V0), _t(W0))
    assert info["converged"]
    Ug, Vg, Wg, Fg = (x.cpu().numpy() for x in (U, V, W, F))
    for Q in (Ug, Vg, Wg):
        assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-12
    g, nf, Fo = O.gen_gradient_global(A, Ug, Vg, Wg)
    assert g / nf ** 2 <= 2e-9
    assert np.abs(Fg - Fo).max() <= 1e-10 * np.abs(Fo).max()
