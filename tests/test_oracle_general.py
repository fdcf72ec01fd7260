"""Pins of the general (l x m x n, three-basis) oracle: storage, contractions,
closed forms, planted recovery, the symmetric special case, Lemma 1,
Proposition 2, monotone inner sweeps and BKS/HOOI agreement (Section 5)."""
import numpy as np
import pytest

import oracle as O
import synth


def _gen(c):
    return O.gen_tensor(c.l, c.m, c.n, c.i, c.j, c.k, c.v)


def test_storage_dict_model():
    """Sorted by (i, j, k), duplicates summed left to right in input order,
    zeros kept, nothing mirrored."""
    c = synth.general_random_coo(1, 7, 5, 4, 400)
    c.v[::7] = 0.0
    A = _gen(c)
    model = {}
    for a, b, d, x in zip(c.i.tolist(), c.j.tolist(), c.k.tolist(), c.v.tolist()):
        model[(a, b, d)] = model[(a, b, d)] + x if (a, b, d) in model else x
    keys = sorted(model)
    assert [tuple(t) for t in zip(A.i.tolist(), A.j.tolist(), A.k.tolist())] == keys
    assert all(np.float64(model[kk]).tobytes() == np.float64(x).tobytes()
               for kk, x in zip(keys, A.v.tolist()))
    with pytest.raises(ValueError):
        O.gen_tensor(3, 3, 3, [0], [3], [0], [1.0])


def test_contractions_and_core_by_einsum():
    c = synth.general_random_coo(2, 9, 7, 5, 250)
    A = _gen(c)
    T = A.dense()
    g = synth.rng(5)
    U, V, W = g.standard_normal((9, 3)), g.standard_normal((7, 2)), g.standard_normal((5, 4))
    e1 = np.einsum("ijk,ja,kb->iab", T, V, W).reshape(9, -1, order="F")
    e2 = np.einsum("ijk,ia,kb->jab", T, U, W).reshape(7, -1, order="F")
    e3 = np.einsum("ijk,ia,jb->kab", T, U, V).reshape(5, -1, order="F")
    assert np.allclose(O.gmode1(A, V, W), e1, atol=1e-12)
    assert np.allclose(O.gmode2(A, U, W), e2, atol=1e-12)
    assert np.allclose(O.gmode3(A, U, V), e3, atol=1e-12)
    C = O.gcore(A, U, V, W)
    assert np.allclose(C, np.einsum("ijk,ia,jb,kc->abc", T, U, V, W), atol=1e-12)
    # unfoldings of the core are the contractions' projections
    assert np.allclose(O.gunfold(C, 0), U.T @ e1, atol=1e-12)
    assert np.allclose(O.gunfold(C, 1), V.T @ e2, atol=1e-12)
    assert np.allclose(O.gunfold(C, 2), W.T @ e3, atol=1e-12)


def test_gcore_by_einsum_over_several_entry_blocks():
    """The core over more stored entries than one of the oracle's entry
    blocks (2048): every entry counted exactly once."""
    c = synth.general_random_coo(6, 20, 18, 16, 9000)
    A = _gen(c)
    assert A.nnz > 2 * 2048
    g = synth.rng(6)
    X, Y, Z = g.standard_normal((20, 3)), g.standard_normal((18, 4)), g.standard_normal((16, 2))
    ref = np.einsum("ijk,ia,jb,kc->abc", A.dense(), X, Y, Z)
    assert np.allclose(O.gcore(A, X, Y, Z), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_schedule_counts_first_stages():
    # stage 1 adds r_a r_b columns per mode; stage 2 of BK adds the two
    # off-diagonal pairs (0,1), (1,0) of p-column bars
    assert O.gen_schedule_counts((2, 3, 4), 2, 4) == [
        (2 + 12, 3 + 8, 4 + 6), (2 + 12 + 3 * 4 + 4 * 4, 3 + 8 + 2 * 4 + 4 * 4, 4 + 6 + 2 * 4 + 4 * 3)]
    assert O.gen_schedule_counts((2, 2, 2), 3, 4, "min") == [(6, 6, 6), (22, 22, 22), (38, 38, 38)]
    # caps at the dimensions
    assert O.gen_schedule_counts((2, 2, 2), 2, 4, dims=(50, 40, 7))[-1][2] == 7


def test_matrix_case_eckart_young():
    """n = 1: A is an l x m matrix M and the best rank-(r, r, 1)
    approximation keeps its r leading singular pairs:
    ||F||^2 = sigma_1^2 + ... + sigma_r^2 (Eckart-Young)."""
    g = synth.rng(7)
    l, m, r = 30, 22, 3
    Mx = g.standard_normal((l, m)) @ np.diag(np.linspace(3, 0.1, m)) @ g.standard_normal((m, m))
    A = _gen(synth.general_dense_to_coo(Mx[:, :, None]))
    s = np.linalg.svd(Mx, compute_uv=False)
    U0 = synth.orthonormal(g, l, r); V0 = synth.orthonormal(g, m, r); W0 = np.ones((1, 1))
    res = O.gen_bks(A, U0, V0, W0, s=2, p=3, tol=1e-11)
    assert res.converged
    assert abs(res.normF - np.sqrt(np.sum(s[:r] ** 2))) <= 1e-10 * res.normF
    u, _, vt = np.linalg.svd(Mx)
    assert O.sin_theta_max(u[:, :r], res.U) < 1e-8
    assert O.sin_theta_max(vt[:r].T, res.V) < 1e-8
    h = O.gen_hooi(A, U0, V0, W0, tol=1e-11)
    assert abs(h.normF - res.normF) <= 1e-10 * res.normF


@pytest.mark.parametrize("variant", ["bk", "min", "max"])
def test_planted_exact_rank_recovered(variant):
    """A tensor of exact multilinear rank (2, 3, 2) with l, m, n all
    different: the solve returns its factor spans and ||F|| = ||A||."""
    T, U0, V0, W0, F0 = synth.general_dense_planted(3, 26, 19, 9, (2, 3, 2))
    A = _gen(synth.general_dense_to_coo(T))
    g = synth.rng(8)
    Us = synth.orthonormal(g, 26, 2); Vs = synth.orthonormal(g, 19, 3); Ws = synth.orthonormal(g, 9, 2)
    res = O.gen_bks(A, Us, Vs, Ws, s=2, p=2, tol=1e-11, variant=variant)
    assert res.converged
    assert abs(res.normF - np.sqrt(A.fro2())) <= 1e-10 * res.normF
    for X, Y in ((U0, res.U), (V0, res.V), (W0, res.W)):
        assert O.sin_theta_max(X, Y) < 1e-8


def test_hosvd_of_exact_rank_core():
    T, U0, V0, W0, F0 = synth.general_dense_planted(4, 12, 10, 8, (3, 2, 2))
    Uh, Vh, Wh = O.gen_hosvd(T, (3, 2, 2))
    for X, Y in ((U0, Uh), (V0, Vh), (W0, Wh)):
        assert O.sin_theta_max(X, Y) < 1e-12


def test_symmetric_special_case_matches_symmetric_oracle():
    """On a (1,2)-symmetric tensor with V = U, the three-term gradient
    equals the symmetric oracle's 2 ||g1||^2 + ||g3||^2 form, and the
    general solve from (U0, U0, W0) reaches the symmetric optimum with
    span(U) = span(V)."""
    c, meta = synth.small_planted(seed=11, m=60, n=20, draws=1500)
    S = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    A = O.gen_tensor(S.m, S.m, S.n, S.i, S.j, S.k, S.v)
    g = synth.rng(9)
    U = synth.orthonormal(g, 60, 2); W = synth.orthonormal(g, 20, 2)
    gs, nfs, Fs = O.gradient_global(S, U, W)
    gg, nfg, Fg = O.gen_gradient_global(A, U, U, W)
    assert abs(gs - gg) <= 1e-12 * gs and abs(nfs - nfg) <= 1e-13 * nfs
    assert np.allclose(Fs, Fg, atol=1e-13)
    rs = O.bks(S, U, W, s=2, p=2, tol=1e-10)
    rg = O.gen_bks(A, U, U.copy(), W, s=2, p=2, tol=1e-10)
    assert rs.converged and rg.converged
    assert abs(rs.normF - rg.normF) <= 1e-10 * rs.normF
    assert O.sin_theta_max(rg.U, rg.V) < 1e-7
    assert O.sin_theta_max(rs.U, rg.U) < 1e-7
    assert O.sin_theta_max(rs.W, rg.W) < 1e-7


def test_lemma1_on_the_expansion():
    """Lemma 1: A.(U_j, V0, W0) = 0 for j >= 2 (and the same in modes 2 and
    3), for the blocks the general BK schedule makes."""
    A = _gen(synth.general_random_coo(12, 40, 33, 11, 1500))
    g = synth.rng(10)
    U0 = synth.orthonormal(g, 40, 2); V0 = synth.orthonormal(g, 33, 2); W0 = synth.orthonormal(g, 11, 2)
    X, Y, Z, info, blocks = O.gen_expand(A, U0, V0, W0, 2, 2)
    assert len(blocks[0]) >= 4
    for j in range(2, len(blocks[0])):
        assert np.abs(O.gcore(A, blocks[0][j], V0, W0)).max() < 1e-12
    for j in range(2, len(blocks[1])):
        assert np.abs(O.gcore(A, U0, blocks[1][j], W0)).max() < 1e-12
    for j in range(2, len(blocks[2])):
        assert np.abs(O.gcore(A, U0, V0, blocks[2][j])).max() < 1e-12
    for B, K in ((X, 40), (Y, 33), (Z, 11)):
        assert np.abs(B.T @ B - np.eye(B.shape[1])).max() < 1e-13


def test_prop2_equals_global_gradient():
    A = _gen(synth.general_random_coo(13, 35, 28, 9, 1200))
    g = synth.rng(11)
    for r in [(2, 2, 2), (3, 2, 2), (2, 3, 1)]:
        U = synth.orthonormal(g, 35, r[0]); V = synth.orthonormal(g, 28, r[1])
        W = synth.orthonormal(g, 9, r[2])
        _, _, _, info, _ = O.gen_expand(A, U, V, W, 1, 2)
        gp, nfp, Fp = O.gen_gradient_prop2(info, r)
        gg, nfg, Fg = O.gen_gradient_global(A, U, V, W)
        assert abs(gp - gg) <= 1e-12 * gg and abs(nfp - nfg) <= 1e-13 * nfg
        assert np.allclose(Fp, O.gcore(A, U, V, W), atol=1e-13)


def test_gradient_finite_difference_mode2():
    """The mode-2 term is the projected derivative of ||F||^2 / 2 in V."""
    A = _gen(synth.general_random_coo(14, 20, 16, 6, 500))
    g = synth.rng(12)
    U = synth.orthonormal(g, 20, 2); V = synth.orthonormal(g, 16, 2); W = synth.orthonormal(g, 6, 2)
    T2 = O.gmode2(A, U, W)
    F2 = V.T @ T2
    G2 = T2 @ F2.T
    G2 -= V @ (V.T @ G2)
    D = g.standard_normal(V.shape); D -= V @ (V.T @ D)
    h = 1e-6
    phi = lambda Vx: 0.5 * np.sum(O.gcore(A, U, np.linalg.qr(Vx)[0], W) ** 2)
    fd = (phi(V + h * D) - phi(V - h * D)) / (2 * h)
    assert abs(fd - np.sum(G2 * D)) < 1e-5 * max(1.0, abs(fd))


def test_inner_sweeps_monotone_and_stationary():
    g = synth.rng(15)
    C = g.standard_normal((12, 10, 8))
    Uh, Vh, Wh, info = O.gen_inner_solve(C, (2, 3, 2), 1e-11, max_inner=2000)
    h = info["normF_history"]
    assert all(b >= a * (1 - 1e-14) for a, b in zip(h, h[1:]))
    assert info["grad"] <= 1e-11 * info["normF"]
    F = np.einsum("abc,ai,bj,ck->ijk", C, Uh, Vh, Wh)
    assert abs(np.linalg.norm(F) - info["normF"]) <= 1e-12 * info["normF"]


def test_bks_and_hooi_agree_on_a_sparse_planted_tensor():
    A = _gen(synth.general_sampled_planted(16, 90, 70, 25, 6000, (2, 2, 2)))
    g = synth.rng(13)
    U0 = synth.orthonormal(g, 90, 2); V0 = synth.orthonormal(g, 70, 2); W0 = synth.orthonormal(g, 25, 2)
    rb = O.gen_bks(A, U0, V0, W0, s=2, p=2, tol=1e-10)
    rh = O.gen_hooi(A, U0, V0, W0, tol=1e-10)
    assert rb.converged and rh.converged
    assert abs(rb.normF - rh.normF) <= 1e-9 * rb.normF
    for X, Y in ((rb.U, rh.U), (rb.V, rh.V), (rb.W, rh.W)):
        assert O.sin_theta_max(X, Y) < 1e-6


def test_inner_solve_takes_the_better_start():
    """The HOSVD candidate of an exact-rank core is exact, so it wins over a
    current point ([I;0]) that misses the core's subspaces; a core whose
    subspaces are the current point's keeps that point's ||F||."""
    T, U0, V0, W0, F0 = synth.general_dense_planted(17, 14, 12, 9, (2, 2, 2))
    Uh, Vh, Wh, info = O.gen_inner_solve(T, (2, 2, 2), 1e-12, max_inner=0)
    assert info["hosvd_won"]
    assert abs(info["normF"] - np.linalg.norm(T)) <= 1e-12 * np.linalg.norm(T)
    E = [np.eye(d, 2) for d in (14, 12, 9)]
    T2 = np.einsum("ia,jb,kc,abc->ijk", E[0], E[1], E[2], F0)
    Uh, Vh, Wh, info = O.gen_inner_solve(T2, (2, 2, 2), 1e-12, max_inner=0)
    assert abs(info["normF"] - np.linalg.norm(F0)) <= 1e-12 * np.linalg.norm(F0)


def test_inner_gradient_is_the_global_gradient_of_the_core():
    """The general inner solve's gradient on a dense core C is the
    three-term G-gradient of C itself (gen_gradient_global on C stored as
    a sparse tensor)."""
    from oracle import bks_general_oracle as G
    g = synth.rng(24)
    for k, r in [((9, 8, 6), (2, 3, 2)), ((7, 10, 5), (3, 2, 2))]:
        C = g.standard_normal(k)
        facs = tuple(np.linalg.qr(g.standard_normal((k[d], r[d])))[0] for d in range(3))
        gi, nfi = G._ginner_grad(C, facs)
        ii, jj, kk = np.meshgrid(*(np.arange(x) for x in k), indexing="ij")
        A = O.gen_tensor(*k, ii.ravel(), jj.ravel(), kk.ravel(), C.ravel())
        gg, nfg, _ = O.gen_gradient_global(A, *facs)
        assert abs(gi - gg) <= 1e-12 * gg and abs(nfi - nfg) <= 1e-13 * nfg


def test_expansion_sizes_follow_the_bar_rule():
    """With blocks wider than p after stage 1 (r_a r_b = 6 > p = 4), later
    stages contract only the first p columns of each block but U_0, V_0,
    W_0 (the bars of Tables 1-3 in their general form): on a tensor large
    enough that nothing is dropped, the bases have the sizes the pair and
    bar rule gives."""
    A = _gen(synth.general_random_coo(14, 90, 80, 70, 60000))
    g = synth.rng(12)
    r = (2, 3, 2)
    facs = [synth.orthonormal(g, d, rr) for d, rr in zip((90, 80, 70), r)]
    for s in (2, 3):
        X, Y, Z, _, _ = O.gen_expand(A, *facs, s, 4)
        assert (X.shape[1], Y.shape[1], Z.shape[1]) == O.gen_schedule_counts(r, s, 4, dims=(90, 80, 70))[-1]


def test_general_schedule_in_modes_1_and_2_is_the_symmetric_u_schedule():
    """Modes 1 and 2 of the general BK schedule pair blocks of the other two
    factors as the (1,2)-symmetric schedule pairs (U, W) blocks, in the same
    order, which Table 3's diagrams number."""
    from oracle import bks_oracle as B
    done_s, done_w = set(), set()
    done_g = [set(), set(), set()]
    for stage in range(1, 5):
        us, _ = B._stage_pairs("bk", stage, 100, 100, done_s, done_w)
        gp = O.gen_stage_pairs("bk", stage, (100, 100, 100), done_g)
        sym = [(a, b) for a, b, _ in us]
        assert gp[0] == sym and gp[1] == sym


def test_general_inner_solve_runs_five_start_sweeps():
    g = synth.rng(25)
    C = g.standard_normal((9, 8, 7))
    _, _, _, info = O.gen_inner_solve(C, (2, 2, 2), 1e-14, max_inner=0)
    assert info["hosvd_won"] and info["sweeps"] == 5


def test_hosvd_of_exact_rank_cube():
    """Equal dimensions in all three modes, a different factor in each: the
    HOSVD takes each mode's own unfolding."""
    T, U0, V0, W0, F0 = synth.general_dense_planted(5, 10, 10, 10, (3, 2, 2))
    Uh, Vh, Wh = O.gen_hosvd(T, (3, 2, 2))
    for X, Y in ((U0, Uh), (V0, Vh), (W0, Wh)):
        assert O.sin_theta_max(X, Y) < 1e-12


def test_general_hooi_checks_the_gradient_every_ten_iterations():
    A = _gen(synth.general_random_coo(15, 20, 18, 6, 500))
    g = synth.rng(13)
    facs = [synth.orthonormal(g, d, 2) for d in (20, 18, 6)]
    res = O.gen_hooi(A, *facs, tol=0.0, max_iter=25)
    assert [h["iter"] for h in res.history] == [0, 10, 20, 25]
