"""Pins of the oracle's block orthogonalisation and block schedules."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_orth_block_reconstruction_and_orthonormality():
    g = synth.rng(11)
    m = 200
    Q = np.linalg.qr(g.standard_normal((m, 7)))[0]
    B = g.standard_normal((m, 6)) + Q @ g.standard_normal((7, 6)) * 10
    Qn, H, R, kept, S = O.orth_block(Q, B, 1e-12)
    assert kept == list(range(6))
    Z = np.concatenate([Q, Qn], axis=1)
    assert np.linalg.norm(Z.T @ Z - np.eye(13)) < 1e-13
    assert np.linalg.norm(B - Q @ H - Qn @ R) < 1e-12 * np.linalg.norm(B)
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) > 0)


def test_orth_block_drops_dependent_columns():
    g = synth.rng(12)
    m = 100
    Q = np.linalg.qr(g.standard_normal((m, 4)))[0]
    a = g.standard_normal(m); b = g.standard_normal(m)
    # col0 free, col1 inside span(Q), col2 free, col3 = 2*col0 - col2 + Q-part, col4 = 0
    B = np.stack([a, Q @ np.ones(4), b, 2 * a - b + Q[:, 0], np.zeros(m)], axis=1)
    Qn, H, R, kept, S = O.orth_block(Q, B, 1e-12)
    assert kept == [0, 2]
    assert Qn.shape == (m, 2)
    assert np.linalg.norm(B - Q @ H - Qn @ R) < 1e-12 * np.linalg.norm(B)
    # the cap on the total number of basis vectors (k3 <= n) also drops
    Qn2, _, _, kept2, _ = O.orth_block(Q, B, 1e-12, max_total=5)
    assert kept2 == [0]


def _gold():
    with open(os.path.join(GOLD, "schedule_counts.json")) as f:
        return json.load(f)


def test_orth_block_projected_block_orthogonal_when_nearly_dependent():
    """Projecting twice leaves the projected block orthogonal to Q to
    working precision relative to its own norm, even when the block lies in
    span(Q) but for a 1e-10 residual (the stage-1 block near convergence,
    whose residual carries the gradient).  One classical Gram-Schmidt round
    would leave about eps ||B|| / ||P|| = 1e-6 of it in span(Q)."""
    g = synth.rng(13)
    m = 300
    Q = np.linalg.qr(g.standard_normal((m, 9)))[0]
    N = g.standard_normal((m, 4))
    N -= Q @ (Q.T @ N)
    B = Q @ g.standard_normal((9, 4)) + 1e-10 * N
    Qn, H, R, kept, P = O.orth_block(Q, B, 1e-14)
    for c in range(4):
        assert np.linalg.norm(Q.T @ P[:, c]) <= 1e-12 * np.linalg.norm(P[:, c])
    assert np.linalg.norm(P - 1e-10 * N) <= 1e-5 * np.linalg.norm(1e-10 * N)
    assert kept == [0, 1, 2, 3]


def test_orth_block_drop_rule_is_relative():
    """The drop rule compares a column's residual with its own raw norm, so
    the kept columns do not depend on the scale of the block: a tiny
    independent column is kept, a huge nearly dependent one is dropped."""
    g = synth.rng(14)
    m = 120
    Q = np.linalg.qr(g.standard_normal((m, 5)))[0]
    N = g.standard_normal((m, 3))
    N -= Q @ (Q.T @ N)
    B = Q @ g.standard_normal((5, 3)) + N
    ref = O.orth_block(Q, B, 1e-12)[3]
    assert ref == [0, 1, 2]
    for scale in (1e-20, 1.0, 1e20):
        assert O.orth_block(Q, scale * B, 1e-12)[3] == ref
    # column 1 dependent on Q up to a 1e-14 relative residual, at a large scale
    B2 = B.copy()
    B2[:, 1] = Q @ g.standard_normal(5) + 1e-14 * N[:, 1]
    for scale in (1e-20, 1.0, 1e20):
        assert O.orth_block(Q, scale * B2, 1e-12)[3] == [0, 2]


def test_bk_block_numbering_follows_the_printed_diagrams():
    """The order in which the BK schedule generates its blocks (within a
    stage U-blocks first, then W-blocks) numbers them as Table 3's
    diagrams do; later stages take the first p columns of blocks by these
    numbers, so the order fixes the bases from stage 3 on."""
    with open(os.path.join(GOLD, "bk_block_numbering.json")) as f:
        gold = json.load(f)
    from oracle import bks_oracle as B
    done_u, done_w = set(), set()
    U, W = [], []
    for stage in range(1, 5):
        us, ws = B._stage_pairs("bk", stage, 100, 100, done_u, done_w)
        U += [(a, b) for a, b, _ in us]
        W += [(a, b) for a, b, _ in ws]
        assert [t for _, _, t in ws] == ([True] if stage == 1 else [False] * len(ws))
    assert [[a, b, k + 1] for k, (a, b) in enumerate(U)] == gold["U"]
    assert [[a, b, k + 1] for k, (a, b) in enumerate(W)] == gold["W"]


def test_schedule_tables():
    gold = _gold()
    for t in gold["tables"]:
        got = O.schedule_counts(t["r"], t["r"], len(t["stages"]), t["p"], t["variant"])
        for st, (want, have) in enumerate(zip(t["stages"], got)):
            if want[0] is not None:
                assert have[0] == want[0], (t["cite"], st + 1)
            assert have[1] == want[1], (t["cite"], st + 1)


def test_schedule_captions():
    for c in _gold()["captions"]:
        got = O.schedule_counts(c["r"], c["r"], c["s"], c["p"], c["variant"], n=c["n"])
        assert got[-1] == (c["k1"], c["k3"]), c["cite"]


def test_schedule_disagreements_are_the_rule_values():
    d = {x["cite"]: x for x in _gold()["disagree"]}
    assert O.schedule_counts(2, 2, 4, 4, "bk")[3][0] == 140
    assert O.schedule_counts(10, 10, 4, 4, "bk")[3][0] == 446
    assert O.schedule_counts(2, 2, 2, 4, "bk")[-1] == (20, 13)
    assert len(d) == 3


def _sym_case(seed, m=30, n=8, draws=400):
    c = synth.random_coo(seed, m, n, draws)
    return O.symmetrise(m, n, c.i, c.j, c.k, c.v)


@pytest.mark.parametrize("variant,s,p", [("bk", 2, 2), ("bk", 3, 2), ("min", 3, 2), ("max", 2, 0)])
def test_expand_counts_and_lemma1(variant, s, p):
    A = _sym_case(5)
    g = synth.rng(9)
    r = 2
    U0 = synth.orthonormal(g, A.m, r); W0 = synth.orthonormal(g, A.n, r)
    X, Z, info = O.expand(A, U0, W0, s, p, variant)
    want = O.schedule_counts(r, r, s, p, variant, m=A.m, n=A.n)[-1]
    assert (X.shape[1], Z.shape[1]) == want
    assert np.linalg.norm(X.T @ X - np.eye(X.shape[1])) < 1e-12
    assert np.linalg.norm(Z.T @ Z - np.eye(Z.shape[1])) < 1e-12
    assert np.allclose(X[:, :r], U0) and np.allclose(Z[:, :r], W0)
    # Lemma 1: A.(U_j, U0, W0) = 0 for blocks j >= 2 (columns past U0 and U1)
    k_u1 = r + r * r
    Hj = X[:, k_u1:].T @ O.mode1(A, U0, W0)
    assert np.linalg.norm(Hj) < 1e-12 * max(1.0, np.linalg.norm(O.mode1(A, U0, W0)))
    # and its mode-3 counterpart: A.(U0, U0, W_j) = 0 for j >= 2
    k_w1 = r + r * (r + 1) // 2
    Gj = Z[:, k_w1:].T @ O.mode3(A, U0)
    assert np.linalg.norm(Gj) < 1e-12 * max(1.0, np.linalg.norm(O.mode3(A, U0)))


def test_k3_cap():
    A = _sym_case(6, m=30, n=5, draws=500)
    g = synth.rng(1)
    U0 = synth.orthonormal(g, A.m, 3); W0 = synth.orthonormal(g, A.n, 3)
    X, Z, _ = O.expand(A, U0, W0, 2, 4, "bk")
    assert Z.shape[1] == 5
    assert np.linalg.norm(Z.T @ Z - np.eye(5)) < 1e-12
