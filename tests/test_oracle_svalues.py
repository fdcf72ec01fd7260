"""Pins of the S-values (Section 2.6) and the slice normalisations
(Section 7) of the oracle (not GPU)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


def _brute_svalues(T, U, W):
    """S-values from the definitions with an explicit orthogonal complement
    and einsum on the dense tensor: F = T.(U,U,W), F_perp^1 = T.(U_perp,U,W),
    F_perp^3 = T.(U,U,W_perp)."""
    m, n = T.shape[0], T.shape[2]
    Qu, _ = np.linalg.qr(np.hstack([U, np.eye(m)]))
    Qw, _ = np.linalg.qr(np.hstack([W, np.eye(n)]))
    Up, Wp = Qu[:, U.shape[1]:m], Qw[:, W.shape[1]:n]
    F = np.einsum("ijk,ia,jb,kc->abc", T, U, U, W)
    F1p = np.einsum("ijk,ia,jb,kc->abc", T, Up, U, W)
    F3p = np.einsum("ijk,ia,jb,kc->abc", T, U, U, Wp)
    out = []
    for G, Gp, mode in ((F, F1p, 0), (F, F3p, 2)):
        Gk = np.moveaxis(G, mode, 0).reshape(G.shape[mode], -1)
        s = np.sqrt(np.maximum(np.linalg.eigvalsh(Gk @ Gk.T)[::-1], 0))
        Pk = np.moveaxis(Gp, mode, 0).reshape(Gp.shape[mode], -1)
        lam = np.linalg.eigvalsh(Pk @ Pk.T)[-1] if Pk.size else 0.0
        out.append(np.append(s, math.sqrt(max(lam, 0.0))))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_svalues_match_brute_force(seed):
    g = synth.rng(300 + seed)
    c = synth.random_coo(seed, 9, 5, 150)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    U = synth.orthonormal(g, 9, 3)
    W = synth.orthonormal(g, 5, 2)
    s1, s3, gap1, gap3 = O.s_values_gaps(A, U, W)
    b1, b3 = _brute_svalues(A.dense(), U, W)
    assert np.allclose(s1, b1, rtol=1e-12, atol=1e-12 * b1.max())
    assert np.allclose(s3, b3, rtol=1e-12, atol=1e-12 * b3.max())
    assert gap1 == pytest.approx(b1[-2] - b1[-1], abs=1e-12 * b1.max())
    assert gap3 == pytest.approx(b3[-2] - b3[-1], abs=1e-12 * b3.max())


def test_svalues_of_a_planted_exact_rank_tensor():
    """T = (U0,U0,W0).F0: at (U0, W0) the S-values are those of F0 and the
    (r+1)-st are zero (T.(U_perp,...) vanishes), so the gaps are s_r."""
    T, U0, W0, F0 = synth.dense_planted(7, m=12, n=6, r1=2, r3=2)
    c = synth.dense_to_coo(T)
    A = O.symmetrise(12, 6, c.i, c.j, c.k, c.v, mirror=False)
    s1, s3, gap1, gap3 = O.s_values_gaps(A, U0, W0)
    f = O.s_values(F0)
    scale = f[0][0]
    assert np.allclose(s1[:2], f[0], atol=1e-12 * scale)
    assert np.allclose(s3[:2], f[2], atol=1e-12 * scale)
    assert s1[2] < 1e-12 * scale and s3[2] < 1e-12 * scale
    assert gap1 == pytest.approx(f[0][1], abs=1e-12 * scale)


def test_svalues_invariant_under_a_change_of_basis():
    g = synth.rng(310)
    c = synth.random_coo(3, 11, 4, 200)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    U = synth.orthonormal(g, 11, 3)
    W = synth.orthonormal(g, 4, 2)
    Qa, _ = np.linalg.qr(g.standard_normal((3, 3)))
    Qb, _ = np.linalg.qr(g.standard_normal((2, 2)))
    a = O.s_values_gaps(A, U, W)
    b = O.s_values_gaps(A, U @ Qa, W @ Qb)
    assert np.allclose(a[0], b[0], rtol=1e-12) and np.allclose(a[1], b[1], rtol=1e-12)


def _graph_slice(edges, m, k):
    i = np.array([a for a, b in edges], dtype=np.int32)
    j = np.array([b for a, b in edges], dtype=np.int32)
    return i, j, np.full(i.shape, k, dtype=np.int32)


def test_slice_lmax_closed_forms():
    """Adjacency slices with known spectra: path P_m (2 cos(pi/(m+1))),
    cycle C_m (2), star K_{1,m-1} (sqrt(m-1)), complete K_m (m - 1); an
    empty slice has norm 0 and keeps scale 1."""
    m = 9
    path = [(a, a + 1) for a in range(m - 1)]
    cycle = path + [(m - 1, 0)]
    star = [(0, b) for b in range(1, m)]
    comp = [(a, b) for a in range(m) for b in range(a + 1, m)]
    parts = [_graph_slice(e, m, kk) for kk, e in enumerate((path, cycle, star, comp))]
    i = np.concatenate([p[0] for p in parts]); j = np.concatenate([p[1] for p in parts])
    k = np.concatenate([p[2] for p in parts])
    A = O.symmetrise(m, 5, i, j, k, np.ones(i.size))     # slice 4 empty
    lm = O.slice_norms(A, "lmax")
    want = [2 * math.cos(math.pi / (m + 1)), 2.0, math.sqrt(m - 1), m - 1.0, 0.0]
    assert np.allclose(lm, want, atol=1e-12)
    fro = O.slice_norms(A, "fro")
    assert np.allclose(fro, [math.sqrt(2 * len(e)) for e in (path, cycle, star, comp)] + [0.0])
    sc = O.slice_scales(lm)
    assert sc[4] == 1.0 and np.allclose(sc[:4], 1.0 / np.array(want[:4]))


def sc_max(B, A):
    a = np.abs(A.vf())
    return float(np.max(np.abs(B.vf())[a > 0] / a[a > 0])) if (a > 0).any() else 1.0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_scaled_slices_have_unit_norms_and_stay_symmetric(dtype):
    c = synth.random_coo(5, 30, 6, 900, vdtype=dtype)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    for kind in ("fro", "lmax"):
        B = O.scale_slices(A, O.slice_scales(O.slice_norms(A, kind)))
        assert B.v.dtype == dtype
        nb = O.slice_norms(B, kind)
        tol = 1e-6 if dtype == np.float32 else 1e-12
        assert np.allclose(nb[nb > 0], 1.0, atol=tol)
        # symmetric as far as the stored tensor is (duplicates summed in
        # input order make A(i,j,k) and A(j,i,k) differ by rounding)
        T, T0 = B.dense(), A.dense()
        asym0 = np.abs(T0 - T0.transpose(1, 0, 2)).max()
        assert np.abs(T - T.transpose(1, 0, 2)).max() <= 2 * asym0 * sc_max(B, A) + tol * np.abs(T).max()
    # a dict model of the Frobenius norms
    acc = {}
    for kk, x in zip(A.k.tolist(), A.vf().tolist()):
        acc[kk] = acc.get(kk, 0.0) + x * x
    fro = O.slice_norms(A, "fro")
    assert np.allclose(fro, [math.sqrt(acc.get(kk, 0.0)) for kk in range(A.n)], rtol=1e-14)
