"""Pins of the oracle's storage and contractions (not GPU)."""
import numpy as np
import pytest

import oracle as O
import synth


def dict_model(m, n, i, j, k, v, mirror=True):
    """Mirror rule written out with a dict: entries in input order, then the
    mirrors of the off-diagonal entries in input order; equal keys summed left
    to right in the value dtype; sorted by (i, j, k)."""
    seq = list(zip(i.tolist(), j.tolist(), k.tolist(), list(v)))
    if mirror:
        seq = seq + [(b, a, c, x) for (a, b, c, x) in seq if a != b]
    acc = {}
    for a, b, c, x in seq:
        key = (a, b, c)
        acc[key] = x if key not in acc else acc[key] + x
    keys = sorted(acc)
    return (np.array([t[0] for t in keys]), np.array([t[1] for t in keys]),
            np.array([t[2] for t in keys]), np.array([acc[t] for t in keys], dtype=v.dtype))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symmetrise_matches_dict_model_bitwise(dtype, seed):
    g = synth.rng(seed)
    m, n, N = 6, 3, 400          # small index ranges force many duplicates
    i = g.integers(0, m, N).astype(np.int32)
    j = g.integers(0, m, N).astype(np.int32)
    k = g.integers(0, n, N).astype(np.int32)
    v = g.standard_normal(N).astype(dtype)
    A = O.symmetrise(m, n, i, j, k, v, mirror=True)
    ri, rj, rk, rv = dict_model(m, n, i, j, k, v)
    assert np.array_equal(A.i, ri) and np.array_equal(A.j, rj) and np.array_equal(A.k, rk)
    assert A.v.dtype == dtype
    assert rv.tobytes() == A.v.tobytes()
    # the result is (1,2)-symmetric
    T = A.dense()
    assert np.allclose(T, T.transpose(1, 0, 2), rtol=0, atol=1e-5 if dtype == np.float32 else 1e-12)


def test_symmetrise_keeps_zeros_and_diagonal():
    i = np.array([0, 1, 1], np.int32); j = np.array([0, 2, 2], np.int32)
    k = np.array([0, 0, 0], np.int32); v = np.array([0.0, 1.0, -1.0])
    A = O.symmetrise(3, 1, i, j, k, v)
    # (0,0) diagonal not mirrored; (1,2) and (2,1) sum to exact zero but are kept
    assert A.nnz == 3
    assert list(zip(A.i, A.j)) == [(0, 0), (1, 2), (2, 1)]
    assert np.all(A.v == 0.0)
    # an explicit zero that is not the first key of the list keeps its own entry
    B = O.symmetrise(2, 1, np.array([0, 1]), np.array([1, 1]), np.array([0, 0]),
                     np.array([2.0, 0.0]))
    assert list(zip(B.i, B.j, B.v)) == [(0, 1, 2.0), (1, 0, 2.0), (1, 1, 0.0)]


def test_symmetrise_errors():
    with pytest.raises(ValueError):
        O.symmetrise(3, 2, np.array([3]), np.array([0]), np.array([0]), np.array([1.0]))
    with pytest.raises(ValueError):
        O.symmetrise(3, 2, np.array([0]), np.array([1]), np.array([2]), np.array([1.0]))
    with pytest.raises(ValueError):
        O.symmetrise(3, 2, np.array([0]), np.array([1]), np.array([0]), np.array([1.0]),
                     mirror=False, validate=True)
    A = O.symmetrise(3, 2, np.array([0, 1]), np.array([1, 0]), np.array([0, 0]),
                     np.array([2.5, 2.5]), mirror=False, validate=True)
    assert A.nnz == 2
    # both halves present, values one rounding apart: not (1,2)-symmetric
    with pytest.raises(ValueError):
        O.symmetrise(3, 2, np.array([0, 1]), np.array([1, 0]), np.array([0, 0]),
                     np.array([2.5, np.nextafter(2.5, 3.0)]), mirror=False, validate=True)


def test_empty():
    A = O.symmetrise(4, 2, np.array([], np.int32), np.array([], np.int32),
                     np.array([], np.int32), np.array([], np.float64))
    assert A.nnz == 0
    assert np.all(O.mode1(A, np.ones((4, 2)), np.ones((2, 2))) == 0)


def _dense_case(seed, m, n, binary=False):
    g = synth.rng(seed)
    T = g.standard_normal((m, m, n))
    if binary:
        T = (g.random((m, m, n)) < 0.3).astype(np.float64)
    T = T + T.transpose(1, 0, 2)
    T[g.random((m, m, n)) < 0.5] = 0.0
    T = T + T.transpose(1, 0, 2)          # zero pattern symmetric too
    c = synth.dense_to_coo(T)
    A = O.symmetrise(m, n, c.i, c.j, c.k, c.v, mirror=False)
    return T, A


@pytest.mark.parametrize("shape,binary", [((7, 5), False), ((9, 4), False), ((7, 5), True)])
def test_contractions_vs_einsum(shape, binary):
    m, n = shape
    T, A = _dense_case(3, m, n, binary)
    g = synth.rng(7)
    X = g.standard_normal((m, 3)); X2 = g.standard_normal((m, 4)); Y = g.standard_normal((n, 2))
    # mode-1: Out[i, a + p b] = sum_jk T[i,j,k] X[j,a] Y[k,b]
    ref1 = np.einsum("ijk,ja,kb->iab", T, X, Y).reshape(m, -1, order="F")
    assert np.allclose(O.mode1(A, X, Y), ref1, rtol=1e-13, atol=1e-12)
    ref3 = np.einsum("ijk,ia,jb->kab", T, X, X2).reshape(n, -1, order="F")
    assert np.allclose(O.mode3(A, X, X2), ref3, rtol=1e-13, atol=1e-12)
    full = np.einsum("ijk,ia,jb->kab", T, X, X)
    tri = O.mode3(A, X)
    for b in range(3):
        for a in range(b + 1):
            assert np.allclose(tri[:, O.tri_index(a, b)], full[:, a, b], rtol=1e-13, atol=1e-12)
    # symmetric tensor => full mode-3 with X2 = X is symmetric in (a, b)
    assert np.allclose(full, full.transpose(0, 2, 1), atol=1e-12)
    U = np.linalg.qr(g.standard_normal((m, 3)))[0]; W = np.linalg.qr(g.standard_normal((n, 2)))[0]
    F = O.core(A, U, W)
    assert np.allclose(F, O.core_dense_check(T, U, W), rtol=1e-13, atol=1e-12)
    assert np.allclose(F, F.transpose(1, 0, 2), atol=1e-12)
    assert np.sum(F * F) <= np.sum(T * T) * (1 + 1e-12)


def test_tri_index_layout():
    cols = [(a, b) for b in range(5) for a in range(b + 1)]
    assert [O.tri_index(a, b) for a, b in cols] == list(range(15))


def test_mode1_rows_from_input_matches_stored_tensor():
    """Row-sampled mode-1 values computed from the one-sided list equal the
    rows of the contraction of the stored (mirrored, summed) tensor; the
    input has duplicates and diagonal entries."""
    g = np.random.default_rng(5)
    m, n, N = 40, 6, 900
    i = g.integers(0, m, N); j = g.integers(0, m, N); k = g.integers(0, n, N)
    i[:50] = j[:50]                       # diagonal entries (not mirrored)
    i[50:100] = i[100:150]; j[50:100] = j[100:150]; k[50:100] = k[100:150]  # duplicates
    v = g.standard_normal(N)
    A = O.symmetrise(m, n, i, j, k, v)
    X = g.standard_normal((m, 3)); Y = g.standard_normal((n, 2))
    rows = np.array([0, 3, 17, 39, 22])
    got = O.mode1_rows_from_input(i, j, k, v, X, Y, rows)
    ref = O.mode1(A, X, Y)[rows]
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_openmp_contraction_loop_equals_the_oracle():
    """The benchmark's all-cores CPU column (the oracle's mode-1 loop in C
    with OpenMP) computes unfold_1 of A.(X,Y)_{2,3} like the numpy oracle."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from oracle import omp
    c = synth.zipf_tensor(12, 700, 9, 20_000, 1.1)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    g = synth.rng(13)
    for p, q in [(3, 4), (5, 5), (1, 1), (8, 8)]:
        X = g.standard_normal((A.m, p)); Y = g.standard_normal((A.n, q))
        got = omp.mode1_omp(A, X, Y)
        ref = O.mode1(A, X, Y)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert omp.threads() >= 1


def test_openmp_mode1_loop_matches_einsum():
    """The OpenMP build of the oracle's mode-1 loop (the all-cores column of
    the benchmark's CPU baseline) against the dense definition, on a dense
    tensor and on a sparse one with empty rows."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from oracle import omp
    try:
        omp.build()
    except RuntimeError as e:
        pytest.skip(f"OpenMP build failed: {e}")
    T, A = _dense_case(3, 9, 5, False)
    g = synth.rng(8)
    for p, q in [(1, 1), (3, 2), (4, 4)]:
        X = g.standard_normal((9, p)); Y = g.standard_normal((5, q))
        ref = np.einsum("ijk,ja,kb->iab", T, X, Y).reshape(9, -1, order="F")
        assert np.allclose(omp.mode1_omp(A, X, Y), ref, rtol=1e-13, atol=1e-12)
    c = synth.random_coo(9, 40, 6, 15)
    S = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    assert np.unique(S.i).size < 40             # some rows are empty
    X = g.standard_normal((40, 3)); Y = g.standard_normal((6, 4))
    ref = np.einsum("ijk,ja,kb->iab", S.dense(), X, Y).reshape(40, -1, order="F")
    assert np.allclose(omp.mode1_omp(S, X, Y), ref, rtol=1e-13, atol=1e-12)
