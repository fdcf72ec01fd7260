"""S-values (Section 2.6) and slice normalisations (Section 7) on the GPU
against the oracle."""
import math

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


@pytest.mark.parametrize("r1,r3", [(3, 2), (5, 5), (8, 4), (1, 1)])
def test_s_values_match_the_oracle(r1, r3):
    import torch
    bk = _bk()
    c = synth.zipf_tensor(5, 3000, 23, 60_000, 1.1)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    g = synth.rng(400 + r1)
    U = synth.orthonormal(g, c.m, r1)
    W = synth.orthonormal(g, c.n, r3)
    s1, s3, gap1, gap3 = bk.bks_s_values(T, torch.tensor(U), torch.tensor(W))
    o1, o3, og1, og3 = O.s_values_gaps(A, U, W)
    scale = max(o1[0], o3[0])
    assert np.abs(s1 - o1).max() <= 1e-10 * scale, (s1, o1)
    assert np.abs(s3 - o3).max() <= 1e-10 * scale, (s3, o3)
    assert abs(gap1 - og1) <= 2e-10 * scale and abs(gap3 - og3) <= 2e-10 * scale


def test_s_values_of_a_planted_tensor_have_zero_tails():
    import torch
    bk = _bk()
    Td, U0, W0, F0 = synth.dense_planted(11, m=30, n=8, r1=2, r3=2)
    c = synth.dense_to_coo(Td)
    T = bk.bks_tensor_create_coo(30, 8, c.i, c.j, c.k, c.v, mirror=False)
    s1, s3, gap1, gap3 = bk.bks_s_values(T, torch.tensor(U0), torch.tensor(W0))
    f = O.s_values(F0)
    assert np.allclose(s1[:2], f[0], atol=1e-10 * f[0][0])
    assert np.allclose(s3[:2], f[2], atol=1e-10 * f[0][0])
    assert s1[2] <= 1e-7 * f[0][0] and s3[2] <= 1e-7 * f[0][0]


def test_s_values_at_a_converged_solve():
    """At a BKS result the mode-wise gaps say how well the subspaces are
    determined; the device values equal the oracle's at that point."""
    import torch
    bk = _bk()
    c = synth.zipf_tensor(9, 2000, 17, 40_000, 1.2)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    g = synth.rng(9)
    U0 = synth.orthonormal(g, c.m, 3)
    W0 = synth.orthonormal(g, c.n, 3)
    U, W, F, info = bk.bks_solve(T, bk.BksParams(r1=3, r3=3, stages=2, block_p=4, tol=1e-10),
                                 torch.tensor(U0), torch.tensor(W0))
    assert info["converged"]
    s1, s3, gap1, gap3 = bk.bks_s_values(T, U, W)
    o1, o3, og1, og3 = O.s_values_gaps(A, U.cpu().numpy(), W.cpu().numpy())
    assert np.abs(s1 - o1).max() <= 1e-9 * o1[0] and np.abs(s3 - o3).max() <= 1e-9 * o1[0]
    # the S-values of F are its singular values per mode: sum of squares = ||F||^2
    assert sum(s1[:-1] ** 2) == pytest.approx(info["normF"] ** 2, rel=1e-10)
    assert sum(s3[:-1] ** 2) == pytest.approx(info["normF"] ** 2, rel=1e-10)


def _graph_tensor(m):
    path = [(a, a + 1) for a in range(m - 1)]
    cycle = path + [(m - 1, 0)]
    star = [(0, b) for b in range(1, m)]
    comp = [(a, b) for a in range(m) for b in range(a + 1, m)]
    i, j, k = [], [], []
    for kk, edges in enumerate((path, cycle, star, comp)):
        for a, b in edges:
            i.append(a); j.append(b); k.append(kk)
    want = [2 * math.cos(math.pi / (m + 1)), 2.0, math.sqrt(m - 1), m - 1.0, 0.0, 0.0]
    return (np.array(i, np.int32), np.array(j, np.int32), np.array(k, np.int32),
            np.ones(len(i)), want)


@pytest.mark.parametrize("m", [9, 150])
def test_slice_lmax_closed_forms(m):
    bk = _bk()
    i, j, k, v, want = _graph_tensor(m)
    T = bk.bks_tensor_create_coo(m, 6, i, j, k, v)      # slices 4 and 5 empty
    lm = bk.bks_slice_norms(T, "lmax").cpu().numpy()
    assert np.allclose(lm, want, rtol=1e-10, atol=1e-12), (lm, want)
    fro = bk.bks_slice_norms(T, "fro").cpu().numpy()
    A = O.symmetrise(m, 6, i, j, k, v)
    assert np.allclose(fro, O.slice_norms(A, "fro"), rtol=1e-14, atol=0)


@pytest.mark.parametrize("vdtype", [np.float64, np.float32])
def test_slice_norms_match_the_oracle(vdtype):
    bk = _bk()
    c = synth.zipf_tensor(12, 300, 9, 6_000, 1.1, values="absnormal", vdtype=vdtype)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    fro = bk.bks_slice_norms(T, "fro").cpu().numpy()
    assert np.allclose(fro, O.slice_norms(A, "fro"), rtol=1e-13, atol=0)
    lm = bk.bks_slice_norms(T, "lmax").cpu().numpy()
    ol = O.slice_norms(A, "lmax")
    # FP32 duplicates summed in input order leave A(i,j,k) and A(j,i,k)
    # unequal by a rounding: the slices are symmetric to FP32 precision only
    rtol = 1e-9 if vdtype == np.float64 else 1e-6
    assert np.allclose(lm, ol, rtol=rtol, atol=0), np.abs(lm - ol).max()
    # signed values: the largest algebraic eigenvalue
    c2 = synth.random_coo(13, 200, 5, 3_000, vdtype=vdtype)
    A2 = O.symmetrise(c2.m, c2.n, c2.i, c2.j, c2.k, c2.v)
    T2 = bk.bks_tensor_create_coo(c2.m, c2.n, c2.i, c2.j, c2.k, c2.v)
    lm2 = bk.bks_slice_norms(T2, "lmax").cpu().numpy()
    assert np.allclose(lm2, O.slice_norms(A2, "lmax"), rtol=max(rtol, 1e-8), atol=0)


@pytest.mark.parametrize("vdtype", [np.float64, np.float32])
def test_scaled_tensor_is_bitwise_the_oracles_and_normalised(vdtype):
    import torch
    bk = _bk()
    c = synth.zipf_tensor(14, 500, 11, 8_000, 1.1, values="absnormal", vdtype=vdtype)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    scales = 1.0 / (np.arange(c.n) + 1.5)
    S = bk.bks_tensor_scale_slices(T, scales)
    B = O.scale_slices(A, scales)
    i, j, k, v = (x.cpu().numpy() for x in bk.bks_tensor_export_coo(S))
    assert np.array_equal(i, B.i) and np.array_equal(j, B.j) and np.array_equal(k, B.k)
    assert v.tobytes() == B.v.tobytes()
    for kind in ("fro", "lmax"):
        nrm = bk.bks_slice_norms(T, kind)
        sc = torch.where(nrm > 0, 1.0 / nrm, torch.ones_like(nrm))
        N = bk.bks_tensor_scale_slices(T, sc)
        after = bk.bks_slice_norms(N, kind).cpu().numpy()
        tol = 1e-6 if vdtype == np.float32 else 1e-12
        assert np.allclose(after[after > 0], 1.0, atol=tol), after
        N.close()
