"""Checks at the benchmark's full sizes, in the launch configurations
`bench.py` times (GPU only).

* The mode-1 contraction on the 1e6 x 1e6 x 200 Zipf(1.2) tensor (60M
  one-sided draws, 48.5M stored, the (128, 2048) work plan): sampled output
  rows against the oracle's definition evaluated from the input list, FP64
  and FP32.
* The mixed-precision solve on the 1e5 x 1e5 x 50 Zipf(1.1) tensor (5.0M
  stored) with the benchmark's parameters: properties that hold at any
  size, evaluated by the oracle at the returned point (orthonormal bases,
  the core, the gradient below the tolerance, F symmetric, ||F|| <= ||A||).
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _bk():
    import paper_2012_07595_gb300 as bk
    return bk


def _sample_rows(coo, count, seed):
    """Rows of every weight: a few heavy ones (split into pieces), medium
    ones (one warp each), light ones (one lane each) and empty ones."""
    deg = np.bincount(coo.i, minlength=coo.m) + np.bincount(coo.j, minlength=coo.m)
    order = np.argsort(-deg, kind="stable")
    g = synth.rng(seed)
    heavy = order[200:210]                       # about 40k entries each: cut into pieces
    medium = order[g.integers(2_000, 50_000, count // 3)]
    light = order[g.integers(100_000, coo.m, count // 3)]
    empty = np.nonzero(deg == 0)[0][:4]
    return np.unique(np.concatenate([heavy, medium, light, empty]))


def test_mode1_full_size_sampled_rows():
    import torch
    bk = _bk()
    coo = synth.zipf_tensor(3, 1_000_000, 200, 60_000_000, 1.2, values="absnormal",
                            vdtype=np.float32)
    rows = _sample_rows(coo, 60, 7)
    g = synth.rng(8)
    # FP64 values for the FP64 check (duplicates are summed in the value
    # dtype at ingest), the FP32 input for the FP32 check
    for dt, p, q in ((torch.float64, 3, 4), (torch.float32, 4, 4)):
        vals = coo.v.astype(np.float64) if dt == torch.float64 else coo.v
        T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, vals)
        X = torch.tensor(g.standard_normal((coo.m, p)), device="cuda", dtype=dt)
        Y = torch.tensor(g.standard_normal((coo.n, q)), device="cuda", dtype=dt)
        got = bk.bks_contract_mode1(T, X, Y).cpu().numpy()[rows]
        Xh = X.cpu().double().numpy(); Yh = Y.cpu().double().numpy()
        ref = O.mode1_rows_from_input(coo.i, coo.j, coo.k, coo.v, Xh, Yh, rows)
        absref = O.mode1_rows_from_input(coo.i, coo.j, coo.k, np.abs(coo.v.astype(np.float64)),
                                         np.abs(Xh), np.abs(Yh), rows)
        if dt == torch.float64:
            bound = 1e-12 * absref + 1e-300
        else:
            # FP32 sums of at most a few thousand terms per row piece plus the
            # fixed-order piece reduction: well inside 1e-4 of the absolute sum
            bound = 1e-4 * absref + 1e-30
        assert np.all(np.abs(got - ref) <= bound), (dt, float(np.max(np.abs(got - ref) / (absref + 1e-300))))
        T.close()


def test_bench_solve_full_size_properties():
    import torch
    bk = _bk()
    from bench import WORKLOAD as w, make_input, start_matrices
    coo = make_input()
    A = O.symmetrise(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    U0h, W0h = start_matrices(w["m"], w["n"], w["r"])
    prm = bk.BksParams(r1=w["r"], r3=w["r"], stages=w["stages"], block_p=w["block_p"],
                       tol=w["tol"], precision=bk.BKS_PREC_MIXED, mixed_tol=w["mixed_tol"],
                       tol_scale_free=w["tol_scale_free"], refine_sweeps=50, max_outer=500)
    U, W, F, info = bk.bks_solve(T, prm, torch.tensor(U0h, device="cuda"),
                                 torch.tensor(W0h, device="cuda"))
    assert info["converged"]
    Uh, Wh, Fh = U.cpu().numpy(), W.cpu().numpy(), F.cpu().numpy()
    r = w["r"]
    assert np.abs(Uh.T @ Uh - np.eye(r)).max() < 1e-12
    assert np.abs(Wh.T @ Wh - np.eye(r)).max() < 1e-12
    gg, nf, Fo = O.gradient_global(A, Uh, Wh)
    assert abs(nf - info["normF"]) <= 1e-10 * nf
    assert np.allclose(Fh, Fo, rtol=0, atol=1e-10 * nf)
    assert np.allclose(Fo, Fo.transpose(1, 0, 2), rtol=0, atol=1e-12 * nf)
    assert nf ** 2 <= A.fro2() * (1 + 1e-12)
    # the scale-free test ||grad|| / ||F||^2 <= tol, evaluated by the oracle
    assert gg / nf ** 2 <= 2 * w["tol"]
    T.close()
