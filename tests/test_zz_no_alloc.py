"""bks_contract_mode1_noalloc -- the mode-1 contraction for callers that
cannot allocate device memory (for example a framework that has reserved the
whole device for its own pool) -- gives the same result as
bks_contract_mode1, call after call, while using the library's fixed device
scratch array instead of allocating.  Collected last on purpose."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _bk():
    import paper_2012_07595_gb300 as bk
    from paper_2012_07595_gb300 import _build
    _build.build()
    return bk


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_noalloc_matches_allocating_contraction_twice(dtype):
    """Bitwise the same output as bks_contract_mode1 (the same code path and
    kernels, only the temporaries live elsewhere), on two calls in a row."""
    import torch
    bk = _bk()
    tdt = getattr(torch, dtype)
    # long rows (cut into pieces: the partial-sum scratch is used) and a
    # power-law tensor; widths that split the Y columns into two chunks, and
    # the unpadded 3-column FP64 operands
    cases = [synth.random_coo(2, 50, 4, 30_000), synth.zipf_tensor(3, 20_000, 23, 200_000, 1.1)]
    for c in cases:
        T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v.astype(dtype))
        g = synth.rng(31)
        for p, q in [(3, 4), (4, 3), (3, 3), (5, 6), (1, 1), (8, 8)]:
            outs = []
            for call in range(2):   # two calls in a row share the scratch array
                X = torch.tensor(g.standard_normal((c.m, p)), device="cuda", dtype=tdt)
                Y = torch.tensor(g.standard_normal((c.n, q)), device="cuda", dtype=tdt)
                Xc = X.t().contiguous().t()
                Yc = Y.t().contiguous().t()
                ref = bk.bks_contract_mode1(T, Xc, Yc)
                out = torch.full((p * q, c.m), float("nan"), device="cuda", dtype=tdt).t()
                bk.bks_contract_mode1_noalloc(T, Xc, Yc, out)
                torch.cuda.synchronize()
                r, o = ref.cpu().numpy(), out.cpu().numpy()
                assert np.all(np.isfinite(o))
                assert np.array_equal(o, r), (p, q, float(np.abs(o - r).max()))
                outs.append(o)
            assert not np.array_equal(outs[0], outs[1])  # different inputs, fresh results


def test_noalloc_rejects_bad_operands_without_copying():
    """The wrapper allocates nothing: operands of the wrong shape, dtype or
    layout raise instead of being converted."""
    import torch
    bk = _bk()
    c = synth.random_coo(6, 40, 5, 800)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    X = torch.zeros((3, c.m), device="cuda", dtype=torch.float64).t()
    Y = torch.zeros((2, c.n), device="cuda", dtype=torch.float64).t()
    good = torch.zeros((6, c.m), device="cuda", dtype=torch.float64).t()
    bk.bks_contract_mode1_noalloc(T, X, Y, good)
    bad = [
        (X, Y, torch.zeros((5, c.m), device="cuda", dtype=torch.float64).t()),   # p*q columns
        (X, Y, torch.zeros((6, c.m), device="cuda", dtype=torch.float32).t()),   # dtype
        (X, Y, torch.zeros((c.m, 6), device="cuda", dtype=torch.float64)),       # row-major out
        (torch.zeros((c.m, 3), device="cuda", dtype=torch.float64), Y, good),    # row-major X
        (X, Y.float(), good),                                                     # Y dtype
        (X[:-1], Y, good),                                                        # rows
    ]
    for a, b, o in bad:
        with pytest.raises(ValueError):
            bk.bks_contract_mode1_noalloc(T, a, b, o)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    bk = _bk()
    m = 1_200_000  # packed X alone: 1.2e6 rows x 8 doubles > 32 MiB
    c = synth.random_coo(5, m, 3, 1000)
    T = bk.bks_tensor_create_coo(m, 3, c.i, c.j, c.k, c.v)
    X = torch.zeros((8, m), device="cuda", dtype=torch.float64).t()
    Y = torch.zeros((2, 3), device="cuda", dtype=torch.float64).t()
    out = torch.zeros((16, m), device="cuda", dtype=torch.float64).t()
    with pytest.raises(bk.BksError) as e:
        bk.bks_contract_mode1_noalloc(T, X, Y, out)
    assert e.value.code == bk.BKS_EUNSUPPORTED
    assert "scratch" in str(e.value)
