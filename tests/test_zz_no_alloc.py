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
    import torch
    bk = _bk()
    tdt = getattr(torch, dtype)
    # long rows (cut into pieces: the partial-sum scratch is used) and a
    # power-law tensor; widths that split the Y columns into two chunks
    cases = [synth.random_coo(2, 50, 4, 30_000), synth.zipf_tensor(3, 20_000, 23, 200_000, 1.1)]
    tol = 1e-13 if dtype == "float64" else 1e-5
    for c in cases:
        T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v.astype(dtype))
        g = synth.rng(31)
        for p, q in [(3, 4), (5, 6), (1, 1)]:
            outs = []
            for call in range(2):   # two calls in a row share the scratch array
                X = torch.tensor(g.standard_normal((c.m, p)), device="cuda", dtype=tdt)
                Y = torch.tensor(g.standard_normal((c.n, q)), device="cuda", dtype=tdt)
                ref = bk.bks_contract_mode1(T, X, Y)
                out = torch.full((p * q, c.m), float("nan"), device="cuda", dtype=tdt).t()
                bk.bks_contract_mode1_noalloc(T, X, Y, out)
                torch.cuda.synchronize()
                r, o = ref.cpu().numpy(), out.cpu().numpy()
                assert np.all(np.isfinite(o))
                scale = max(1.0, float(np.abs(r).max()))
                assert float(np.abs(o - r).max()) <= tol * scale
                outs.append(o)
            assert not np.array_equal(outs[0], outs[1])  # different inputs, fresh results


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    bk = _bk()
    m = 1_200_000  # packed X alone: 1.2e6 rows x 8 doubles > 32 MiB
    c = synth.random_coo(5, m, 3, 1000)
    T = bk.bks_tensor_create_coo(m, 3, c.i, c.j, c.k, c.v)
    X = torch.zeros((m, 8), device="cuda", dtype=torch.float64)
    Y = torch.zeros((3, 2), device="cuda", dtype=torch.float64)
    out = torch.zeros((16, m), device="cuda", dtype=torch.float64).t()
    with pytest.raises(bk.BksError) as e:
        bk.bks_contract_mode1_noalloc(T, X, Y, out)
    assert e.value.code == bk.BKS_EUNSUPPORTED
    assert "scratch" in str(e.value)
