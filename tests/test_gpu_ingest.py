"""Ingest (symmetrise / dedupe / sort) on the GPU vs the oracle, bitwise."""
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


@pytest.mark.parametrize("vdtype", [np.float32, np.float64])
@pytest.mark.parametrize("m,n,draws,seed", [(6, 3, 400, 0), (300, 100, 10_000, 1),
                                            (5000, 37, 60_000, 2), (1, 1, 50, 3)])
def test_ingest_bitwise(vdtype, m, n, draws, seed):
    bk = _bk()
    c = synth.random_coo(seed, m, n, draws, vdtype=vdtype)
    A = O.symmetrise(m, n, c.i, c.j, c.k, c.v, mirror=True)
    T = bk.bks_tensor_create_coo(m, n, c.i, c.j, c.k, c.v, mirror=True)
    assert T.nnz == A.nnz
    i, j, k, v = (x.cpu().numpy() for x in bk.bks_tensor_export_coo(T))
    assert np.array_equal(i, A.i) and np.array_equal(j, A.j) and np.array_equal(k, A.k)
    assert v.dtype == A.v.dtype and v.tobytes() == A.v.tobytes()
    assert abs(T.fro2 - A.fro2()) <= 1e-12 * max(1.0, A.fro2())


def test_ingest_zipf_duplicates_bitwise():
    bk = _bk()
    c = synth.zipf_tensor(5, 20_000, 17, 300_000, 1.2, values="absnormal", vdtype=np.float32)
    A = O.symmetrise(c.m, c.n, c.i, c.j, c.k, c.v)
    T = bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v)
    i, j, k, v = (x.cpu().numpy() for x in bk.bks_tensor_export_coo(T))
    assert np.array_equal(i, A.i) and np.array_equal(j, A.j) and np.array_equal(k, A.k)
    assert v.tobytes() == A.v.tobytes()


def test_ingest_device_input_and_validation():
    import torch
    bk = _bk()
    c = synth.random_coo(9, 40, 5, 700)
    A = O.symmetrise(40, 5, c.i, c.j, c.k, c.v)
    dev = [torch.tensor(x, device="cuda") for x in (c.i, c.j, c.k, c.v)]
    T = bk.bks_tensor_create_coo(40, 5, *dev, mirror=True)
    _, _, _, v = bk.bks_tensor_export_coo(T)
    assert v.cpu().numpy().tobytes() == A.v.tobytes()
    # both halves given explicitly: validation passes, then fails when broken
    T2 = bk.bks_tensor_create_coo(40, 5, A.i, A.j, A.k, A.v, mirror=False, validate=True)
    assert T2.nnz == A.nnz
    vb = A.v.copy()
    off = np.nonzero(A.i != A.j)[0][0]
    vb[off] += 1.0
    with pytest.raises(bk.BksError) as e:
        bk.bks_tensor_create_coo(40, 5, A.i, A.j, A.k, vb, mirror=False, validate=True)
    assert e.value.code == bk.BKS_EASYM


def test_ingest_errors_and_empty():
    bk = _bk()
    with pytest.raises(bk.BksError) as e:
        bk.bks_tensor_create_coo(4, 2, np.array([4]), np.array([0]), np.array([0]), np.array([1.0]))
    assert e.value.code == bk.BKS_EINVAL
    with pytest.raises(bk.BksError):
        bk.bks_tensor_create_coo(4, 2, np.array([0]), np.array([1]), np.array([2]), np.array([1.0]))
    with pytest.raises(bk.BksError):
        bk.bks_tensor_create_coo(0, 2, np.array([], np.int32), np.array([], np.int32),
                                 np.array([], np.int32), np.array([]))
    T = bk.bks_tensor_create_coo(4, 2, np.array([], np.int32), np.array([], np.int32),
                                 np.array([], np.int32), np.array([], np.float64))
    assert T.nnz == 0
