"""The C-ABI library builds and exports every symbol include/bks.h declares
(no compute: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "bks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted({n for n in names if n.startswith(("bks_", "hooi_"))})


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["bks_tensor_create_coo", "bks_tensor_destroy", "bks_tensor_info",
                 "bks_tensor_export_coo", "bks_contract_mode1", "bks_contract_mode3", "bks_core",
                 "bks_solve", "hooi_solve", "bks_params_default", "hooi_params_default",
                 "bks_last_error_string"]:
        assert want in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2012_07595_gb300 import _build
    path = _build.build()
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_params_defaults_without_gpu():
    import paper_2012_07595_gb300 as bk
    p = bk._Params()
    bk.lib().bks_params_default(ctypes.byref(p))
    assert (p.r1, p.r3, p.stages, p.block_p) == (2, 2, 2, 4)
    assert p.tol == 1e-10 and p.drop_tol == 1e-14
    h = bk._HooiParams()
    bk.lib().hooi_params_default(ctypes.byref(h))
    assert h.grad_every == 10
    # the Python dataclass mirrors the C defaults
    d = bk.BksParams()
    assert (d.r1, d.r3, d.stages, d.block_p, d.tol, d.drop_tol) == (2, 2, 2, 4, 1e-10, 1e-14)
