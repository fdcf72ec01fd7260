"""CPU oracle for the Block Krylov-Schur (BKS) / HOOI hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the CUDA library and its Python binding)
never calls it, and it shares no code with that path.

It is a plain, slow FP64 numpy restatement of the paper (Eldén & Dehghan,
"A Krylov-Schur like method for computing the best rank-(r1,r2,r3)
approximation of large and sparse tensors"):

* symmetrise / dedupe / canonical order of a sparse (1,2)-symmetric tensor
  (Definition 2.1; duplicate handling is this library's reading);
* the block contractions A.(X,Y)_{2,3}, A.(X,X')_{1,2} and the core
  A.(U,U,W) (Section 2.2, Algorithm 3 step (i), eq. (Rayleigh));
* block Gram-Schmidt + thin QR (Algorithm 3 steps (ii)-(iv), Appendix B);
* the BK / min-BK / max-BK block schedules (Tables 1-3, Algorithm 4);
* the G-gradient by Proposition 2 and in global coordinates (Section 2.5);
* the inner best rank-(r1,r1,r3) solve of the dense core (Section 6.2:
  truncated HOSVD + HOOI sweeps);
* the tensor Krylov-Schur outer loop (Algorithm 5) and HOOI (Section 6.1);
* the same method for a general l x m x n tensor with three bases
  (``bks_general_oracle``: Section 5, Proposition 2 with three terms).

Parity status per function is stated in ``bks_oracle``'s module docstring.
"""
from .bks_oracle import *  # noqa: F401,F403
from .bks_oracle import __all__ as _sym_all
from .bks_general_oracle import *  # noqa: F401,F403
from .bks_general_oracle import __all__ as _gen_all

__all__ = list(_sym_all) + list(_gen_all)
