"""Plain FP64 numpy oracle of the BKS / HOOI hot path (test infrastructure).

Only tests, the smoke check and the benchmark's CPU-baseline legs use this
module.  Every function cites the passage of the paper it follows.

Pins (what fixes each function other than itself) live in
``tests/test_oracle_*.py``:

* ``symmetrise``          -- dict model of the mirror/sum rule, bitwise;
                             explicit zeros kept; validation refuses values
                             one rounding apart.
* ``mode1/mode3/core``    -- brute-force dense ``einsum`` on tiny tensors.
* ``mode1_rows_from_input`` -- equals the rows of ``mode1`` of the stored
                             tensor (duplicates, diagonal entries, mirrors).
* ``orth_block``          -- orthonormality, reconstruction B = Q H + Qn R,
                             exact rank drops on planted dependent columns;
                             near dependence the projected block orthogonal
                             to Q to working precision (two rounds); the
                             same kept columns at any scale (relative drop).
* ``schedule_counts``     -- every k1/k3 printed in Tables 1-3 and in the
                             figure captions of Section 6.2 (three printed
                             values disagree with the rule; see the tests);
                             the BK block numbering printed in Table 3's
                             diagrams.
* ``gradient_prop2``      -- equals ``gradient_global`` (two derivations).
* ``hosvd_truncated``     -- returns the exact factor subspaces of a core of
                             exact multilinear rank (U,U,W).F0.
* ``sin_theta_max``       -- sin of a known planted principal angle.
* ``ng_model``/``ng_step`` -- finite differences of the pulled-back
                             objective; quadratic convergence; the same
                             optimum as HOOI; the safeguard refuses a step
                             that lowers ||F||.
* ``s_values_gaps``        -- brute force with an explicit orthogonal
                             complement and einsum; S-values of a planted
                             exact-rank tensor are those of F0 with zero
                             (r+1)-st values; invariance under a change of
                             basis.
* ``slice_norms``/``scale_slices`` -- closed-form largest eigenvalues of
                             path, cycle, star and complete graphs; the
                             Frobenius norm by a dict sum; scaled slices
                             have unit norm and stay (1,2)-symmetric.
* ``inner_solve``/``bks``/``hooi`` -- closed forms n=1 (Eckart-Young) and
                             rank-one slices, exact recovery of a planted
                             multilinear-rank tensor, monotone ||F||, and
                             BKS/HOOI agreement; the five start sweeps
                             counted; the inner and HOOI gradients equal
                             ``gradient_global``; HOOI's gradient every 10
                             iterations and W from the new U.

``tests/test_oracle_mutations.py`` plants one plausible mistake at a time
in a copy of this package and checks that the named pin catches it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "SymTensor", "symmetrise", "mode1", "mode3", "core", "core_dense_check",
    "orth_block", "schedule_counts", "expand", "gradient_prop2", "mode1_rows_from_input",
    "gradient_global", "inner_solve", "bks", "hooi", "sin_theta_max",
    "top_left_singular", "unfold1", "unfold3", "s_values", "tri_index",
    "BKSResult", "hosvd_truncated", "INNER_INIT_SWEEPS", "ng_model", "ng_step",
    "s_values_gaps", "slice_norms", "slice_scales", "scale_slices",
]


# ----------------------------------------------------------------------------
# Storage (Definition 2.1: A(i,j,k) = A(j,i,k))
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SymTensor:
    """Canonical stored form: entries sorted by (i, j, k), duplicates summed,
    both halves present.  ``v`` keeps the input value dtype (the sums are
    taken in that dtype); arithmetic below promotes to float64."""
    m: int
    n: int
    i: np.ndarray
    j: np.ndarray
    k: np.ndarray
    v: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.i.shape[0])

    def vf(self) -> np.ndarray:
        return self.v.astype(np.float64)

    def fro2(self) -> float:
        x = self.vf()
        return float(np.dot(x, x))

    def dense(self) -> np.ndarray:
        T = np.zeros((self.m, self.m, self.n))
        np.add.at(T, (self.i, self.j, self.k), self.vf())
        return T


def symmetrise(m, n, i, j, k, v, mirror=True, validate=False) -> SymTensor:
    """Store a (1,2)-symmetric tensor (Definition 2.1).

    The paper does not say how a sparse list becomes (1,2)-symmetric; this
    library's reading: with ``mirror`` the stored list is every input entry
    in input order followed by the mirror (j, i, k, v) of every input entry
    with i != j, again in input order (diagonal entries are not mirrored).
    The list is stably sorted by the key (i, j, k) and entries with equal
    keys are summed left to right in the value dtype; exact zeros are kept.
    Without ``mirror`` the input must already hold both halves; with
    ``validate`` the summed tensor must satisfy A(i,j,k) == A(j,i,k)
    bitwise, else ValueError.
    """
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    v = np.asarray(v)
    if m <= 0 or n <= 0:
        raise ValueError("m and n must be positive")
    if i.size and (i.min() < 0 or j.min() < 0 or k.min() < 0 or i.max() >= m
                   or j.max() >= m or k.max() >= n):
        raise ValueError("index out of range")
    if mirror:
        off = i != j
        ii = np.concatenate([i, j[off]])
        jj = np.concatenate([j, i[off]])
        kk = np.concatenate([k, k[off]])
        vv = np.concatenate([v, v[off]])
    else:
        ii, jj, kk, vv = i, j, k, v
    order = np.lexsort((kk, jj, ii))          # stable: primary i, then j, then k
    ii, jj, kk, vv = ii[order], jj[order], kk[order], vv[order]
    if ii.size == 0:
        return SymTensor(m, n, ii.astype(np.int32), jj.astype(np.int32),
                         kk.astype(np.int32), vv.copy())
    new = np.ones(ii.size, dtype=bool)
    new[1:] = (ii[1:] != ii[:-1]) | (kk[1:] != kk[:-1]) | (jj[1:] != jj[:-1])
    starts = np.nonzero(new)[0]
    lengths = np.diff(np.append(starts, ii.size))
    # left-to-right sum inside each run of equal keys, in the value dtype:
    # acc = v[s]; acc = acc + v[s+1]; ... (one vector step per position)
    acc = vv[starts].copy()
    for d in range(1, int(lengths.max())):
        sel = lengths > d
        acc[sel] = acc[sel] + vv[starts[sel] + d]
    out = SymTensor(m, n, ii[starts].astype(np.int32), jj[starts].astype(np.int32),
                    kk[starts].astype(np.int32), acc)
    if validate:
        key = {}
        for a, b, c, x in zip(out.i.tolist(), out.j.tolist(), out.k.tolist(),
                              out.v.tolist()):
            key[(a, b, c)] = x
        for (a, b, c), x in key.items():
            y = key.get((b, a, c))
            if y is None or np.float64(y).tobytes() != np.float64(x).tobytes():
                raise ValueError("input is not (1,2)-symmetric")
    return out


# ----------------------------------------------------------------------------
# Contractions (Section 2.2; Algorithm 3 step (i); Section 4.3.1)
# ----------------------------------------------------------------------------
def tri_index(a: int, b: int) -> int:
    """Column of the pair a <= b in triunfold_3 (Section 4.3.1): the upper
    triangle in column-major order, a + b(b+1)/2."""
    assert a <= b
    return a + b * (b + 1) // 2


def mode1(A: SymTensor, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """unfold_1 of A.(X,Y)_{2,3} (Algorithm 3 step (i)):
    Out[i, a + p*b] = sum over stored (i,j,k) of v * X[j,a] * Y[k,b].
    X is m x p, Y is n x q; Out is m x (p*q)."""
    p, q = X.shape[1], Y.shape[1]
    out = np.zeros((A.m, p * q))
    v = A.vf()
    for b in range(q):
        vy = v * Y[A.k, b]
        for a in range(p):
            out[:, a + p * b] = np.bincount(A.i, weights=vy * X[A.j, a], minlength=A.m)
    return out


def mode1_rows_from_input(i, j, k, v, X: np.ndarray, Y: np.ndarray, rows) -> np.ndarray:
    """Selected rows of unfold_1(A.(X,Y)_{2,3}) (Algorithm 3 step (i)) for
    the tensor that `symmetrise(..., mirror=True)` stores from the one-sided
    list (i, j, k, v), computed from the list itself: the stored tensor is
    the input entries plus the mirror (j, i, k, v) of every entry with
    i != j, with equal keys summed, and the contraction is linear in the
    stored values, so
        Out[r, a + p*b] = sum_{e: i_e = r} v_e X[j_e,a] Y[k_e,b]
                        + sum_{e: j_e = r, i_e != j_e} v_e X[i_e,a] Y[k_e,b].
    For checks at sizes where forming the stored tensor on the host is too
    slow.  Returns len(rows) x (p*q)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    p, q = X.shape[1], Y.shape[1]
    order = np.argsort(rows)
    srt = rows[order]
    out = np.zeros((rows.size, p * q))
    # the input entries (row i_e) and the mirrors (row j_e, i_e != j_e)
    for r_idx, c_idx, keep in ((i, j, np.ones(i.shape, dtype=bool)), (j, i, i != j)):
        sel = np.isin(r_idx, rows) & keep
        if not sel.any():
            continue
        slot = order[np.searchsorted(srt, r_idx[sel])]
        contrib = np.einsum("ea,eb->eba", v[sel][:, None] * X[c_idx[sel]], Y[k[sel]])
        np.add.at(out, slot, contrib.reshape(slot.size, p * q))
    return out


def mode3(A: SymTensor, X: np.ndarray, X2: np.ndarray | None = None) -> np.ndarray:
    """unfold_3 of A.(X,X2)_{1,2} (Section 4.3.1).  Full form:
    Out[k, a + p*b] = sum v * X[i,a] * X2[j,b]  (n x p*q).
    Triangle form (X2 is None, i.e. X2 = X): only the columns a <= b of the
    full form, at column a + b(b+1)/2 (triunfold_3)."""
    v = A.vf()
    p = X.shape[1]
    if X2 is None:
        out = np.zeros((A.n, p * (p + 1) // 2))
        for b in range(p):
            vb = v * X[A.j, b]
            for a in range(b + 1):
                out[:, tri_index(a, b)] = np.bincount(A.k, weights=vb * X[A.i, a],
                                                      minlength=A.n)
        return out
    q = X2.shape[1]
    out = np.zeros((A.n, p * q))
    for b in range(q):
        vb = v * X2[A.j, b]
        for a in range(p):
            out[:, a + p * b] = np.bincount(A.k, weights=vb * X[A.i, a], minlength=A.n)
    return out


def core(A: SymTensor, U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """F = A.(U,U,W) (eq. (Rayleigh)), r1 x r1 x r3 with
    F[a,b,c] = sum v U[i,a] U[j,b] W[k,c].  Computed as U^T (A.(U,W)_{2,3})
    (mode products in different modes commute, Section 2.2)."""
    r1, r3 = U.shape[1], W.shape[1]
    M = mode1(A, U, W)                     # m x (r1*r3), column b + r1*c
    F1 = U.T @ M                           # unfold_1(F): r1 x (r1*r3)
    return F1.reshape(r1, r1, r3, order="F")


def core_dense_check(T: np.ndarray, U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Brute force A.(U,U,W) on a dense array (the definition of Section 2.2)."""
    return np.einsum("ijk,ia,jb,kc->abc", T, U, U, W, optimize=True)


def unfold1(F: np.ndarray) -> np.ndarray:
    """Mode-1 unfolding, column index b + r2*c (first remaining index fastest)."""
    return F.reshape(F.shape[0], -1, order="F")


def unfold3(F: np.ndarray) -> np.ndarray:
    """Mode-3 unfolding, column index a + r1*b."""
    return F.reshape(-1, F.shape[2], order="F").T


# ----------------------------------------------------------------------------
# Block Gram-Schmidt + thin QR (Algorithm 3 (ii)-(iv), Appendix B)
# ----------------------------------------------------------------------------
def orth_block(Q: np.ndarray, B: np.ndarray, drop_tol: float, max_total: int | None = None):
    """Orthogonalise the new block B (m x b) against the orthonormal basis
    Q (m x K) and orthonormalise it (Algorithm 3 steps (ii)-(iv); Appendix B
    replaces the tensor form by a QR of the matrix form).

    Reading of this library: the block is projected against Q twice
    (classical Gram-Schmidt with one reorthogonalisation); then its columns
    are orthonormalised left to right, each projected twice against Q and
    the new columns kept so far.  A column is dropped when its residual
    norm is not above ``drop_tol`` times its raw norm, or when it would take
    the basis past ``max_total`` columns.

    Returns (Qn, H, R, kept, P): B = Q H + Qn R up to the dropped
    residuals, H is K x b, R is b' x b (b' = len(kept)) with R[t, c] = 0
    whenever kept[t] > c, and P = B - Q H, the projected block (equal to
    Qn R when no column is dropped).
    """
    m, b = B.shape
    K = Q.shape[1]
    raw = np.linalg.norm(B, axis=0)
    H = np.zeros((K, b))
    Bt = B.copy()
    for _ in range(2):
        h = Q.T @ Bt
        Bt -= Q @ h
        H += h
    Pb = Bt.copy()
    cap = b if max_total is None else max(0, min(b, max_total - K))
    cols, kept = [], []
    R = np.zeros((b, b))
    for c in range(b):
        x = Bt[:, c].copy()
        P = np.concatenate([Q] + [cc[:, None] for cc in cols], axis=1)
        g = np.zeros(P.shape[1])
        for _ in range(2):
            h = P.T @ x
            x -= P @ h
            g += h
        H[:, c] += g[:K]
        R[: len(cols), c] = g[K:]
        nx = float(np.linalg.norm(x))
        if len(cols) < cap and raw[c] > 0.0 and nx > drop_tol * raw[c]:
            R[len(cols), c] = nx
            cols.append(x / nx)
            kept.append(c)
    bp = len(cols)
    Qn = np.stack(cols, axis=1) if cols else np.zeros((m, 0))
    return Qn, H, R[:bp].copy(), kept, Pb


# ----------------------------------------------------------------------------
# Block schedules (Tables 1-3, Algorithm 4, Section 4.3.4)
# ----------------------------------------------------------------------------
def _stage_pairs(variant: str, stage: int, nU: int, nW: int, done_u: set, done_w: set):
    """The (left, right, triangle) block pairs of one stage, U-blocks first
    then W-blocks, each list in the order of the paper's diagrams.

    BK (Table 3): stage 1 uses (U0,W0) and the triangle (U0,U0).  At stage
    t >= 2 with q = t-1 the U-blocks come from (U0,Wq), (Uq,W0), (U1,Wq),
    (Uq,W1), ..., (U_{q-1},Wq), (Uq,W_{q-1}) (the diagonal (Uq,Wq) is left
    out) and the W-blocks from (U0,Uq), (U1,Uq), ..., (U_{q-1},Uq).  Blocks
    are numbered in generation order; bars (first p columns) are applied by
    the caller.
    min-BK (Algorithm 4, Table 1): stage t uses (U_{t-1},W_{t-1}) and the
    triangle (U_{t-1},U_{t-1}).
    max-BK (Table 2): every not yet used pair of whole blocks that exist at
    the start of the stage, by shells max(i,j) = s with (i,s),(s,i) for
    i < s then (s,s); W pairs i <= j, diagonal pairs as triangles.
    """
    us, ws = [], []
    if stage == 1:
        return [(0, 0, False)], [(0, 0, True)]
    if variant == "bk":
        q = stage - 1
        if q >= nU or q >= nW:
            return [], []
        for t in range(q):
            us.append((t, q, False))
            us.append((q, t, False))
        for t in range(q):
            ws.append((t, q, False))
        return us, ws
    if variant == "min":
        q = stage - 1
        if q >= nU or q >= nW:
            return [], []
        return [(q, q, False)], [(q, q, True)]
    if variant == "max":
        top = max(nU, nW)
        for s in range(top):
            for t in range(s):
                for (a, b_) in ((t, s), (s, t)):
                    if a < nU and b_ < nW and (a, b_) not in done_u:
                        us.append((a, b_, False))
            if s < nU and s < nW and (s, s) not in done_u:
                us.append((s, s, False))
        for s in range(nU):
            for t in range(s + 1):
                if (t, s) not in done_w:
                    ws.append((t, s, t == s))
        return us, ws
    raise ValueError(variant)


def schedule_counts(r1: int, r3: int, s: int, p: int, variant: str = "bk",
                    m: int | None = None, n: int | None = None):
    """(k1, k3) after each of the s stages when no column is dropped, with
    the caps k1 <= m and k3 <= n of Section 4.3.4 (bookkeeping of Tables
    1-3).  Bars take min(p, width) leading columns except for U0 and W0,
    which are always used whole (Section 4.3.2)."""
    uw, ww = [r1], [r3]
    done_u, done_w = set(), set()
    out = []
    k1, k3 = r1, r3
    for st in range(1, s + 1):
        us, ws = _stage_pairs(variant, st, len(uw), len(ww), done_u, done_w)
        nu, nw = list(uw), list(ww)
        for (a, b_, _) in us:
            wa = _bar(variant, a, uw[a], p)
            wb = _bar(variant, b_, ww[b_], p)
            cols = wa * wb
            if m is not None:
                cols = max(0, min(cols, m - k1))
            nu.append(cols)
            k1 += cols
            done_u.add((a, b_))
        for (a, b_, tri) in ws:
            wa = _bar(variant, a, uw[a], p)
            wb = _bar(variant, b_, uw[b_], p)
            cols = wa * (wa + 1) // 2 if tri else wa * wb
            if n is not None:
                cols = max(0, min(cols, n - k3))
            nw.append(cols)
            k3 += cols
            done_w.add((a, b_))
        uw, ww = nu, nw
        out.append((k1, k3))
    return out


def _bar(variant, idx, width, p):
    if variant == "max" or idx == 0:
        return width
    return min(p, width)


def expand(A: SymTensor, U0: np.ndarray, W0: np.ndarray, s: int, p: int,
           variant: str = "bk", drop_tol: float = 1e-14):
    """Expand (U0, W0) to the bases X = [U0 U1 ...] (m x k1) and
    Z = [W0 W1 ...] (n x k3) with s stages of the chosen block schedule
    (Algorithm 5 steps (iii) and (v)).  Within a stage all U-blocks are made
    first, then all W-blocks, each in diagram order; every contraction of a
    stage uses only blocks that existed when the stage began.

    Returns (X, Z, info) with info holding the stage-1 factors used by
    Proposition 2: H1 = U0^T A.(U0,W0)_{2,3}, R1 (its residual's R factor),
    H3 and R3 for the triangle (U0,U0) block.
    """
    m, n = A.m, A.n
    Ub = [U0.copy()]
    Wb = [W0.copy()]
    X = U0.copy()
    Z = W0.copy()
    done_u, done_w = set(), set()
    info = {}
    for st in range(1, s + 1):
        us, ws = _stage_pairs(variant, st, len(Ub), len(Wb), done_u, done_w)
        newU, newW = [], []
        for (a, b_, _) in us:
            L = Ub[a] if (variant == "max" or a == 0) else Ub[a][:, :p]
            Rr = Wb[b_] if (variant == "max" or b_ == 0) else Wb[b_][:, :p]
            done_u.add((a, b_))
            if L.shape[1] == 0 or Rr.shape[1] == 0:
                newU.append(np.zeros((m, 0)))
                continue
            Bm = mode1(A, L, Rr)
            Qn, H, R, kept, P = orth_block(X, Bm, drop_tol, max_total=m)
            if st == 1:
                info["H1"], info["R1"], info["P1"] = H, R, P
            X = np.concatenate([X, Qn], axis=1)
            newU.append(Qn)
        for (a, b_, tri) in ws:
            L = Ub[a] if (variant == "max" or a == 0) else Ub[a][:, :p]
            Rr = Ub[b_] if (variant == "max" or b_ == 0) else Ub[b_][:, :p]
            done_w.add((a, b_))
            if L.shape[1] == 0 or Rr.shape[1] == 0:
                newW.append(np.zeros((n, 0)))
                continue
            Bm = mode3(A, L) if tri else mode3(A, L, Rr)
            Qn, H, R, kept, P = orth_block(Z, Bm, drop_tol, max_total=n)
            if st == 1:
                info["H3"], info["R3"], info["P3"] = H, R, P
            Z = np.concatenate([Z, Qn], axis=1)
            newW.append(Qn)
        Ub.extend(newU)
        Wb.extend(newW)
        if st == 1:
            info["stage1_done"] = True
    return X, Z, info


# ----------------------------------------------------------------------------
# Gradient (Section 2.5; Proposition 2)
# ----------------------------------------------------------------------------
def _tri_weights_F3(F: np.ndarray) -> np.ndarray:
    """r3 x r1(r1+1)/2 matrix with column tri(a,b) = w_ab * F[a,b,:],
    w_aa = 1, w_ab = 2 (a < b): the mode-3 partial contraction of F with a
    (1,2)-symmetric tensor stored as its triangle."""
    r1, _, r3 = F.shape
    out = np.zeros((r3, r1 * (r1 + 1) // 2))
    for b in range(r1):
        for a in range(b + 1):
            out[:, tri_index(a, b)] = (1.0 if a == b else 2.0) * F[a, b, :]
    return out


def gradient_prop2(H1, P1, P3, r1, r3):
    """||grad|| and ||F|| at (U0,U0,W0) from the first block-Krylov step
    (Proposition 2).  H1 = unfold_1(F) = U0^T A.(U0,W0)_{2,3} (r1 x r1 r3)
    and P1 = U1 R1 is the projected mode-1 block, so the mode-1 term
    ||<H0, H1^1>_{-1}|| = ||H1 R1^T|| = ||P1 H1^T||; the mode-3 term is
    ||P3 F3w^T|| with P3 = W1 R3 the projected triangle block and F3w the
    weighted triangle of F.  Evaluating through P rather than R keeps the
    mass of columns the QR dropped.  For a (1,2)-symmetric tensor the
    mode-2 term equals the mode-1 term, hence
    ||grad||^2 = 2 ||P1 H1^T||^2 + ||P3 F3w^T||^2 (this library's reading
    of Proposition 2 with V = U)."""
    F = H1.reshape(r1, r1, r3, order="F")
    F3w = _tri_weights_F3(F)
    g1 = float(np.linalg.norm(P1 @ H1.T))
    g3 = float(np.linalg.norm(P3 @ F3w.T))
    grad = math.sqrt(2.0 * g1 * g1 + g3 * g3)
    return grad, float(np.linalg.norm(F)), F


def gradient_global(A: SymTensor, U: np.ndarray, W: np.ndarray):
    """||grad||, ||F|| in global coordinates (Section 2.5):
    mode 1: (I - U U^T) Gamma1, Gamma1 = <A.(U,W)_{2,3}, F>_{-1};
    mode 3: (I - W W^T) Gamma3, Gamma3 = <A.(U,U)_{1,2}, F>_{-3};
    mode 2 equals mode 1 by (1,2)-symmetry."""
    r1, r3 = U.shape[1], W.shape[1]
    T1 = mode1(A, U, W)
    F1 = U.T @ T1
    F = F1.reshape(r1, r1, r3, order="F")
    G1 = T1 @ F1.T
    G1 -= U @ (U.T @ G1)
    T3 = mode3(A, U, U)                    # n x r1^2, column a + r1*b
    G3 = T3 @ unfold3(F).T
    G3 -= W @ (W.T @ G3)
    g = math.sqrt(2.0 * np.linalg.norm(G1) ** 2 + np.linalg.norm(G3) ** 2)
    return g, float(np.linalg.norm(F)), F


def s_values(F: np.ndarray):
    """S-values of Section 2.6: s_i^(k) = sqrt(lambda_i(<F,F>_{-k}))."""
    out = []
    for k in range(3):
        Fk = np.moveaxis(F, k, 0).reshape(F.shape[k], -1)
        ev = np.linalg.eigvalsh(Fk @ Fk.T)[::-1]
        out.append(np.sqrt(np.maximum(ev, 0.0)))
    return out


def s_values_gaps(A: SymTensor, U: np.ndarray, W: np.ndarray):
    """S-values and gaps of Section 2.6 at (U, U, W).

    For k = 1 and 3 (mode 2 equals mode 1 by the (1,2)-symmetry):
    s_i^(k) = sqrt(lambda_i(<F,F>_{-k})), i <= r_k, and
    s_{r_k+1}^(k) = sqrt(lambda_max(<F_perp^k, F_perp^k>_{-k})) with
    F_perp^1 = A.(U_perp, U, W) and F_perp^3 = A.(U, U, W_perp)
    (Section 2.5), (U U_perp) orthogonal.  unfold_1(F_perp^1) is
    U_perp^T T1 with T1 = unfold_1(A.(I, U, W)) (m x r1 r3), so
    lambda_max(<F_perp^1, F_perp^1>_{-1}) = ||(I - U U^T) T1||_2^2; likewise
    mode 3 with T3 = unfold_3(A.(U, U, I)) (n x r1^2).  Returns
    (s1, s3, gap1, gap3), s1 holding r1 + 1 values and s3 r3 + 1, and
    gap_k = s_{r_k}^(k) - s_{r_k+1}^(k)."""
    T1 = mode1(A, U, W)
    F = (U.T @ T1).reshape(U.shape[1], U.shape[1], W.shape[1], order="F")
    sv = s_values(F)
    P1 = T1 - U @ (U.T @ T1)
    P3 = mode3(A, U, U)
    P3 = P3 - W @ (W.T @ P3)
    s1 = np.append(sv[0], np.linalg.norm(P1, 2) if P1.size else 0.0)
    s3 = np.append(sv[2], np.linalg.norm(P3, 2) if P3.size else 0.0)
    return s1, s3, float(s1[-2] - s1[-1]), float(s3[-2] - s3[-1])


# ----------------------------------------------------------------------------
# Slice normalisation (Section 7: slices of an adjacency tensor scaled so that
# the largest eigenvalue of each is 1, or to unit Frobenius norm)
# ----------------------------------------------------------------------------
def slice_norms(A: SymTensor, kind: str) -> np.ndarray:
    """Per frontal slice A(:,:,k) (a symmetric m x m matrix): "fro" the
    Frobenius norm, "lmax" the largest eigenvalue (algebraic; for the
    nonnegative slices of an adjacency tensor it is the spectral radius),
    from the library eigensolver on the dense slice."""
    out = np.zeros(A.n)
    x = A.vf()
    for kk in range(A.n):
        sel = A.k == kk
        if kind == "fro":
            out[kk] = math.sqrt(float(np.dot(x[sel], x[sel])))
        elif kind == "lmax":
            if not sel.any():
                continue
            S = np.zeros((A.m, A.m))
            np.add.at(S, (A.i[sel], A.j[sel]), x[sel])
            out[kk] = float(np.linalg.eigvalsh(S)[-1])
        else:
            raise ValueError(kind)
    return out


def slice_scales(norms: np.ndarray) -> np.ndarray:
    """Scale factor per slice: 1 / norm where the norm is positive, else 1
    (an empty slice, or a slice whose largest eigenvalue is not positive,
    keeps its values; this library's reading, the paper normalises
    adjacency slices only)."""
    norms = np.asarray(norms, dtype=np.float64)
    sc = np.ones_like(norms)
    pos = norms > 0
    sc[pos] = 1.0 / norms[pos]
    return sc


def scale_slices(A: SymTensor, scales: np.ndarray) -> SymTensor:
    """The stored tensor with slice k multiplied by scales[k]: each value
    times its scale, rounded once to the value dtype (the order and the
    entries are unchanged, so the result is still (1,2)-symmetric)."""
    sc = np.asarray(scales, dtype=np.float64)[A.k]
    v = (A.vf() * sc).astype(A.v.dtype)
    return SymTensor(A.m, A.n, A.i.copy(), A.j.copy(), A.k.copy(), v)


# ----------------------------------------------------------------------------
# Small dense helpers
# ----------------------------------------------------------------------------
def top_left_singular(M: np.ndarray, r: int) -> np.ndarray:
    """The r leading left singular vectors of M (descending singular
    values), by the library SVD."""
    u, s, vt = np.linalg.svd(M, full_matrices=False)
    return u[:, :r].copy()


def hosvd_truncated(C: np.ndarray, r1: int, r3: int):
    """Truncated HOSVD of the (1,2)-symmetric core C (k1 x k1 x k3)
    (Section 2.3, multilinear rank via the SVDs of the unfoldings): Uh holds
    the r1 leading left singular vectors of unfold_1(C) (which equal those of
    unfold_2(C) by the symmetry) and Wh the r3 leading left singular vectors
    of unfold_3(C)."""
    k1, _, k3 = C.shape
    return (top_left_singular(C.reshape(k1, -1, order="F"), r1),
            top_left_singular(unfold3(C), r3))


def sin_theta_max(Ua: np.ndarray, Ub: np.ndarray) -> float:
    """sin of the largest principal angle between span(Ua) and span(Ub):
    ||(I - Ua Ua^T) Ub||_2 for orthonormal Ua, Ub."""
    D = Ub - Ua @ (Ua.T @ Ub)
    return float(np.linalg.norm(D, 2)) if D.size else 0.0


# ----------------------------------------------------------------------------
# Inner solve on the dense core (Algorithm 5 step (i); Section 6.2)
# ----------------------------------------------------------------------------
def _c_t1(C, Uh, Wh):
    # unfold_1(C x_2 Uh^T x_3 Wh^T): k1 x (r1 r3), column b + r1 c
    T = np.einsum("abc,bi,cj->aij", C, Uh, Wh, optimize=True)
    return T.reshape(C.shape[0], -1, order="F")


def _c_t3(C, Uh):
    # unfold_3(C x_1 Uh^T x_2 Uh^T): k3 x r1^2, column a + r1 b
    T = np.einsum("abc,ai,bj->ijc", C, Uh, Uh, optimize=True)
    return T.reshape(-1, C.shape[2], order="F").T


def _inner_grad(Uh, Wh, T1, T3):
    F1 = Uh.T @ T1
    F3 = Wh.T @ T3
    G1 = T1 @ F1.T
    G1 -= Uh @ (Uh.T @ G1)
    G3 = T3 @ F3.T
    G3 -= Wh @ (Wh.T @ G3)
    g = math.sqrt(2.0 * np.sum(G1 * G1) + np.sum(G3 * G3))
    return g, float(np.linalg.norm(F1)), F1


def _hooi_sweeps(C, Uh, Wh, sweeps, tol):
    """Symmetric HOOI sweeps on the dense core (Section 6.1 applied to C):
    Uh <- top r1 left singular vectors of unfold_1(C.(Uh,Wh)_{2,3}) (old Uh),
    then Wh <- top r3 of unfold_3(C.(Uh,Uh)_{1,2}) (new Uh).  The G-gradient
    is checked before each sweep; stops at ||grad|| <= tol ||F|| or after
    ``sweeps`` sweeps.  Returns (Uh, Wh, grad, normF, sweeps_done)."""
    r1, r3 = Uh.shape[1], Wh.shape[1]
    T3 = _c_t3(C, Uh)
    done = 0
    while True:
        T1 = _c_t1(C, Uh, Wh)
        g, nf, _ = _inner_grad(Uh, Wh, T1, T3)
        if done >= sweeps or g <= tol * nf:
            return Uh, Wh, g, nf, done
        Uh = top_left_singular(T1, r1)
        T3 = _c_t3(C, Uh)
        Wh = top_left_singular(T3, r3)
        done += 1


# ----------------------------------------------------------------------------
# Newton-Grassmann on the dense core (Section 6.2 names the method; the
# step below is this library's derivation for the symmetric problem)
# ----------------------------------------------------------------------------
def _complement(Q: np.ndarray) -> np.ndarray:
    """An orthonormal basis of the orthogonal complement of span(Q)."""
    k, r = Q.shape
    full = np.linalg.qr(np.concatenate([Q, np.eye(k)], axis=1))[0]
    # Householder QR of [Q I]: the first r columns span Q; the next k - r
    # complete the orthogonal basis
    return full[:, r:k].copy()


def ng_model(C: np.ndarray, Uh: np.ndarray, Wh: np.ndarray):
    """Gradient and Hessian of g(X, Y) = 1/2 ||C.(U(X), U(X), W(Y))||^2 at
    X = 0, Y = 0, where U(X) = (Uh + Up X)(I + X^T X)^{-1/2} and W(Y) =
    (Wh + Wp Y)(I + Y^T Y)^{-1/2} with [Uh Up], [Wh Wp] orthogonal: local
    coordinates of the product of Grassmann manifolds around (Uh, Wh), U
    used in modes 1 and 2 (the (1,2)-symmetric problem).  With B1 =
    C.(Up,Uh,Wh), B11 = C.(Up,Up,Wh), B3 = C.(Uh,Uh,Wp), B13 = C.(Up,Uh,Wp)
    and F0 = C.(Uh,Uh,Wh), the second-order expansion of the core gives
      grad_X = 2 unfold_1(B1) unfold_1(F0)^T,  grad_Y = unfold_3(B3) unfold_3(F0)^T,
      H = J^T J + [[2K - 2 (M1 (x) I), 2L], [2L^T, -(M3 (x) I)]],
    J the Jacobian of the first-order core term, K[(s,a),(p,b)] =
    sum_c F0[a,b,c] B11[s,p,c], L[(s,a),(t,c)] = sum_b F0[a,b,c] B13[s,b,t],
    M1 = unfold_1(F0) unfold_1(F0)^T, M3 = unfold_3(F0) unfold_3(F0)^T.
    Coordinates are ordered x = vec(X) (column-major), then y = vec(Y).
    Returns (grad, H, Up, Wp)."""
    r1, r3 = Uh.shape[1], Wh.shape[1]
    Up, Wp = _complement(Uh), _complement(Wh)
    d1, d3 = Up.shape[1], Wp.shape[1]
    c3 = lambda A, B, Cm: np.einsum("ijk,ia,jb,kc->abc", C, A, B, Cm, optimize=True)
    F0 = c3(Uh, Uh, Wh)
    B1 = c3(Up, Uh, Wh)
    B11 = c3(Up, Up, Wh)
    B3 = c3(Uh, Uh, Wp)
    B13 = c3(Up, Uh, Wp)
    gX = 2.0 * np.einsum("abc,sbc->sa", F0, B1)
    gY = np.einsum("abc,abt->tc", F0, B3)
    I1, I3 = np.eye(r1), np.eye(r3)
    Jx = (np.einsum("aA,sbc->abcsA", I1, B1) + np.einsum("bA,sac->abcsA", I1, B1))
    Jx = Jx.reshape(r1 * r1 * r3, d1 * r1, order="F")
    Jy = np.einsum("cC,abt->abctC", I3, B3).reshape(r1 * r1 * r3, d3 * r3, order="F")
    J = np.concatenate([Jx, Jy], axis=1)
    K = np.einsum("abc,spc->sapb", F0, B11).reshape(d1 * r1, d1 * r1, order="F")
    L = np.einsum("abc,sbt->satc", F0, B13).reshape(d1 * r1, d3 * r3, order="F")
    M1 = unfold1(F0) @ unfold1(F0).T
    M3 = unfold3(F0) @ unfold3(F0).T
    H = J.T @ J
    H[: d1 * r1, : d1 * r1] += 2.0 * K - 2.0 * np.kron(M1, np.eye(d1))
    H[: d1 * r1, d1 * r1:] += 2.0 * L
    H[d1 * r1:, : d1 * r1] += 2.0 * L.T
    H[d1 * r1:, d1 * r1:] -= np.kron(M3, np.eye(d3))
    grad = np.concatenate([gX.ravel(order="F"), gY.ravel(order="F")])
    return grad, H, Up, Wp


def ng_step(C: np.ndarray, Uh: np.ndarray, Wh: np.ndarray):
    """One Newton step for max ||C.(U,U,W)|| on the Grassmann product:
    solve H z = -grad in the local coordinates of ``ng_model`` and move to
    the orthonormalised (Uh + Up X, Wh + Wp Y).  Returns (Uh, Wh, ok) with
    ok False, and the point unchanged, when -H is not positive definite
    (the point is not near a nondegenerate maximum)."""
    r1, r3 = Uh.shape[1], Wh.shape[1]
    grad, H, Up, Wp = ng_model(C, Uh, Wh)
    try:
        Lc = np.linalg.cholesky(-H)
    except np.linalg.LinAlgError:
        return Uh, Wh, False
    z = np.linalg.solve(Lc.T, np.linalg.solve(Lc, grad))    # z = (-H)^{-1} grad
    d1 = Up.shape[1]
    X = z[: d1 * r1].reshape(d1, r1, order="F")
    Y = z[d1 * r1:].reshape(-1, r3, order="F")
    Un = np.linalg.qr(Uh + Up @ X)[0]
    Wn = np.linalg.qr(Wh + Wp @ Y)[0]
    return Un, Wn, True


# Section 6.2: the inner problem starts from the truncated HOSVD of C
# followed by 5 HOOI iterations
INNER_INIT_SWEEPS = 5


def _ng_try(C: np.ndarray, Uh: np.ndarray, Wh: np.ndarray, nf: float):
    """One Newton-Grassmann step from (Uh, Wh), kept only when ``ng_step``
    takes it (-H positive definite) and ||F|| does not drop below ``nf``
    (relative 1e-14): this library's safeguard away from a maximum.
    Returns (Uh', Wh', grad', normF', taken); a refused step returns the
    old point."""
    Un, Wn, ok = ng_step(C, Uh, Wh)
    if not ok:
        return Uh, Wh, None, nf, False
    T1, T3 = _c_t1(C, Un, Wn), _c_t3(C, Un)
    gn, nfn, _ = _inner_grad(Un, Wn, T1, T3)
    if nfn < nf * (1.0 - 1e-14):
        return Uh, Wh, None, nf, False
    return Un, Wn, gn, nfn, True


def inner_solve(C: np.ndarray, r1: int, r3: int, tol: float, max_inner: int = 1000,
                init_sweeps: int = INNER_INIT_SWEEPS, method: str = "ng"):
    """Best rank-(r1,r1,r3) approximation of the dense (1,2)-symmetric core
    C (k1 x k1 x k3), Algorithm 5 step (i).

    Section 6.2: start from the truncated HOSVD of C followed by 5 HOOI
    iterations, then Newton-Grassmann with the outer stopping criterion.
    Here: after the HOSVD start and its ``init_sweeps`` HOOI sweeps,
    ``method`` "ng" takes Newton steps (``ng_step``) until the G-gradient
    is below ``tol`` relative to ||F|| or ``max_inner`` steps are done; a
    step is refused where -H is not positive definite or ||F|| would drop,
    and a HOOI sweep is taken instead (this library's safeguard away from a
    maximum).  ``method`` "hooi" continues with HOOI sweeps alone.
    Safeguard (this library's reading): the current point (Uh = [I;0],
    Wh = [I;0], which is (U0, W0) in the bases) is kept as a second
    candidate, and the continuation starts from whichever of the two has
    the larger ||F||, so the start never lies below the current point
    (eq. (Fnon-decr)).  A symmetric HOOI sweep (U in modes 1 and 2 at once)
    is not an ascent step, so a solve stopped by ``max_inner`` before
    converging can end below its start.  Returns (Uh, Wh, info)."""
    k1, _, k3 = C.shape
    Uh_a, Wh_a = hosvd_truncated(C, r1, r3)
    Uh_b = np.eye(k1, r1)
    Wh_b = np.eye(k3, r3)
    A_ = _hooi_sweeps(C, Uh_a, Wh_a, init_sweeps, 0.0)
    B_ = _hooi_sweeps(C, Uh_b, Wh_b, 0, 0.0)
    start = A_ if A_[3] >= B_[3] else B_
    pre = A_[4] if start is A_ else 0
    if method == "hooi":
        Uh, Wh, g, nf, done = _hooi_sweeps(C, start[0], start[1], max_inner, tol)
        return Uh, Wh, {"grad": g, "normF": nf, "sweeps": done + pre, "ng_steps": 0,
                        "hosvd_won": start is A_}
    Uh, Wh = start[0], start[1]
    g, nf = start[2], start[3]
    sweeps, steps = pre, 0
    while g > tol * nf and steps + sweeps - pre < max_inner:
        Un, Wn, gn, nfn, ok = _ng_try(C, Uh, Wh, nf)
        if ok:
            Uh, Wh, g, nf = Un, Wn, gn, nfn
            steps += 1
        else:
            Uh, Wh, g, nf, _ = _hooi_sweeps(C, Uh, Wh, 1, 0.0)
            sweeps += 1
    return Uh, Wh, {"grad": g, "normF": nf, "sweeps": sweeps, "ng_steps": steps,
                    "hosvd_won": start is A_}


# ----------------------------------------------------------------------------
# Tensor Krylov-Schur (Algorithm 5) and HOOI (Section 6.1)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class BKSResult:
    U: np.ndarray
    W: np.ndarray
    F: np.ndarray
    converged: bool
    iters: int
    grad_rel: float
    normF: float
    history: list


def bks(A: SymTensor, U0: np.ndarray, W0: np.ndarray, s: int = 2, p: int = 4,
        tol: float = 1e-10, max_outer: int = 500, variant: str = "bk",
        drop_tol: float = 1e-14, inner_tol: float | None = None,
        max_inner: int = 1000, scale_free: bool = False,
        inner_method: str = "ng") -> BKSResult:
    """Tensor Krylov-Schur for a (1,2)-symmetric tensor (Algorithm 5 with
    U = V, X = Y, Section 5).  Each outer iteration: one BK stage from
    (U0, W0) gives the G-gradient by Proposition 2 (steps (iii)-(iv)); stop
    if ||grad||/||F|| <= tol (Section 6.2); else finish the s-stage
    expansion (step (v)), form C = A.(X,X,Z) (eq. (tkd)), solve the inner
    problem (step (i)) to the same criterion, ||grad_C||/||F_C|| <= tol
    (Section 6.2) by Newton-Grassmann (``inner_method`` "hooi": HOOI
    sweeps), and restart from U0 = X Uh, W0 = Z Wh (eq. (tks1), step (ii)).
    ``inner_tol`` replaces the inner tolerance when given.
    ``scale_free`` (this library's option) stops on ||grad||/||F||^2 <= tol
    instead, a test that does not change when A is scaled; the inner
    tolerance is then carried over through ||F|| (tol * ||F||)."""
    r1, r3 = U0.shape[1], W0.shape[1]
    U, W = U0.copy(), W0.copy()
    hist = []
    F = None
    for it in range(max_outer + 1):
        X, Z, info = expand(A, U, W, 1, p, variant, drop_tol)
        g, nf, F = gradient_prop2(info["H1"], info["P1"], info["P3"], r1, r3)
        rel = (g / (nf * nf) if scale_free else g / nf) if nf > 0 else math.inf
        hist.append({"grad_rel": rel, "normF": nf})
        if nf > 0 and rel <= tol:
            return BKSResult(U, W, F, True, it, rel, nf, hist)
        if it == max_outer:
            break
        X, Z, _ = expand(A, U, W, s, p, variant, drop_tol)
        hist[-1]["k1"], hist[-1]["k3"] = X.shape[1], Z.shape[1]
        Cc = core(A, X, Z)
        itol = inner_tol if inner_tol is not None else (tol * nf if scale_free else tol)
        Uh, Wh, iinfo = inner_solve(Cc, r1, r3, itol, max_inner, method=inner_method)
        hist[-1]["inner_sweeps"] = iinfo["sweeps"]
        hist[-1]["ng_steps"] = iinfo["ng_steps"]
        U = X @ Uh
        W = Z @ Wh
    return BKSResult(U, W, F, False, max_outer, hist[-1]["grad_rel"], hist[-1]["normF"], hist)


def hooi(A: SymTensor, U0: np.ndarray, W0: np.ndarray, tol: float = 1e-10,
         max_iter: int = 5000, grad_every: int = 10) -> BKSResult:
    """HOOI for a (1,2)-symmetric tensor (Section 6.1): U <- the r1 leading
    left singular vectors of unfold_1(A.(U,W)_{2,3}) with the previous U,
    then W <- the r3 leading left singular vectors of unfold_3(A.(U,U)_{1,2})
    with the new U.  The G-gradient (global coordinates, Section 2.5) is
    evaluated every ``grad_every`` iterations, at the start of the
    iteration, from the contractions that iteration needs anyway."""
    r1, r3 = U0.shape[1], W0.shape[1]
    U, W = U0.copy(), W0.copy()
    T3 = mode3(A, U, U)
    hist = []
    F1 = None
    for it in range(max_iter + 1):
        T1 = mode1(A, U, W)
        if it % grad_every == 0 or it == max_iter:
            F1 = U.T @ T1
            F3 = W.T @ T3
            G1 = T1 @ F1.T
            G1 -= U @ (U.T @ G1)
            G3 = T3 @ F3.T
            G3 -= W @ (W.T @ G3)
            g = math.sqrt(2.0 * np.linalg.norm(G1) ** 2 + np.linalg.norm(G3) ** 2)
            nf = float(np.linalg.norm(F1))
            hist.append({"iter": it, "grad_rel": g / nf if nf > 0 else math.inf,
                         "normF": nf})
            if (nf > 0 and g <= tol * nf) or it == max_iter:
                F = F1.reshape(r1, r1, r3, order="F")
                return BKSResult(U, W, F, nf > 0 and g <= tol * nf, it, g / nf, nf, hist)
        U = top_left_singular(T1, r1)
        T3 = mode3(A, U, U)
        W = top_left_singular(T3, r3)
    raise AssertionError("unreachable")
