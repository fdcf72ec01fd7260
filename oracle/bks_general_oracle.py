"""Plain FP64 numpy oracle of the tensor Krylov-Schur method for a general
(nonsymmetric) l x m x n tensor: separate bases X, Y, Z for the three modes
(Section 5, Algorithm 5 as stated there; Section 4.3, Algorithm 3 in each
mode; Proposition 2 with three terms) and HOOI (Section 6.1).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline legs use this module; the CUDA library never
calls it.

Readings of this library (the paper tabulates block schedules only for the
(1,2)-symmetric case):

* BK schedule, general form: stage 1 makes U1 from (V0, W0), V1 from
  (U0, W0) and W1 from (U0, V0) (Section 4.3: the blocks with subscript 1
  come from U0, V0, W0).  Stage t >= 2, q = t - 1: each mode takes the pairs
  (0, q), (q, 0), (1, q), (q, 1), ..., (q-1, q), (q, q-1) of the other two
  modes' blocks (the diagonal (q, q) left out, as in Table 3); without the
  (1,2)-symmetry no pair is a transpose of another, so mode 3 takes both
  orders too.  min-BK: stage t uses the blocks t-1 of the other two modes
  in every mode (Algorithm 4 without the symmetry).  max-BK: every pair of
  whole blocks not used before, by shells as in Table 2.  Within a stage
  the mode-1 blocks are made first, then mode 2, then mode 3, each in the
  order above, from the blocks that existed when the stage began.
* The inner problem (Algorithm 5 step (i)) is solved by the truncated
  HOSVD start, 5 HOOI sweeps and then HOOI sweeps to the tolerance
  (Section 6.2 continues with Newton-Grassmann, which this library derives
  for the symmetric problem only); the current point competes with the
  HOSVD start by ||F|| (eq. (Fnon-decr)).  Each general HOOI update
  maximises ||F|| over one factor exactly, so the sweeps never lower it.

Pins (``tests/test_oracle_general.py``): the storage rule by a dict model;
contractions and core by dense einsum; the matrix case n = 1 (Eckart-Young,
best rank-(r, r, 1) from the SVD); exact recovery of a planted
multilinear-rank (r1, r2, r3) tensor with l, m, n all different; on a
(1,2)-symmetric tensor with V = U the gradient equals the symmetric
oracle's and the solve reaches the symmetric optimum; Lemma 1 on the
expansion; Proposition 2 against the global gradient; monotone inner
sweeps; BKS and HOOI agreement; the core over several entry blocks; basis
sizes from the pair and bar rule; modes 1 and 2 in the symmetric
schedule's order; the inner gradient equal to the global gradient of the
core; the five start sweeps counted; the HOSVD of a core with equal
dimensions; HOOI's gradient every 10 iterations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "GenTensor", "gen_tensor", "gmode1", "gmode2", "gmode3", "gcore", "gen_stage_pairs",
    "gen_schedule_counts", "gen_expand", "gen_gradient_prop2", "gen_gradient_global",
    "gen_hosvd", "gen_inner_solve", "gen_bks", "gen_hooi", "GenBKSResult", "gunfold",
    "GEN_INNER_INIT_SWEEPS",
]

GEN_INNER_INIT_SWEEPS = 5  # Section 6.2: HOOI iterations after the HOSVD start


# ----------------------------------------------------------------------------
# Storage: a general sparse tensor, entries sorted by (i, j, k), duplicates
# summed left to right in input order
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class GenTensor:
    l: int
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
        T = np.zeros((self.l, self.m, self.n))
        np.add.at(T, (self.i, self.j, self.k), self.vf())
        return T


def gen_tensor(l, m, n, i, j, k, v) -> GenTensor:
    """The stored form of a general sparse tensor: the input list stably
    sorted by (i, j, k), entries with equal keys summed left to right in the
    value dtype (exact zeros kept).  No mirroring."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    v = np.asarray(v)
    if l <= 0 or m <= 0 or n <= 0:
        raise ValueError("l, m and n must be positive")
    if i.size and (min(i.min(), j.min(), k.min()) < 0 or i.max() >= l or j.max() >= m
                   or k.max() >= n):
        raise ValueError("index out of range")
    order = np.lexsort((k, j, i))
    ii, jj, kk, vv = i[order], j[order], k[order], v[order]
    if ii.size == 0:
        return GenTensor(l, m, n, ii.astype(np.int32), jj.astype(np.int32),
                         kk.astype(np.int32), vv.copy())
    new = np.ones(ii.size, dtype=bool)
    new[1:] = (ii[1:] != ii[:-1]) | (jj[1:] != jj[:-1]) | (kk[1:] != kk[:-1])
    starts = np.nonzero(new)[0]
    lengths = np.diff(np.append(starts, ii.size))
    acc = vv[starts].copy()
    for d in range(1, int(lengths.max())):
        sel = lengths > d
        acc[sel] = acc[sel] + vv[starts[sel] + d]
    return GenTensor(l, m, n, ii[starts].astype(np.int32), jj[starts].astype(np.int32),
                     kk[starts].astype(np.int32), acc)


# ----------------------------------------------------------------------------
# Contractions (Section 2.2; Algorithm 3 step (i) in each mode)
# ----------------------------------------------------------------------------
def gmode1(A: GenTensor, V: np.ndarray, W: np.ndarray) -> np.ndarray:
    """unfold_1(A.(V,W)_{2,3}): l x (p q), column a + p b,
    Out[i, a + p b] = sum v V[j, a] W[k, b]."""
    p, q = V.shape[1], W.shape[1]
    out = np.zeros((A.l, p * q))
    v = A.vf()
    for b in range(q):
        wb = W[A.k, b] * v
        for a in range(p):
            np.add.at(out[:, a + p * b], A.i, wb * V[A.j, a])
    return out


def gmode2(A: GenTensor, U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """unfold_2(A.(U,W)_{1,3}): m x (p q), column a + p b,
    Out[j, a + p b] = sum v U[i, a] W[k, b]."""
    p, q = U.shape[1], W.shape[1]
    out = np.zeros((A.m, p * q))
    v = A.vf()
    for b in range(q):
        wb = W[A.k, b] * v
        for a in range(p):
            np.add.at(out[:, a + p * b], A.j, wb * U[A.i, a])
    return out


def gmode3(A: GenTensor, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """unfold_3(A.(U,V)_{1,2}): n x (p q), column a + p b,
    Out[k, a + p b] = sum v U[i, a] V[j, b]."""
    p, q = U.shape[1], V.shape[1]
    out = np.zeros((A.n, p * q))
    v = A.vf()
    for b in range(q):
        vb = V[A.j, b] * v
        for a in range(p):
            np.add.at(out[:, a + p * b], A.k, vb * U[A.i, a])
    return out


def gcore(A: GenTensor, X: np.ndarray, Y: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """C = A.(X,Y,Z) (eq. (tkd)): C[a,b,c] = sum v X[i,a] Y[j,b] Z[k,c]."""
    v = A.vf()
    # per entry the outer product v X[i,:] x Y[j,:] x Z[k,:], summed; in
    # slices of entries to bound memory
    C = np.zeros((X.shape[1], Y.shape[1], Z.shape[1]))
    step = 2048
    for s in range(0, A.nnz, step):
        e = slice(s, s + step)
        C += np.einsum("e,ea,eb,ec->abc", v[e], X[A.i[e]], Y[A.j[e]], Z[A.k[e]], optimize=True)
    return C


def gunfold(F: np.ndarray, mode: int) -> np.ndarray:
    """Mode-k unfolding, the other two indices in their natural order with
    the first fastest (column a + r b)."""
    return np.moveaxis(F, mode, 0).reshape(F.shape[mode], -1, order="F")


# ----------------------------------------------------------------------------
# Block orthogonalisation (Algorithm 3 steps (ii)-(iv), Appendix B) is the
# symmetric oracle's: the step does not depend on the tensor.
# ----------------------------------------------------------------------------
from .bks_oracle import orth_block, top_left_singular  # noqa: E402


# ----------------------------------------------------------------------------
# Block schedules, general form (see the module docstring)
# ----------------------------------------------------------------------------
def gen_stage_pairs(variant: str, stage: int, counts, done):
    """Pairs of one stage for the three modes: a list per mode of
    (left block, right block), where mode 1 pairs (V, W) blocks, mode 2
    (U, W) and mode 3 (U, V).  ``counts`` = (nU, nV, nW) blocks existing
    at the start of the stage; ``done`` = three sets of used pairs."""
    nU, nV, nW = counts
    sides = ((nV, nW), (nU, nW), (nU, nV))
    if stage == 1:
        return [[(0, 0)], [(0, 0)], [(0, 0)]]
    out = [[], [], []]
    q = stage - 1
    if variant == "bk":
        for md in range(3):
            na, nb = sides[md]
            if q >= na or q >= nb:
                continue
            for t in range(q):
                out[md].append((t, q))
                out[md].append((q, t))
        return out
    if variant == "min":
        for md in range(3):
            na, nb = sides[md]
            if q < na and q < nb:
                out[md].append((q, q))
        return out
    if variant == "max":
        for md in range(3):
            na, nb = sides[md]
            for s in range(max(na, nb)):
                for t in range(s):
                    for (a, b) in ((t, s), (s, t)):
                        if a < na and b < nb and (a, b) not in done[md]:
                            out[md].append((a, b))
                if s < na and s < nb and (s, s) not in done[md]:
                    out[md].append((s, s))
        return out
    raise ValueError(variant)


def _gbar(variant, idx, width, p):
    if variant == "max" or idx == 0:
        return width
    return min(p, width)


def gen_schedule_counts(r, s: int, p: int, variant: str = "bk", dims=None):
    """(k1, k2, k3) after each stage when no column is dropped, with the
    caps k_i <= dim_i."""
    widths = [[r[0]], [r[1]], [r[2]]]
    done = [set(), set(), set()]
    k = list(r)
    out = []
    others = ((1, 2), (0, 2), (0, 1))
    for st in range(1, s + 1):
        pairs = gen_stage_pairs(variant, st, tuple(len(w) for w in widths), done)
        new = [list(w) for w in widths]
        for md in range(3):
            ma, mb = others[md]
            for (a, b) in pairs[md]:
                cols = _gbar(variant, a, widths[ma][a], p) * _gbar(variant, b, widths[mb][b], p)
                if dims is not None:
                    cols = max(0, min(cols, dims[md] - k[md]))
                new[md].append(cols)
                k[md] += cols
                done[md].add((a, b))
        widths = new
        out.append(tuple(k))
    return out


def _contract(A: GenTensor, md: int, L: np.ndarray, R: np.ndarray) -> np.ndarray:
    if md == 0:
        return gmode1(A, L, R)
    if md == 1:
        return gmode2(A, L, R)
    return gmode3(A, L, R)


def gen_expand(A: GenTensor, U0, V0, W0, s: int, p: int, variant: str = "bk",
               drop_tol: float = 1e-14):
    """Expand (U0, V0, W0) to X (l x k1), Y (m x k2), Z (n x k3) with s
    stages (Algorithm 5 steps (iii), (v)).  Returns (X, Y, Z, info, blocks):
    info[md] = (H, P) of the stage-1 block of mode md (H = Q^T B = the
    mode's unfolding of F, P = B - Q H), blocks = the ON-blocks per mode."""
    dims = (A.l, A.m, A.n)
    blocks = [[U0.copy()], [V0.copy()], [W0.copy()]]
    bases = [U0.copy(), V0.copy(), W0.copy()]
    done = [set(), set(), set()]
    others = ((1, 2), (0, 2), (0, 1))
    info = {}
    for st in range(1, s + 1):
        pairs = gen_stage_pairs(variant, st, tuple(len(b) for b in blocks), done)
        new = [[], [], []]
        for md in range(3):
            ma, mb = others[md]
            for (a, b) in pairs[md]:
                L = blocks[ma][a] if (variant == "max" or a == 0) else blocks[ma][a][:, :p]
                R = blocks[mb][b] if (variant == "max" or b == 0) else blocks[mb][b][:, :p]
                done[md].add((a, b))
                if L.shape[1] == 0 or R.shape[1] == 0:
                    new[md].append(np.zeros((dims[md], 0)))
                    continue
                B = _contract(A, md, L, R)
                Qn, H, Rf, kept, P = orth_block(bases[md], B, drop_tol, max_total=dims[md])
                if st == 1:
                    info[md] = (H, P)
                bases[md] = np.concatenate([bases[md], Qn], axis=1)
                new[md].append(Qn)
        for md in range(3):
            blocks[md].extend(new[md])
    return bases[0], bases[1], bases[2], info, blocks


# ----------------------------------------------------------------------------
# Gradient (Section 2.5; Proposition 2 with three terms)
# ----------------------------------------------------------------------------
def gen_gradient_prop2(info, r):
    """||grad|| and ||F|| at (U0, V0, W0) from the first block-Krylov step
    in each mode (Proposition 2): mode term ||<H0, H1^k>_{-k}|| =
    ||P_k H_k^T||, with H_k = unfold_k(F) the projection of the stage-1
    block on the current factor and P_k the projected block."""
    r1, r2, r3 = r
    H1, P1 = info[0]
    F = H1.reshape(r1, r2, r3, order="F")
    g2 = 0.0
    for md in range(3):
        H, P = info[md]
        g2 += float(np.linalg.norm(P @ H.T)) ** 2
    return math.sqrt(g2), float(np.linalg.norm(F)), F


def gen_gradient_global(A: GenTensor, U, V, W):
    """||grad||, ||F|| in global coordinates (Section 2.5): mode k term
    (I - Q_k Q_k^T) T_k F_k^T with T_k the mode-k contraction with the
    other two factors and F_k = Q_k^T T_k = unfold_k(F)."""
    r = (U.shape[1], V.shape[1], W.shape[1])
    Ts = (gmode1(A, V, W), gmode2(A, U, W), gmode3(A, U, V))
    Qs = (U, V, W)
    g2 = 0.0
    for Q, T in zip(Qs, Ts):
        Fk = Q.T @ T
        G = T @ Fk.T
        G -= Q @ (Q.T @ G)
        g2 += float(np.sum(G * G))
    F = (U.T @ Ts[0]).reshape(r, order="F")
    return math.sqrt(g2), float(np.linalg.norm(F)), F


# ----------------------------------------------------------------------------
# Inner solve on the dense core (Algorithm 5 step (i); Section 6.2)
# ----------------------------------------------------------------------------
def gen_hosvd(C: np.ndarray, r):
    """Truncated HOSVD (Section 2.3): the r_k leading left singular vectors
    of unfold_k(C), k = 1, 2, 3."""
    return tuple(top_left_singular(gunfold(C, md), r[md]) for md in range(3))


def _gt(C, facs, md):
    """unfold_md of C multiplied in the other two modes by the transposed
    factors: k_md x (r_a r_b), column a + r_a b (a the lower mode)."""
    Uh, Vh, Wh = facs
    if md == 0:
        T = np.einsum("abc,bi,cj->aij", C, Vh, Wh, optimize=True)
    elif md == 1:
        T = np.einsum("abc,ai,cj->bij", C, Uh, Wh, optimize=True)
    else:
        T = np.einsum("abc,ai,bj->cij", C, Uh, Vh, optimize=True)
    return T.reshape(C.shape[md], -1, order="F")


def _ginner_grad(C, facs):
    g2 = 0.0
    nf = 0.0
    for md in range(3):
        T = _gt(C, facs, md)
        Q = facs[md]
        Fk = Q.T @ T
        G = T @ Fk.T
        G -= Q @ (Q.T @ G)
        g2 += float(np.sum(G * G))
        if md == 0:
            nf = float(np.linalg.norm(Fk))
    return math.sqrt(g2), nf


def _ghooi_sweeps(C, facs, sweeps, tol):
    """General HOOI sweeps on the dense core (Section 6.1 applied to C):
    Uh from (Vh, Wh), then Vh from (new Uh, Wh), then Wh from (new Uh, new
    Vh), each the leading left singular vectors of the mode's contraction.
    The gradient is checked before each sweep.  Returns (facs, grad, normF,
    sweeps_done, history of ||F|| before each sweep)."""
    facs = list(facs)
    r = [f.shape[1] for f in facs]
    done = 0
    hist = []
    while True:
        g, nf = _ginner_grad(C, facs)
        hist.append(nf)
        if done >= sweeps or g <= tol * nf:
            return tuple(facs), g, nf, done, hist
        for md in range(3):
            facs[md] = top_left_singular(_gt(C, facs, md), r[md])
        done += 1


def gen_inner_solve(C: np.ndarray, r, tol: float, max_inner: int = 1000,
                    init_sweeps: int = GEN_INNER_INIT_SWEEPS):
    """Best rank-(r1,r2,r3) approximation of the dense core C (k1 x k2 x
    k3).  Candidates: the truncated HOSVD after ``init_sweeps`` HOOI sweeps,
    and the current point ([I;0] in each mode) unswept; the one with the
    larger ||F|| continues with HOOI sweeps until ||grad|| <= tol ||F|| or
    ``max_inner`` sweeps.  Returns (Uh, Vh, Wh, info)."""
    k = C.shape
    A_ = _ghooi_sweeps(C, gen_hosvd(C, r), init_sweeps, 0.0)
    B_ = _ghooi_sweeps(C, tuple(np.eye(k[md], r[md]) for md in range(3)), 0, 0.0)
    start = A_ if A_[2] >= B_[2] else B_
    pre = A_[3] if start is A_ else 0
    facs, g, nf, done, hist = _ghooi_sweeps(C, start[0], max_inner, tol)
    return facs[0], facs[1], facs[2], {"grad": g, "normF": nf, "sweeps": done + pre,
                                       "hosvd_won": start is A_, "normF_history": hist}


# ----------------------------------------------------------------------------
# Tensor Krylov-Schur (Algorithm 5) and HOOI (Section 6.1), general form
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class GenBKSResult:
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    F: np.ndarray
    converged: bool
    iters: int
    grad_rel: float
    normF: float
    history: list


def gen_bks(A: GenTensor, U0, V0, W0, s: int = 2, p: int = 4, tol: float = 1e-10,
            max_outer: int = 500, variant: str = "bk", drop_tol: float = 1e-14,
            inner_tol: float | None = None, max_inner: int = 1000,
            scale_free: bool = False) -> GenBKSResult:
    """Algorithm 5 for a general tensor: one BK stage from (U0, V0, W0)
    gives the gradient by Proposition 2; stop when ||grad||/||F|| <= tol
    (``scale_free``: ||grad||/||F||^2); else expand with s stages, form
    C = A.(X,Y,Z), solve the inner problem to the same criterion and restart
    from U0 = X Uh, V0 = Y Vh, W0 = Z Wh (eq. (tks1))."""
    r = (U0.shape[1], V0.shape[1], W0.shape[1])
    U, V, W = U0.copy(), V0.copy(), W0.copy()
    hist = []
    F = None
    for it in range(max_outer + 1):
        _, _, _, info, _ = gen_expand(A, U, V, W, 1, p, variant, drop_tol)
        g, nf, F = gen_gradient_prop2(info, r)
        rel = (g / (nf * nf) if scale_free else g / nf) if nf > 0 else math.inf
        hist.append({"grad_rel": rel, "normF": nf})
        if nf > 0 and rel <= tol:
            return GenBKSResult(U, V, W, F, True, it, rel, nf, hist)
        if it == max_outer:
            break
        X, Y, Z, _, _ = gen_expand(A, U, V, W, s, p, variant, drop_tol)
        hist[-1]["k"] = (X.shape[1], Y.shape[1], Z.shape[1])
        Cc = gcore(A, X, Y, Z)
        itol = inner_tol if inner_tol is not None else (tol * nf if scale_free else tol)
        Uh, Vh, Wh, iinfo = gen_inner_solve(Cc, r, itol, max_inner)
        hist[-1]["inner_sweeps"] = iinfo["sweeps"]
        U, V, W = X @ Uh, Y @ Vh, Z @ Wh
    return GenBKSResult(U, V, W, F, False, max_outer, hist[-1]["grad_rel"],
                        hist[-1]["normF"], hist)


def gen_hooi(A: GenTensor, U0, V0, W0, tol: float = 1e-10, max_iter: int = 5000,
             grad_every: int = 10) -> GenBKSResult:
    """HOOI for a general tensor (Section 6.1): U <- leading left singular
    vectors of unfold_1(A.(V,W)_{2,3}), then V from A.(U,W)_{1,3} with the
    new U, then W from A.(U,V)_{1,2} with the new U and V; the global
    gradient every ``grad_every`` iterations at the start of the
    iteration."""
    r = (U0.shape[1], V0.shape[1], W0.shape[1])
    U, V, W = U0.copy(), V0.copy(), W0.copy()
    hist = []
    for it in range(max_iter + 1):
        if it % grad_every == 0 or it == max_iter:
            g, nf, F = gen_gradient_global(A, U, V, W)
            hist.append({"iter": it, "grad_rel": g / nf if nf > 0 else math.inf, "normF": nf})
            if (nf > 0 and g <= tol * nf) or it == max_iter:
                return GenBKSResult(U, V, W, F, nf > 0 and g <= tol * nf, it,
                                    g / nf if nf > 0 else math.inf, nf, hist)
        U = top_left_singular(gmode1(A, V, W), r[0])
        V = top_left_singular(gmode2(A, U, W), r[1])
        W = top_left_singular(gmode3(A, U, V), r[2])
    raise AssertionError("unreachable")
