"""Seeded synthetic inputs for the (1,2)-symmetric sparse tensor workloads.

This module is shared by the CPU oracle, the CUDA path's tests and the
benchmark.  It only *draws* inputs: COO index/value lists, random starting
matrices with orthonormal columns, and the planted signal tensors used by the
pins.  It holds none of the method's arithmetic (no symmetrisation, no
contraction, no orthogonalisation, no solver step).

Every generator uses ``numpy.random.Generator(PCG64(seed))`` so the same seed
gives the same bytes on x86-64 and aarch64.

Workload shapes follow the paper's experiments on (1,2)-symmetric tensors
(adjacency-like slices, Section 6.2) at the sizes of the five benchmark
configurations:

* ``small_planted``    300x300x100, 10,000 uniform draws + planted (2,2,2) term
* ``zipf_tensor``      power-law rows (finite Zipf), uniform mode-3 index
* ``batch_jobs``       256 heterogeneous jobs (lognormal sizes)
* ``serving_stream``   Poisson arrivals of batch-like jobs
* ``dense_planted``    exact multilinear rank (U0,U0,W0).F0 on a dense support
* ``example1``         signal + rho * noise, Example 1 of Section 6.2.1
* ``general_*``        general (nonsymmetric) l x m x n tensors for the
                       three-basis form of the method (Section 5)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "COO", "rng", "orthonormal", "small_planted", "zipf_tensor", "zipf_table",
    "dense_planted", "example1", "batch_jobs", "serving_stream", "dense_to_coo",
    "random_coo", "CONFIG_SEEDS", "GenCOO", "general_random_coo", "general_zipf_tensor",
    "general_dense_planted", "general_dense_to_coo", "general_sampled_planted",
    "general_noisy_planted",
]

CONFIG_SEEDS = {"small": 1, "medium": 2, "large": 3, "batch": 4, "serve": 5}


@dataclasses.dataclass
class COO:
    """A sparse 3-tensor of shape m x m x n as a list of (i, j, k, v) entries.

    ``mirror`` tells the consumer how the list is meant: ``True`` means every
    off-diagonal entry (i != j) stands for itself and its mirror (j, i, k),
    which the ingest step adds; ``False`` means the list already holds both
    halves.  Indices are 0-based int32.
    """
    m: int
    n: int
    i: np.ndarray
    j: np.ndarray
    k: np.ndarray
    v: np.ndarray
    mirror: bool = True

    @property
    def nnz(self) -> int:
        return int(self.i.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def orthonormal(g: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """A random rows x cols matrix with orthonormal columns (column-major
    float64), the Q factor of a Gaussian matrix.  This is the random starting
    point that both the oracle and the CUDA path receive as an input."""
    a = g.standard_normal((rows, cols))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    return np.asfortranarray(q)


def _draw_uniform_offdiag(g, m, count):
    i = g.integers(0, m, size=count)
    j = g.integers(0, m, size=count)
    bad = i == j
    while bad.any():
        j[bad] = g.integers(0, m, size=int(bad.sum()))
        bad = i == j
    return i, j


def random_coo(seed: int, m: int, n: int, draws: int, vdtype=np.float64,
               allow_diag: bool = True) -> COO:
    """Uniform random (i, j, k) draws with N(0,1) values (duplicates and
    diagonal entries allowed unless ``allow_diag`` is False).  Used by the
    ingest and contraction tests."""
    g = rng(seed)
    if allow_diag:
        i = g.integers(0, m, size=draws)
        j = g.integers(0, m, size=draws)
    else:
        i, j = _draw_uniform_offdiag(g, m, draws)
    k = g.integers(0, n, size=draws)
    v = g.standard_normal(draws).astype(vdtype)
    return COO(m, n, i.astype(np.int32), j.astype(np.int32),
               k.astype(np.int32), v, mirror=True)


def _planted_values(i, j, k, U0, W0, F0):
    # value of the tensor (U0, U0, W0).F0 at the listed positions
    ui = U0[i]          # nnz x r1
    uj = U0[j]
    wk = W0[k]          # nnz x r3
    return np.einsum("za,zb,zc,abc->z", ui, uj, wk, F0, optimize=True)


def small_planted(seed: int = 1, m: int = 300, n: int = 100, draws: int = 10_000,
                  r: int = 2, snr: float = 10.0) -> tuple[COO, dict]:
    """The 300x300x100 workload: ``draws`` entries with i, j uniform on
    [0, m), i != j, k uniform on [0, n), noise values |N(0,1)|, plus a
    planted rank-(r,r,r) term alpha * ((U0,U0,W0).F0)(i,j,k) evaluated at the
    drawn positions.  F0 has N(0,1) entries symmetrised in modes 1 and 2.
    alpha makes the planted part's norm ``snr`` times the noise part's norm
    over the drawn entries.  The list is given one-sided (mirror=True); since
    the planted tensor is (1,2)-symmetric, a mirror carries the same planted
    value."""
    g = rng(seed)
    i, j = _draw_uniform_offdiag(g, m, draws)
    k = g.integers(0, n, size=draws)
    noise = np.abs(g.standard_normal(draws))
    U0 = orthonormal(g, m, r)
    W0 = orthonormal(g, n, r)
    F0 = g.standard_normal((r, r, r))
    F0 = 0.5 * (F0 + F0.transpose(1, 0, 2))
    P = _planted_values(i, j, k, U0, W0, F0)
    alpha = snr * np.linalg.norm(noise) / max(np.linalg.norm(P), 1e-300)
    v = noise + alpha * P
    coo = COO(m, n, i.astype(np.int32), j.astype(np.int32), k.astype(np.int32),
              v.astype(np.float64), mirror=True)
    return coo, {"U0": U0, "W0": W0, "F0": F0, "alpha": alpha}


def zipf_table(m: int, s: float) -> np.ndarray:
    """Inverse-CDF table of the finite Zipf law p(rank) ~ rank^-s on
    ranks 1..m (returned as the cumulative distribution, float64)."""
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _zipf_draw(g, cdf, count):
    u = g.random(count)
    return np.minimum(np.searchsorted(cdf, u, side="right"), cdf.shape[0] - 1)


def zipf_tensor(seed: int, m: int, n: int, draws: int, s: float,
                values: str = "lognormal", vdtype=np.float64) -> COO:
    """Power-law workload: i and j drawn independently from a finite Zipf(s)
    law on m ranks mapped through a seeded permutation of [0, m); a draw with
    i == j redraws j; k uniform on [0, n); values lognormal(0,1) or |N(0,1)|.
    Given one-sided (mirror=True): the stored tensor has about 2*draws
    entries."""
    g = rng(seed)
    cdf = zipf_table(m, s)
    perm = g.permutation(m)
    i = perm[_zipf_draw(g, cdf, draws)]
    j = perm[_zipf_draw(g, cdf, draws)]
    bad = np.nonzero(i == j)[0]
    while bad.size:
        j[bad] = perm[_zipf_draw(g, cdf, bad.size)]
        bad = bad[i[bad] == j[bad]]
    k = g.integers(0, n, size=draws)
    if values == "lognormal":
        v = g.lognormal(0.0, 1.0, size=draws)
    elif values == "absnormal":
        v = np.abs(g.standard_normal(draws))
    else:
        raise ValueError(values)
    return COO(m, n, i.astype(np.int32), j.astype(np.int32), k.astype(np.int32),
               v.astype(vdtype), mirror=True)


def dense_to_coo(T: np.ndarray, mirror_input: bool = False) -> COO:
    """All entries of a dense m x m x n array (zeros included) as a COO list
    holding both halves (mirror=False)."""
    m, m2, n = T.shape
    assert m == m2
    i, j, k = np.meshgrid(np.arange(m), np.arange(m), np.arange(n), indexing="ij")
    return COO(m, n, i.ravel().astype(np.int32), j.ravel().astype(np.int32),
               k.ravel().astype(np.int32), T.ravel().astype(np.float64),
               mirror=mirror_input)


def dense_planted(seed: int, m: int = 40, n: int = 12, r1: int = 2, r3: int = 2):
    """A tensor of exact multilinear rank (r1, r1, r3): (U0,U0,W0).F0 with
    F0 symmetric in modes 1,2, as a dense m x m x n array.  Returns
    (T, U0, W0, F0)."""
    g = rng(seed)
    U0 = orthonormal(g, m, r1)
    W0 = orthonormal(g, n, r3)
    F0 = g.standard_normal((r1, r1, r3))
    F0 = 0.5 * (F0 + F0.transpose(1, 0, 2))
    T = np.einsum("ia,jb,kc,abc->ijk", U0, U0, W0, F0, optimize=True)
    T = 0.5 * (T + T.transpose(1, 0, 2))
    return T, U0, W0, F0


def example1(seed: int, m: int, n: int, r1: int, r3: int, rho: float):
    """Example 1 of Section 6.2.1: an N(0,1) core of size r1 x r1 x r3 placed
    in the top-left corner of an m x m x n zero tensor, plus rho times an
    N(0,1) noise tensor made (1,2)-symmetric, then a random symmetric
    permutation of modes 1,2 (and a random permutation of mode 3).  The core
    is symmetrised in modes 1,2 so that the signal is (1,2)-symmetric too.
    Returns a dense array."""
    g = rng(seed)
    S = g.standard_normal((r1, r1, r3))
    S = 0.5 * (S + S.transpose(1, 0, 2))
    N = g.standard_normal((m, m, n))
    N = 0.5 * (N + N.transpose(1, 0, 2))
    T = rho * N
    T[:r1, :r1, :r3] += S
    p = g.permutation(m)
    q = g.permutation(n)
    return np.ascontiguousarray(T[np.ix_(p, p, q)])


def _lognormal_int(g, lo, hi, count):
    mu = 0.5 * (math.log(lo) + math.log(hi))
    sigma = (math.log(hi) - math.log(lo)) / 4.0
    x = np.exp(g.normal(mu, sigma, size=count))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def batch_jobs(seed: int = 4, count: int = 256, m_range=(1_000, 200_000),
               n_range=(20, 100), nnz_range=(10_000, 5_000_000), ranks=(2, 3, 4),
               scale: float = 1.0):
    """Shapes of the heterogeneous batch: per job m lognormal on m_range,
    n uniform on n_range, stored nnz lognormal on nnz_range (capped at
    0.5*m*m*n), rank r uniform in ``ranks`` (r1 = r3 = r).  ``scale``
    shrinks m and nnz for small test batches.  Returns a list of dicts with
    the per-job seed; ``job_tensor`` draws the tensor itself."""
    g = rng(seed)
    ms = _lognormal_int(g, *m_range, count)
    ns = g.integers(n_range[0], n_range[1] + 1, size=count)
    nz = _lognormal_int(g, *nnz_range, count)
    rs = g.choice(np.asarray(ranks), size=count)
    jobs = []
    for t in range(count):
        m = max(8, int(ms[t] * scale))
        n = int(ns[t])
        stored = int(min(nz[t] * scale, 0.5 * m * m * n))
        jobs.append({"m": m, "n": n, "nnz_stored": max(stored, 16), "r": int(rs[t]),
                     "seed": seed * 100_003 + t})
    return jobs


def job_tensor(job: dict) -> COO:
    """The tensor of one batch job: Zipf(1.1) rows, uniform mode-3 index,
    lognormal(0,1) values, about ``nnz_stored`` stored entries."""
    return zipf_tensor(job["seed"], job["m"], job["n"], max(job["nnz_stored"] // 2, 8),
                       1.1, values="lognormal")


def serving_stream(seed: int = 5, requests: int = 2000, mean_gap_s: float = 0.005,
                   scale: float = 1.0):
    """Poisson arrival stream: exponential inter-arrival gaps of mean
    ``mean_gap_s`` (200 requests/s at the default) over jobs drawn as in
    ``batch_jobs``.  Returns (arrival_times_s, jobs)."""
    g = rng(seed)
    gaps = g.exponential(mean_gap_s, size=requests)
    t = np.cumsum(gaps)
    jobs = batch_jobs(seed=seed, count=requests, scale=scale)
    return t, jobs


# ---- general (nonsymmetric) l x m x n tensors --------------------------------
@dataclasses.dataclass
class GenCOO:
    """A general sparse 3-tensor of shape l x m x n as (i, j, k, v) lists
    (0-based int32 indices; duplicates allowed, summed by the consumer)."""
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


def general_random_coo(seed: int, l: int, m: int, n: int, draws: int,
                       vdtype=np.float64) -> GenCOO:
    """Uniform random (i, j, k) draws with N(0,1) values, duplicates
    allowed."""
    g = rng(seed)
    i = g.integers(0, l, size=draws)
    j = g.integers(0, m, size=draws)
    k = g.integers(0, n, size=draws)
    v = g.standard_normal(draws).astype(vdtype)
    return GenCOO(l, m, n, i.astype(np.int32), j.astype(np.int32), k.astype(np.int32), v)


def general_zipf_tensor(seed: int, l: int, m: int, n: int, draws: int, s: float,
                        values: str = "lognormal", vdtype=np.float64) -> GenCOO:
    """Power-law general workload (a directed, bipartite or rectangular
    relation per slice): i from a finite Zipf(s) law on l ranks and j from
    one on m ranks, each through its own seeded permutation; k uniform on
    [0, n); values lognormal(0,1) or |N(0,1)|.  No mirroring."""
    g = rng(seed)
    pi = g.permutation(l)
    pj = g.permutation(m)
    i = pi[_zipf_draw(g, zipf_table(l, s), draws)]
    j = pj[_zipf_draw(g, zipf_table(m, s), draws)]
    k = g.integers(0, n, size=draws)
    if values == "lognormal":
        v = g.lognormal(0.0, 1.0, size=draws)
    elif values == "absnormal":
        v = np.abs(g.standard_normal(draws))
    else:
        raise ValueError(values)
    return GenCOO(l, m, n, i.astype(np.int32), j.astype(np.int32), k.astype(np.int32),
                  v.astype(vdtype))


def general_dense_to_coo(T: np.ndarray) -> GenCOO:
    """All entries of a dense l x m x n array (zeros included)."""
    l, m, n = T.shape
    i, j, k = np.meshgrid(np.arange(l), np.arange(m), np.arange(n), indexing="ij")
    return GenCOO(l, m, n, i.ravel().astype(np.int32), j.ravel().astype(np.int32),
                  k.ravel().astype(np.int32), T.ravel().astype(np.float64))


def general_dense_planted(seed: int, l: int = 30, m: int = 24, n: int = 10,
                          r=(2, 3, 2)):
    """A dense l x m x n tensor of exact multilinear rank r:
    (U0, V0, W0).F0 with N(0,1) core entries.  Returns (T, U0, V0, W0, F0)."""
    g = rng(seed)
    U0 = orthonormal(g, l, r[0])
    V0 = orthonormal(g, m, r[1])
    W0 = orthonormal(g, n, r[2])
    F0 = g.standard_normal(tuple(r))
    T = np.einsum("ia,jb,kc,abc->ijk", U0, V0, W0, F0, optimize=True)
    return T, U0, V0, W0, F0


def general_sampled_planted(seed: int, l: int, m: int, n: int, draws: int, r=(2, 2, 2),
                            snr: float = 10.0) -> GenCOO:
    """``draws`` uniform (i, j, k) positions with N(0,1) noise plus
    alpha * ((U0,V0,W0).F0)(i,j,k) at the drawn positions, alpha making the
    planted part ``snr`` times the noise part in norm (a sparse general
    analogue of ``small_planted``; zero-mean noise, so that the planted
    multilinear rank is the dominant structure)."""
    g = rng(seed)
    i = g.integers(0, l, size=draws)
    j = g.integers(0, m, size=draws)
    k = g.integers(0, n, size=draws)
    noise = g.standard_normal(draws)
    U0 = orthonormal(g, l, r[0])
    V0 = orthonormal(g, m, r[1])
    W0 = orthonormal(g, n, r[2])
    F0 = g.standard_normal(tuple(r))
    sig = np.einsum("za,zb,zc,abc->z", U0[i], V0[j], W0[k], F0, optimize=True)
    ns, ss = float(np.linalg.norm(noise)), float(np.linalg.norm(sig))
    alpha = snr * ns / ss if ss > 0 else 0.0
    return GenCOO(l, m, n, i.astype(np.int32), j.astype(np.int32), k.astype(np.int32),
                  noise + alpha * sig)


def general_noisy_planted(seed: int, dims=(40, 30, 12), r=(2, 2, 2), rho: float = 0.3):
    """A dense general tensor: (U0,V0,W0).F0 of exact multilinear rank r
    plus N(0,1) noise scaled to rho times its norm, as a COO of every
    entry (a well-separated problem with a unique nearby optimum)."""
    T, _, _, _, _ = general_dense_planted(seed, *dims, r)
    g = rng(seed + 1000)
    N = g.standard_normal(T.shape)
    return general_dense_to_coo(T + rho * np.linalg.norm(T) / np.linalg.norm(N) * N)
