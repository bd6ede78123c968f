"""Seeded synthetic instance generators shared by the tests, the bench and the smoke run.

This module only draws random *data*: graphs, coupling bit-planes, coupling matrices and
size lists.  It holds none of the simulation method's arithmetic (no colouring, no Metropolis
rule, no random numbers drawn by the dynamics, no measurement), so both the CPU oracle and the
CUDA path can consume its output without sharing any method code.

Instance families (paper workloads, restated):
  * Viana-Bray on a Poissonian random graph with mean degree c, J = +-1 equiprobable
    (Eq. 3; the paper itself uses a random regular graph of degree 4).  Couplings are stored
    as 64-bit lane words: bit k = 1 means J = -1 for disorder sample k (SI section 2,
    multispin coding, Table 1 caption: 64 coupling sets per graph).
  * Random regular graph of degree z (the paper's own ensemble, main text after Eq. 3), and its
    bipartite form (the random regular bipartite graph the paper simulates on GPUs, SI section
    3): halves [0, N/2) and [N/2, N), every edge across, so that greedy colouring in vertex
    order yields exactly the two halves.
  * Sherrington-Kirkpatrick with binary symmetric couplings J_ij = +-1, J_ii = 0
    (SI section 1; the 1/sqrt(N) scale is folded into the inverse temperature).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "poisson_graph",
    "regular_graph",
    "random_regular_graph",
    "vb_lane_couplings",
    "sk_couplings",
    "log_uniform_sizes",
    "csr_from_edges",
    "log_schedule",
    "geometric_windows",
    "tritone_windows",
]


def csr_from_edges(n: int, ei: np.ndarray, ej: np.ndarray):
    """Symmetric CSR (row_ptr int32[n+1], col int32[2M]) of an undirected simple edge list.

    Each row's neighbours are sorted ascending.  Also returns, for every directed entry, the
    index of its undirected edge (int64[2M]) so that per-edge data can be mirrored.
    """
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    m = ei.size
    src = np.concatenate([ei, ej])
    dst = np.concatenate([ej, ei])
    eid = np.concatenate([np.arange(m), np.arange(m)])
    order = np.argsort(src * n + dst)  # keys are distinct
    src, dst, eid = src[order], dst[order], eid[order]
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("too many edges for int32 CSR")
    return row_ptr.astype(np.int32), dst.astype(np.int32), eid


def poisson_graph(n: int, c: float, seed: int):
    """Erdos-Renyi G(N, M) graph with M = round(c*N/2) distinct edges, no self-loops.

    The degree distribution is Poisson(c) for large N (the Viana-Bray ensemble).  Returns
    (row_ptr, col, edge_id) as in csr_from_edges.
    """
    if n < 2:
        raise ValueError("need N >= 2")
    m = int(round(c * n / 2.0))
    maxm = n * (n - 1) // 2
    if m > maxm:
        raise ValueError("too many edges requested")
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0001, seed]))
    keys = np.empty(0, dtype=np.int64)
    while True:
        # distinct uniform unordered pairs; a uniform m-subset of them is a uniform G(N, M)
        k = m - keys.size + 64 + (m - keys.size) // 64
        a = rng.integers(0, n, size=k, dtype=np.int64)
        b = rng.integers(0, n, size=k, dtype=np.int64)
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        keys = np.sort(np.concatenate([keys, lo * n + hi]))
        keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
        if keys.size >= m:
            break
    keys = np.sort(rng.choice(keys, size=m, replace=False))
    ei, ej = keys // n, keys % n
    return csr_from_edges(n, ei, ej)


def regular_graph(n: int, z: int, seed: int, max_tries: int = 200):
    """Random z-regular simple graph by the configuration model with rejection of bad pairings.

    Stub pairings that produce a self-loop or a multi-edge are redrawn as a whole; the
    accepted graph is uniform over simple z-regular graphs.  Intended for small-to-moderate N.
    """
    if (n * z) % 2:
        raise ValueError("N*z must be even")
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0002, seed]))
    stubs = np.repeat(np.arange(n, dtype=np.int64), z)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo * n + hi
        if np.unique(keys).size != keys.size:
            continue
        return csr_from_edges(n, lo, hi)
    raise RuntimeError("could not draw a simple regular graph; raise max_tries")


def random_regular_graph(n: int, z: int, seed: int, bipartite: bool = False):
    """Random z-regular simple graph for any N, by stub pairing with local repair.

    Stubs are paired by one random permutation; every pairing that makes a self-loop or repeats
    an edge then swaps its partner stub with that of a uniformly chosen other pairing, until the
    graph is simple (degrees never change).  The result is close to, not exactly, uniform over
    simple z-regular graphs, as in common practice for large N.  bipartite=True pairs the stubs
    of the first half [0, N/2) with those of the second half only (N even).  Returns
    (row_ptr, col, edge_id) as in csr_from_edges.
    """
    if bipartite and n % 2:
        raise ValueError("a bipartite regular graph needs even N")
    if (n * z) % 2:
        raise ValueError("N*z must be even")
    if z >= (n // 2 if bipartite else n):
        raise ValueError("degree too large for N")
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0006, seed, int(bipartite)]))
    if bipartite:
        h = n // 2
        a = np.repeat(np.arange(h, dtype=np.int64), z)
        b = rng.permutation(np.repeat(np.arange(h, n, dtype=np.int64), z))
    else:
        perm = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), z))
        a, b = perm[0::2].copy(), perm[1::2].copy()
    m = a.size
    for _ in range(10000):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo * n + hi
        order = np.argsort(keys, kind="stable")
        dup = np.zeros(m, dtype=bool)
        dup[order[1:]] = keys[order[1:]] == keys[order[:-1]]
        bad = np.flatnonzero(dup | (a == b))
        if bad.size == 0:
            return csr_from_edges(n, lo, hi)
        other = rng.integers(0, m, size=bad.size)
        for i, j in zip(bad, other):  # swap partner stubs (both sides keep their degrees)
            b[i], b[j] = b[j], b[i]
    raise RuntimeError("could not repair the pairing into a simple graph")


def vb_lane_couplings(edge_id: np.ndarray, n_edges: int, seed: int) -> np.ndarray:
    """+-1 couplings for 64 disorder samples per edge, as one uint64 word per directed entry.

    Bit k of the word is 1 when J_ij = -1 in sample k; both directions of an edge carry the
    same word (J is symmetric).
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0003, seed]))
    words = rng.integers(0, 2**64, size=n_edges, dtype=np.uint64, endpoint=False)
    return words[np.asarray(edge_id, dtype=np.int64)]


def sk_couplings(n: int, seed: int) -> np.ndarray:
    """Dense symmetric +-1 coupling matrix (int8, row-major N x N) with a zero diagonal."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0004, seed]))
    bits = rng.integers(0, 2, size=(n, n), dtype=np.int8)
    upper = np.triu(1 - 2 * bits, k=1).astype(np.int8)
    return (upper + upper.T).astype(np.int8)


def log_uniform_sizes(count: int, lo_exp: float, hi_exp: float, seed: int) -> np.ndarray:
    """count sizes N = round(2**U) with U ~ Uniform[lo_exp, hi_exp] (uneven-batch workloads)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED_0005, seed]))
    u = rng.uniform(lo_exp, hi_exp, size=count)
    return np.round(2.0 ** u).astype(np.int64)


def log_schedule(tw, t_max: int):
    """Snapshot times tw and measurement times {t_w + 2^k <= t_max} united with tw itself.

    Measurements at log-spaced times after each waiting time (main text: t_w = 2^2..2^12 and
    t up to 2^25; SI section 1: t_w = 3).  Returns (tw sorted unique, tm sorted unique).
    """
    tw = sorted({int(x) for x in tw if 0 <= int(x) <= t_max})
    tm = set(tw)
    for w in tw:
        k = 0
        while w + (1 << k) <= t_max:
            tm.add(w + (1 << k))
            k += 1
    return np.array(tw, dtype=np.int64), np.array(sorted(tm), dtype=np.int64)


def geometric_windows(t_min: int, t_max: int, ratio_log2: float = 0.25):
    """Window bounds for averaging over geometric time windows [t_m, t_{m+1}) with
    t_{m+1} / t_m = 2^ratio_log2 (2^(1/4): the "minor thirds" of the main text), from t_min
    (>= 1) until t_max is covered; bounds are the distinct integer ceilings."""
    if t_min < 1:
        raise ValueError("t_min must be >= 1")
    b, k = [], 0
    while True:
        v = int(np.ceil(t_min * 2.0 ** (k * ratio_log2) - 1e-9))
        if not b or v > b[-1]:
            b.append(v)
        if v > t_max:
            return np.array(b, dtype=np.int64)
        k += 1


def tritone_windows(t_max: int, t0: int = 4):
    """Window bounds of the SK "tritone" lumps (SI section 1): the times T = t + t_w >= t0 with
    the same floor(ln(T / t0) / (0.5 ln 2)) form one lump, so lump j = [t0 2^(j/2), t0 2^((j+1)/2)).
    Evaluated on every integer T up to t_max exactly as written (double precision)."""
    T = np.arange(t0, t_max + 2, dtype=np.int64)
    j = np.floor(np.log(T / t0) / (0.5 * np.log(2.0))).astype(np.int64)
    starts = np.flatnonzero(np.concatenate([[True], j[1:] != j[:-1]]))
    return T[starts]
