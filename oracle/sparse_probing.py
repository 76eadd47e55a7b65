"""Hierarchical probing of a general sparse matrix (Section 2: Algorithm 1 and Section 2.2).

Oracle (test infrastructure only): plain, slow restatements.

* ``greedy_color`` -- a greedy colouring (vertices in natural order, each takes
  the smallest colour none of its already coloured neighbours has), the kind
  of colouring Algorithm 1 calls GreedyColor.
* ``hierarchical_coloring`` -- Algorithm 1 run literally: colour the block,
  stop if the block is dense or diagonal, order the rows by colour
  (Colors2Perm), and recurse into each colour with the block matrix
  Ablock(rows, :) * Ablock(:, rows).  Besides perm and the (start, end, level)
  records it returns every vertex's colour at each level (its colour path).
* ``path_phases`` -- the probing vectors of Eq. (Hperm-general-recursive) for a
  colour hierarchy: with the radix c(k) of level k, vector m (mixed-radix digits
  d_k(m), the level-1 digit least significant) has entry
      z_m(i) = prod_k exp(2 pi i d_k(m) col_k(i) / c(k)),
  so the first gamma_k = c(1)...c(k) vectors resolve levels 1..k.  Reading of
  the open case of Section 2.2 (blocks of one level coloured with different
  numbers of colours): c(k) is the largest colour count of level k, so the
  construction never needs equal block sizes; a vertex whose block stopped
  recursing keeps colour 0 below it.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np
import scipy.sparse as sp


def greedy_color(A: sp.csr_matrix) -> np.ndarray:
    """Colours 0.. of the graph of A (off-diagonal non-zeros), vertices in natural order."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    col = -np.ones(n, dtype=np.int64)
    for v in range(n):
        used = set()
        for k in range(A.indptr[v], A.indptr[v + 1]):
            u = A.indices[k]
            if u != v and col[u] >= 0:
                used.add(int(col[u]))
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return col


def colors_to_perm(colors: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Colors2Perm: the local order with vertices of one colour adjacent (stable), and the number
    of rows per colour."""
    order = np.argsort(colors, kind="stable")
    counts = np.bincount(colors, minlength=int(colors.max()) + 1 if len(colors) else 0)
    return order, counts


def hierarchical_coloring(A: sp.csr_matrix, max_levels: int = 32):
    """Algorithm 1 on A.  Returns (perm, offsets, paths): perm[k] = original row at position k,
    offsets = [(start, end, level)] of every block visited (0-based, end inclusive), and
    paths[i, l] = colour of vertex i at level l + 1 (0 where its block stopped before)."""
    A = sp.csr_matrix(A, dtype=float)
    n = A.shape[0]
    perm = np.arange(n)
    offsets: List[Tuple[int, int, int]] = []
    paths = np.zeros((n, max_levels), dtype=np.int64)
    pattern = sp.csr_matrix((np.ones_like(A.data), A.indices, A.indptr), shape=A.shape)

    def recurse(Ablock: sp.csr_matrix, start: int, end: int, level: int) -> None:
        offsets.append((start, end, level))
        if level > max_levels:
            return
        colors = greedy_color(Ablock)
        num = int(colors.max()) + 1
        rows_global = perm[start:end + 1].copy()
        paths[rows_global, level - 1] = colors
        if num == end - start + 1 or num == 1:
            return                                   # dense or diagonal block: keep the order
        order, counts = colors_to_perm(colors)
        perm[start:end + 1] = rows_global[order]
        cstart = start
        local_start = 0
        for c in range(num):
            rows_local = order[local_start:local_start + counts[c]]
            sub = Ablock[rows_local, :] @ Ablock[:, rows_local]
            sub = sp.csr_matrix(sub)
            sub.data[:] = 1.0
            recurse(sub, cstart, cstart + counts[c] - 1, level + 1)
            cstart += counts[c]
            local_start += counts[c]

    recurse(pattern, 0, n - 1, 1)
    return perm, offsets, paths


def radices(paths: np.ndarray) -> List[int]:
    """c(k): the largest colour count of each level, trailing levels of one colour dropped."""
    c = [int(paths[:, l].max()) + 1 for l in range(paths.shape[1])]
    while c and c[-1] == 1:
        c.pop()
    return c


def path_phases(paths: np.ndarray, first: int, count: int, z0_seed: int = 0) -> Tuple[np.ndarray, int]:
    """Integer phases of v_m = z_0 (.) z_m, m = first..first+count-1, over the period
    P = lcm(2, c(1), c(2), ...): z_m(i) = exp(2 pi i phase / P)."""
    from math import lcm

    from .probing import z0_signs

    c = radices(paths)
    P = 2
    for r in c:
        P = lcm(P, r)
    n = paths.shape[0]
    z0 = z0_signs(z0_seed, n)
    out = np.zeros((count, n), dtype=np.int64)
    for t in range(count):
        m = first + t
        ph = np.zeros(n, dtype=np.int64)
        rest = m
        for k, r in enumerate(c):
            d = rest % r
            rest //= r
            ph += (P // r) * ((d * paths[:, k]) % r)
        if rest:
            raise ValueError("vector index beyond the hierarchy's prod c(k)")
        out[t] = (ph + np.where(z0 < 0, P // 2, 0)) % P
    return out, P


def quadratures_of_phases(A: sp.csr_matrix, phases: np.ndarray, P: int) -> np.ndarray:
    """q_m = v_m^H A^-1 v_m (Section 1.1.2) for v_m(i) = exp(2 pi i phases[m, i] / P), by a dense
    solve (small matrices)."""
    from .probing import probe_values

    W = probe_values(phases, P)
    X = np.linalg.solve(A.toarray(), W.T)
    return np.array([np.vdot(W[m], X[:, m]) for m in range(W.shape[0])])


def sparse_quadratures(A: sp.csr_matrix, paths: np.ndarray, first: int, count: int, z0_seed: int) -> np.ndarray:
    """q_m for the path probing vectors m = first .. first+count-1."""
    ph, P = path_phases(paths, first, count, z0_seed)
    return quadratures_of_phases(A, ph, P)
