"""Pins of the general sparse-matrix path (Algorithm 1 and the basis of Section 2.2)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

from oracle import operators as O
from oracle import sparse_probing as SP
from oracle.probing import probe_values


def ring_laplacian(n, m=0.3):
    A = sp.lil_matrix((n, n))
    for i in range(n):
        A[i, i] = 2 + m
        A[i, (i + 1) % n] -= 1
        A[i, (i - 1) % n] -= 1
    return sp.csr_matrix(A)


def random_spd(n, deg, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in rng.choice(n, deg, replace=False):
            if j != i:
                rows += [i, j]
                cols += [j, i]
    G = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    G.data[:] = 1.0
    L = sp.diags(np.asarray(G.sum(axis=1)).ravel()) - G
    return sp.csr_matrix(L + 0.5 * sp.eye(n))


def test_ring_gives_bit_reversal():
    """On a ring of 2^K sites, Algorithm 1 with natural-order greedy colouring reproduces the 1-D
    hierarchical permutation of Section 3: bit reversal of the index."""
    K = 5
    n = 1 << K
    perm, offsets, paths = SP.hierarchical_coloring(ring_laplacian(n))
    rev = [int(format(i, "0%db" % K)[::-1], 2) for i in range(n)]
    assert list(perm) == rev
    assert SP.radices(paths) == [2] * K
    assert offsets[0] == (0, n - 1, 1)


def test_ring_color_offsets_are_the_dyadic_intervals():
    """On the ring of 2^K sites every block splits into its two colours down to blocks of two
    (which the distance-2^(K-1) graph joins: dense, so the recursion stops there), so colorOffsets
    is the list of dyadic intervals of sizes 2^K .. 2 in pre-order, interval j of size n / 2^(l-1)
    at level l."""
    K = 5
    n = 1 << K
    _, offsets, _ = SP.hierarchical_coloring(ring_laplacian(n))

    def dyadic(start, size, level):
        out = [(start, start + size - 1, level)]
        if size > 2:
            out += dyadic(start, size // 2, level + 1) + dyadic(start + size // 2, size // 2, level + 1)
        return out

    assert offsets == dyadic(0, n, 1)


def test_torus_first_level_is_red_black():
    dims = (8, 6)
    A = sp.csr_matrix(O.laplacian_dense(dims, 0.1))
    _, _, paths = SP.hierarchical_coloring(A)
    x = np.arange(48) % 8
    y = np.arange(48) // 8
    assert np.array_equal(paths[:, 0], (x + y) % 2)


@pytest.mark.parametrize("n,deg,seed", [(60, 3, 1), (90, 2, 2), (40, 5, 3)])
def test_levels_colour_their_block_graphs(n, deg, seed):
    """Level 1 properly colours A; vertices sharing colours down to level 2 are more than 2 edges
    apart (level 2 colours A^2 over the whole first block), checked with breadth-first distances;
    every level k properly colours its block graph, built here with whole-matrix masks: G_1 = A,
    G_{k+1}(u, w) = OR_v G_k(u, v) G_k(v, w) over v in the block of u at level k, u and w of the
    same colour (Algorithm 1: Ablock(rows, :) * Ablock(:, rows))."""
    A = random_spd(n, deg, seed)
    _, offsets, paths = SP.hierarchical_coloring(A)
    L = len(SP.radices(paths))
    eye = np.eye(n, dtype=bool)
    same = [np.ones((n, n), dtype=bool)] + [np.all(paths[:, None, :k] == paths[None, :, :k], axis=2)
                                           for k in range(1, L + 1)]
    D = shortest_path(sp.csr_matrix(A != 0), unweighted=True)
    assert np.all(D[same[1] & ~eye] >= 2) and np.all(D[same[2] & ~eye] >= 3)
    G = (A != 0).toarray()
    for k in range(1, L + 1):
        assert not np.any(G & same[k] & ~eye), k             # proper colouring of the level-k graph
        Gi = G.astype(np.int64)
        nxt = np.zeros((n, n), dtype=bool)
        for u in range(n):
            mid = G[u] & same[k - 1][u]                       # neighbours of u inside its block
            nxt[u] = (Gi[mid].sum(axis=0) > 0) & same[k][u]
        G = nxt
    assert len({(s, e) for s, e, lvl in offsets if lvl == 1}) == 1


@pytest.mark.parametrize("seed", [1, 2])
def test_path_basis_probes_exactly_at_completion_points(seed):
    """sum_{m < gamma_k} z_m z_m^H = gamma_k [same colour path down to level k] (Section 2.2: the
    first gamma_k vectors of the nested basis resolve the first k levels)."""
    A = random_spd(50, 3, seed)
    _, _, paths = SP.hierarchical_coloring(A)
    c = SP.radices(paths)
    gamma = 1
    for k, r in enumerate(c, start=1):
        gamma *= r
        ph, P = SP.path_phases(paths, 0, gamma)
        Z = probe_values(ph, P)
        C = Z.T @ Z.conj()
        same = np.all(paths[:, None, :k] == paths[None, :, :k], axis=2)
        assert np.allclose(C, gamma * same, atol=1e-9 * gamma)


def test_full_basis_is_exact_when_paths_are_unique():
    """With every colour path distinct the full nested sequence gives Tr A^-1 exactly (s = prod c(k))."""
    A = ring_laplacian(16, 0.2)
    _, _, paths = SP.hierarchical_coloring(A)
    assert len({tuple(p) for p in paths}) == 16
    s = int(np.prod(SP.radices(paths)))
    q = SP.sparse_quadratures(A, paths, 0, s, z0_seed=7)
    assert abs(q.sum().real / s - np.trace(np.linalg.inv(A.toarray()))) <= 1e-12 * np.trace(np.linalg.inv(A.toarray()))


# ------------------------------------------------------------ the seeded sparse inputs
def test_csr_from_entries_merges_and_sorts():
    from paper_1302_4018_gb300 import synth

    rp, ci, v = synth.csr_from_entries(4, [2, 0, 2, 0, 3], [1, 3, 1, 0, 3], [1.0, 2.0, 3.0, 4.0, 5.0])
    A = sp.csr_matrix((v, ci, rp), shape=(4, 4)).toarray()
    expect = np.zeros((4, 4))
    expect[2, 1], expect[0, 3], expect[0, 0], expect[3, 3] = 4.0, 2.0, 4.0, 5.0
    assert np.array_equal(A, expect)
    assert rp.dtype == np.int32 and ci.dtype == np.int32
    for i in range(4):   # column indices sorted within each row
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


@pytest.mark.parametrize("dims", [(7,), (4, 6), (3, 4, 5), (2, 3)])
def test_grid_matrix_is_a_renumbered_weighted_laplacian(dims):
    """Symmetric, row sums = shift, off-diagonal weights in [0.5, 1.5] (per distinct neighbour),
    and the renumbered matrix is a symmetric permutation of the unrenumbered one's pattern."""
    from paper_1302_4018_gb300 import synth

    n = int(np.prod(dims))
    rp, ci, v = synth.grid_matrix(dims, 11, shift=0.25)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    assert np.allclose(A, A.T, atol=0)
    assert np.allclose(A.sum(axis=1), 0.25)
    off = -(A - np.diag(np.diag(A)))
    assert np.all(off[off != 0] >= 0.5 - 1e-12)
    assert np.linalg.eigvalsh(A).min() > 0.25 - 1e-9   # Laplacian (PSD) + 0.25 I
    rp0, ci0, v0 = synth.grid_matrix(dims, 11, shift=0.25, renumber=False)
    deg = np.sort(np.diff(rp))
    assert np.array_equal(deg, np.sort(np.diff(rp0)))


def test_random_graph_matrix_is_spd_and_random_pattern_shapes():
    from paper_1302_4018_gb300 import synth

    rp, ci, v = synth.random_graph_matrix(120, 3, 5, shift=0.1)
    A = sp.csr_matrix((v, ci, rp), shape=(120, 120)).toarray()
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > 0.1 - 1e-9
    rp, ci = synth.random_pattern(50, 2, 6, symmetric=False, diagonal=False)
    P = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(50, 50)).toarray()
    assert not np.any(np.diag(P)) and not np.allclose(P, P.T)
    rp, ci = synth.random_pattern(50, 2, 6, symmetric=True, diagonal=True)
    P = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(50, 50)).toarray()
    assert np.all(np.diag(P)) and np.allclose(P, P.T)
