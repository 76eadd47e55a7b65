"""Pins of the oracle's hierarchical permutation (Section 3) against what the paper fixes."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

from conftest import read_golden
from oracle import permutation as P
from pins import torus_distance


def test_rb_2d_order_golden():
    # Section 3.2: sublattices ordered (00 11 01 10)
    rows = read_golden("rb_order_2d.txt")
    rb = P.rb_table_fast(2)
    for bits, pos in rows:
        assert rb[int(bits, 2)] == int(pos)
    assert P.rb_table_slow(2) == rb


def test_colors_golden_and_thue_morse():
    rows = {r[0]: [int(v) for v in r[1:]] for r in read_golden("colors_c2.txt")}
    assert P.colors_fast(1) == rows["c1"]
    assert P.colors_fast(2) == rows["c2"]
    for d in range(1, 9):
        c = P.colors_fast(d)
        # neighbours on the 2-point torus (differ in one bit) have opposite colours
        for i in range(1 << d):
            for j in range(d):
                assert c[i] != c[i ^ (1 << j)]


@pytest.mark.parametrize("d", range(1, 9))
def test_alg2_equals_alg3(d):
    assert P.rb_table_slow(d) == P.rb_table_fast(d)


@pytest.mark.parametrize("d", range(2, 9))
def test_lemmas_of_section_3_3(d):
    c = P.colors_fast(d)
    cm = P.colors_fast(d - 1)
    rb = P.rb_table_fast(d)
    for i in range(1 << (d - 1)):
        assert c[2 * i] == cm[i]                 # first lemma
        assert c[2 * i] != c[2 * i + 1]          # second lemma
    for i in range(1 << d):                      # third lemma: values of RB_d
        assert rb[i] == i // 2 + c[i] * (1 << (d - 1))
    for m in range(1, d):                        # theorem: RB_m from RB_d
        assert P.rb_sub_table(rb, d, m) == P.rb_table_fast(m)


@pytest.mark.parametrize("k", range(1, 13))
def test_1d_is_bit_reversal(k):
    # Section 3: on the 1-D torus of 2^k points P(x) = bin2dec(bitreverse(dec2bin(x)))
    L = 1 << k
    loc = P.hierarchical_loc([L])
    for x in range(L):
        assert loc[x] == int(format(x, "0%db" % k)[::-1], 2)


@pytest.mark.parametrize("dims", [(4, 4), (8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2)])
def test_alg4_equals_alg5_for_equal_sizes(dims):
    k = P.two_adic(dims[0])[0]
    rb = P.rb_table_fast(len(dims))
    order = P.LatticeOrder(dims)
    for site in range(order.V):
        x = P.coords_of(site, dims)
        assert P.lattice_hier_permutation0(x, k, rb) == order.loc(site)


@pytest.mark.parametrize("dims", [(4, 4), (2, 4, 8), (1, 4, 2, 8), (4, 4, 4, 8), (6, 6, 6, 6), (3, 3, 3, 3),
                                  (12, 6), (5, 4), (10, 6, 2), (7,), (12, 12, 12, 12)])
def test_loc_is_a_bijection(dims):
    loc = P.hierarchical_loc(dims)
    assert sorted(loc) == list(range(len(loc)))


@pytest.mark.parametrize("dims", [(4, 4), (8, 4, 2), (4, 4, 4, 4), (2, 8, 4, 16)])
def test_first_level_is_red_black(dims):
    # Section 3.1: the first-level colour of a site is (sum_j b^j_1) mod 2 = parity of sum x_j
    order = P.LatticeOrder(dims)
    for site in range(order.V):
        x = P.coords_of(site, dims)
        assert order.loc(site) >> (order.K - 1) == sum(x) % 2


def _torus_graph(dims):
    V = int(np.prod(dims))
    rows, cols = [], []
    for i in range(V):
        x = P.coords_of(i, dims)
        for mu in range(len(dims)):
            for s in (1, -1):
                y = list(x)
                y[mu] = (y[mu] + s) % dims[mu]
                j = sum(y[t] * int(np.prod(dims[:t])) for t in range(len(dims)))
                rows.append(i)
                cols.append(j)
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(V, V))


@pytest.mark.parametrize("dims", [(16, 16), (8, 8, 8), (4, 4, 4, 4), (8, 8, 8, 8), (4, 8, 4, 8)])
def test_distance_colouring_by_bfs(dims):
    """Section 3.3: level m gives a distance-2^m colouring with 2^{dm+1} colours.

    Colours after level m are the leading d*m + 1 bits of loc.  Brute-force
    BFS on the torus graph checks that sites sharing a colour are more than
    2^m apart (the paper's claim) and in fact at least 2^{m+1} apart.
    """
    d = len(dims)
    order = P.LatticeOrder(dims)
    loc = np.array(order.all_loc())
    dist = shortest_path(_torus_graph(dims), unweighted=True, directed=False)
    kmin = min(order.ks)
    for m in range(0, kmin):
        nbits = d * m + 1
        color = loc >> (order.K - nbits)
        assert len(set(color.tolist())) == 2 ** (d * m + 1)
        same = color[:, None] == color[None, :]
        np.fill_diagonal(same, False)
        assert dist[same].min() >= 2 ** (m + 1)


def test_completion_points_golden():
    (row,) = read_golden("completion_points.txt")
    assert [2 ** (4 * m + 1) for m in range(3)] == [int(v) for v in row[1:]]


def test_three_colouring_theorem_brute_force():
    # Theorem of Section 3.4: unit-distance neighbours get different colours
    for n in range(2, 41):
        for x in range(n):
            assert P.three_color([x], [n]) != P.three_color([(x + 1) % n], [n])
    for n1, n2 in itertools.product(range(2, 14), repeat=2):
        for x1 in range(n1):
            for x2 in range(n2):
                c = P.three_color([x1, x2], [n1, n2])
                assert c != P.three_color([(x1 + 1) % n1, x2], [n1, n2])
                assert c != P.three_color([x1, (x2 + 1) % n2], [n1, n2])


def test_odd_level_classes():
    o = P.OddLevel([3, 3, 3, 3])
    assert o.sizes == [27, 27, 27] and o.equal
    assert not P.OddLevel([5]).equal
    # sites of one colour class inside a binary class are never torus neighbours
    dims = (12, 12)
    order = P.LatticeOrder(dims)
    for site in range(order.V):
        x = P.coords_of(site, dims)
        q = [x[j] >> order.ks[j] for j in range(2)]
        for mu in range(2):
            y = list(q)
            y[mu] = (y[mu] + 1) % order.p[mu]
            assert P.three_color(q, order.p) != P.three_color(y, order.p)


def test_odd_level_keeps_binary_prefix():
    # the odd level only reorders sites inside one binary colour class
    dims = (12, 6, 4)
    order = P.LatticeOrder(dims)
    for site in range(order.V):
        x = P.coords_of(site, dims)
        lb = P.lattice_hier_permutation(x, order.ks, order.rb)
        assert order.loc(site) // order.Q == lb
