"""Hierarchical permutation of toroidal lattices (Section 3 of arXiv:1302.4018).

Oracle (test infrastructure only).  Everything is written with explicit bit
strings, the way Section 3 states it: ``dec2bin``/``bin2dec``, the red-black
table built by the counters of Algorithms 2 and 3, and the per-level bit
tables of Algorithms 4 and 5.  None of it uses the closed form of Lemma 4;
the CUDA library does, and the tests check one against the other.

Conventions (readings of the paper where it leaves the choice open):
  * site index i = x_1 + L_1 (x_2 + L_2 (x_3 + ...)), x_1 varies fastest;
    dimension j = 1 supplies the most significant bit of each bit section;
  * the section of level 1 (least significant coordinate bits) forms the most
    significant bits of ``loc`` (Section 3, 1-D case: loc = bit reversal);
  * ``loc`` is the 0-based inverse permutation ``iperm`` (Section 2.1 end,
    Section 3 1-D case): site x sits at position loc(x) of the ordering;
  * for L_j = 2^{k_j} p_j with p_j odd, the binary levels use the k_j low bits
    of x_j; then one three-colour level (theorem of Section 3.4) is applied
    on the torus of q_j = floor(x_j / 2^{k_j}) of sizes p_j, and sites of one
    colour are kept in lexicographic q order (q_1 fastest).
"""
from __future__ import annotations

from typing import List, Sequence


# ---------------------------------------------------------------- bit helpers
def dec2bin(value: int, nbits: int) -> List[int]:
    """Binary representation, most significant bit first (Section 3 notation)."""
    assert 0 <= value < (1 << nbits) or nbits == 0 and value == 0
    return [(value >> (nbits - 1 - t)) & 1 for t in range(nbits)]


def bin2dec(bits: Sequence[int]) -> int:
    """Inverse of dec2bin: first bit is the most significant."""
    v = 0
    for b in bits:
        v = 2 * v + int(b)
    return v


def two_adic(n: int) -> tuple[int, int]:
    """Split n = 2^k * p with p odd; returns (k, p)."""
    k = 0
    while n % 2 == 0:
        n //= 2
        k += 1
    return k, n


# ------------------------------------------------- red-black of the 2^d torus
def rb_table_slow(d: int) -> List[int]:
    """Algorithm 2: red-black order of the two-point d-dimensional torus.

    Corner i is red when dec2bin(i) has an even number of ones.  Reds receive
    the positions 0, 1, ... in the order met, blacks 2^{d-1}, ...  Entry i is
    the integer value of the d-bit string ``newbits``.
    """
    rb = [0] * (1 << d)
    reds, blacks = 0, 1 << (d - 1) if d > 0 else 0
    for i in range(1 << d):
        if sum(dec2bin(i, d)) % 2 == 0:
            newbits = dec2bin(reds, d)
            reds += 1
        else:
            newbits = dec2bin(blacks, d)
            blacks += 1
        rb[i] = bin2dec(newbits)
    return rb


def colors_fast(d: int) -> List[int]:
    """Colours c_d of the 2-point d-torus by c_j = [c_{j-1}, not c_{j-1}] (Algorithm 3)."""
    c = [0]
    for _ in range(d):
        c = c + [1 - v for v in c]
    return c


def rb_table_fast(d: int) -> List[int]:
    """Algorithm 3: the same table as Algorithm 2, colours from ``colors_fast``."""
    c = colors_fast(d)
    rb = [0] * (1 << d)
    reds, blacks = 0, 1 << (d - 1) if d > 0 else 0
    for i in range(1 << d):
        if c[i] == 0:
            newbits = dec2bin(reds, d)
            reds += 1
        else:
            newbits = dec2bin(blacks, d)
            blacks += 1
        rb[i] = bin2dec(newbits)
    return rb


def rb_sub_table(rb_d: Sequence[int], d: int, m: int) -> List[int]:
    """RB_m from RB_d by the theorem of Section 3.3: RB_m(i) = floor(RB_d(i 2^{d-m}) / 2^{d-m})."""
    f = 1 << (d - m)
    return [rb_d[i * f] // f for i in range(1 << m)]


# ------------------------------------------------------ lattice permutation
def coords_of(site: int, dims: Sequence[int]) -> List[int]:
    """Coordinates (x_1, ..., x_d) of a lexicographic site index, x_1 fastest."""
    x = []
    for L in dims:
        x.append(site % L)
        site //= L
    return x


def lattice_hier_permutation0(x: Sequence[int], k: int, rb: Sequence[int]) -> int:
    """Algorithm 4 (all k_j = k): concatenate RB(bits of section m) for m = 1..k."""
    d = len(x)
    table = [dec2bin(xj, k) for xj in x]          # row j = (b^j_k, ..., b^j_1)
    loc: List[int] = []
    for m in range(1, k + 1):
        section = [table[j][k - m] for j in range(d)]   # (b^1_m, ..., b^d_m)
        s = dec2bin(rb[bin2dec(section)], d)
        loc = loc + s
    return bin2dec(loc)


def lattice_hier_permutation(x: Sequence[int], ks: Sequence[int], rb: Sequence[int]) -> int:
    """Algorithm 5 (unequal k_j): only dimensions with m <= k_j take part in section m.

    The section's bits are scaled by 2^{d - active} to index the d-dimensional
    table RB and the result is scaled back down (theorem of Section 3.3).
    Returns the binary part of loc (sum(ks) bits).
    """
    d = len(x)
    kmax = max(ks) if ks else 0
    table = [dec2bin(x[j] % (1 << ks[j]), ks[j]) for j in range(d)]
    loc: List[int] = []
    for m in range(1, kmax + 1):
        bits: List[int] = []
        active = 0
        for j in range(d):
            if m <= ks[j]:
                bits = bits + [table[j][ks[j] - m]]
                active += 1
        index = bin2dec(bits) * (1 << (d - active))
        s = rb[index] // (1 << (d - active))
        loc = loc + dec2bin(s, active)
    return bin2dec(loc)


# ------------------------------------------------- odd factors: 3-colouring
def three_color(q: Sequence[int], n: Sequence[int]) -> int:
    """Theorem of Section 3.4: C(x) = (sum x_i + sum delta(x_i)) mod 3,
    delta(x_i) = 1 iff x_i = n_i - 1 and (n_i - 1) mod 3 = 0."""
    s = 0
    for qi, ni in zip(q, n):
        delta = 1 if (qi == ni - 1 and (ni - 1) % 3 == 0) else 0
        s += qi + delta
    return s % 3


class OddLevel:
    """The colour classes of the q-torus (sizes p_j) and each point's rank in its class."""

    def __init__(self, p: Sequence[int]):
        self.p = list(p)
        self.Q = 1
        for v in p:
            self.Q *= v
        self.color = []
        for t in range(self.Q):
            self.color.append(three_color(coords_of(t, p), p))
        self.sizes = [self.color.count(c) for c in range(3)]
        self.rank = []
        seen = [0, 0, 0]
        for t in range(self.Q):
            c = self.color[t]
            self.rank.append(seen[c])
            seen[c] += 1
        self.equal = self.Q > 1 and self.sizes[0] == self.sizes[1] == self.sizes[2]

    def position(self, q: Sequence[int]) -> int:
        """Position inside the binary class: colours in order 0, 1, 2, then rank."""
        t = 0
        for qj, pj in zip(reversed(q), reversed(self.p)):
            t = t * pj + qj
        c = self.color[t]
        return sum(self.sizes[:c]) + self.rank[t]


class LatticeOrder:
    """loc(x) for every site of a torus with sizes ``dims`` (any d >= 1)."""

    def __init__(self, dims: Sequence[int]):
        self.dims = [int(v) for v in dims]
        self.d = len(self.dims)
        kp = [two_adic(L) for L in self.dims]
        self.ks = [k for k, _ in kp]
        self.p = [p for _, p in kp]
        self.K = sum(self.ks)
        self.rb = rb_table_fast(self.d)
        self.odd = OddLevel(self.p)
        self.Q = self.odd.Q
        self.V = 1
        for L in self.dims:
            self.V *= L

    def loc(self, site: int) -> int:
        x = coords_of(site, self.dims)
        lb = lattice_hier_permutation(x, self.ks, self.rb)
        q = [x[j] >> self.ks[j] for j in range(self.d)]
        return lb * self.Q + self.odd.position(q)

    def all_loc(self) -> List[int]:
        return [self.loc(i) for i in range(self.V)]


def hierarchical_loc(dims: Sequence[int], sites: Sequence[int] | None = None) -> List[int]:
    """loc for the given sites (default: all sites, pure Python, keep V small)."""
    order = LatticeOrder(dims)
    if sites is None:
        return order.all_loc()
    return [order.loc(int(i)) for i in sites]
