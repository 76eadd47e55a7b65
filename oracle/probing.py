"""Hierarchical probing vectors (Sections 2.2 and 4 of arXiv:1302.4018).

Oracle (test infrastructure only).  Entries of the probing vectors are kept
as exact integer phases: an entry exp(2 pi i k / P) is stored as k mod P, so
the Hadamard and Fourier constructions below are exact and can be compared
bit for bit with the CUDA library.  P is a common period of every factor
(always even, so that the bias-removal sign -1 = exp(2 pi i (P/2) / P) is a
phase too).

Two independent constructions are provided:
  * ``basis_kron``: the literal Kronecker recursion of Eq. (Hperm-recursive)
    and its Fourier generalisation Eq. (Hperm-general-recursive), as whole
    matrices (small N only) or one column at a time (``basis_column``);
  * ``hadamard_element`` with the column sequence Eq. (HpermSequence) and
    the element formula Eq. (row-col-permutation), power-of-two case.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from typing import List, Sequence

import numpy as np

from .permutation import LatticeOrder

MASK64 = (1 << 64) - 1


# ------------------------------------------------------- Hadamard / Fourier
def hadamard(n: int) -> np.ndarray:
    """Sylvester construction H_2n = [[H_n, H_n], [H_n, -H_n]] (Section 1.1.4)."""
    H = np.array([[1]], dtype=np.int64)
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    assert H.shape[0] == n, "n must be a power of two"
    return H


def hadamard_element(i: int, j: int, n: int) -> int:
    """Eq. (HadamardElements), 1-based: (-1)^{sum_k i_k j_k} over the bits of i-1, j-1."""
    logn = n.bit_length() - 1
    s = 0
    for k in range(logn):
        s += (((i - 1) >> k) & 1) * (((j - 1) >> k) & 1)
    return -1 if s % 2 else 1


def fourier_phase(n: int, P: int) -> np.ndarray:
    """Eq. (FourierElements) F_n(j,k) = exp(2 pi i (j-1)(k-1)/n) as phases mod P."""
    assert P % n == 0
    j = np.arange(n, dtype=np.int64)
    return ((P // n) * np.outer(j, j)) % P


def hperm_sequence(N: int) -> List[int]:
    """Eq. (HpermSequence): 0, N/2, N/4, 3N/4, N/8, 5N/8, 3N/8, 7N/8, ...

    Each new level appends the previous entries shifted by N/2^level.
    """
    seq = [0]
    step = N
    while step > 1:
        step //= 2
        seq = seq + [v + step for v in seq]
    assert len(seq) == N
    return seq


def kron_phase(A: np.ndarray, B: np.ndarray, P: int) -> np.ndarray:
    """Kronecker product of two matrices given as phases: exponents add."""
    ra, ca = A.shape
    rb, cb = B.shape
    out = (A[:, None, :, None] + B[None, :, None, :]) % P
    return out.reshape(ra * rb, ca * cb)


def basis_kron(radices: Sequence[int], P: int) -> np.ndarray:
    """Z~^(L) of Eq. (Hperm-general-recursive) (Eq. (Hperm-recursive) when all radices are 2).

    Z~^(1) = F_{c(1)};  Z~^(k) = [Z~^(k-1) (x) F_{c(k)}(:,1), ..., Z~^(k-1) (x) F_{c(k)}(:,c(k))].
    Returns the gamma_L x gamma_L phase matrix.
    """
    Z = fourier_phase(radices[0], P)
    for c in radices[1:]:
        F = fourier_phase(c, P)
        blocks = [kron_phase(Z, F[:, j:j + 1], P) for j in range(c)]
        Z = np.concatenate(blocks, axis=1)
    return Z


def basis_column(radices: Sequence[int], P: int, m: int) -> np.ndarray:
    """Column m of Z~^(L) by the same recursion, built for one column only.

    Column j*gamma_{k-1} + m' of Z~^(k) is Z~^(k-1)(:, m') (x) F_{c(k)}(:, j).
    """
    gammas = [1]
    for c in radices:
        gammas.append(gammas[-1] * c)
    assert 0 <= m < gammas[-1]

    def column(k: int, mm: int) -> np.ndarray:
        F = fourier_phase(radices[k - 1], P)
        if k == 1:
            return F[:, mm:mm + 1]
        j, mprime = divmod(mm, gammas[k - 1])
        return kron_phase(column(k - 1, mprime), F[:, j:j + 1], P)

    return column(len(radices), m)[:, 0]


# ------------------------------------------------------ lattice basis layout
class LatticeBasis:
    """The probing sequence of a lattice: binary levels, then the odd level.

    radices = [2]*K (one per coordinate bit, Section 2.2: any power-of-two
    split per level gives the same sequence), then 3 for the three-colour
    level and R = Q/3 for the final dense level when the three colour
    classes are equal; otherwise only the first 2^K vectors exist
    (Section 2.2, open problem of unequal colour counts).
    """

    def __init__(self, dims: Sequence[int]):
        self.order = LatticeOrder(dims)
        o = self.order
        self.V, self.K, self.Q = o.V, o.K, o.Q
        self.radices = [2] * self.K
        self.tail = self.Q            # trailing 1_{N/gamma} of the last level
        if self.Q > 1 and o.odd.equal:
            R = self.Q // 3
            self.radices.append(3)
            if R > 1:
                self.radices.append(R)
            self.tail = 1
        self.n_vectors = self.V // self.tail
        P = 2
        for c in self.radices:
            P = P * c // math.gcd(P, c)
        self.P = P

    def column(self, m: int) -> np.ndarray:
        """Phases of z_m in permuted (colour) order: Z^(L)(:, m), Kronecker with 1_tail."""
        if not self.radices:                       # V == 1
            col = np.zeros(1, dtype=np.int64)
        else:
            col = basis_column(self.radices, self.P, m)
        return np.repeat(col, self.tail)

    def matrix(self) -> np.ndarray:
        """The whole Z^(L) (small N): literal Kronecker recursion."""
        if not self.radices:
            return np.zeros((1, 1), dtype=np.int64)
        return np.repeat(basis_kron(self.radices, self.P), self.tail, axis=0)


# ----------------------------------------------------------- bias removal
def splitmix64_output(seed: int, index: int) -> int:
    """Output number ``index`` (0-based) of Vigna's SplitMix64 seeded with ``seed``."""
    z = (seed + (index + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def z0_signs(seed: int, V: int) -> np.ndarray:
    """The Z_2 vector z_0 of Section 4: sign from the top bit of SplitMix64 output number ``site``.

    seed == 0 means no bias removal (z_0 = 1).
    """
    if seed == 0:
        return np.ones(V, dtype=np.int64)
    return np.array([1 - 2 * (splitmix64_output(seed, s) >> 63) for s in range(V)], dtype=np.int64)


def probe_phases(dims: Sequence[int], first: int, count: int, z0_seed: int,
                 loc: Sequence[int] | None = None) -> tuple[np.ndarray, int]:
    """Phases of v_m = z_0 (.) z_m, m = first..first+count-1, in lexicographic site order.

    z_m(i) = Z^(L)(iperm(i), m) (Eq. row-col-permutation with the Kronecker basis);
    returns (phase[count, V], P).
    """
    basis = LatticeBasis(dims)
    V, P = basis.V, basis.P
    if first < 0 or count < 0 or first + count > basis.n_vectors:
        raise ValueError("vector range outside the supported basis")
    if loc is None:
        loc = basis.order.all_loc()
    loc = np.asarray(loc, dtype=np.int64)
    z0 = z0_signs(z0_seed, V)
    shift = np.where(z0 < 0, P // 2, 0)
    out = np.empty((count, V), dtype=np.int64)
    for t in range(count):
        col = basis.column(first + t)
        out[t] = (col[loc] + shift) % P
    return out, P


def probe_phases_hadamard(dims: Sequence[int], first: int, count: int, loc: Sequence[int]) -> np.ndarray:
    """Power-of-two lattices only: z_m(i) = H_N(iperm(i), Hperm(m)) with the sequence of
    Eq. (HpermSequence) and Eq. (HadamardElements); returns phases (0 or 1, P = 2)."""
    V = 1
    for L in dims:
        V *= L
    seq = hperm_sequence(V)
    out = np.empty((count, V), dtype=np.int64)
    for t in range(count):
        col = seq[first + t]
        out[t] = [0 if hadamard_element(int(l) + 1, col + 1, V) == 1 else 1 for l in loc]
    return out


# ------------------------------------------------ the comparison sequences of Section 5
def probe_phases_natural(V: int, first: int, count: int, z0_seed: int) -> np.ndarray:
    """Hadamard vectors in natural order (Section 5.2): z_m(i) = H_V(i, m), the Sylvester
    Hadamard matrix with rows (lexicographic sites) and columns both in natural order, bias
    removed by z_0 as for hierarchical probing; V a power of two.  Phases 0/1 of P = 2."""
    if V & (V - 1) or first < 0 or count < 0 or first + count > V:
        raise ValueError("natural-order Hadamard vectors need V a power of two and m < V")
    z0 = z0_signs(z0_seed, V)
    out = np.empty((count, V), dtype=np.int64)
    for t in range(count):
        m = first + t
        col = np.array([0 if hadamard_element(i + 1, m + 1, V) == 1 else 1 for i in range(V)], dtype=np.int64)
        out[t] = (col + (z0 < 0)) % 2
    return out


def probe_phases_z2(V: int, first: int, count: int, seed: int) -> np.ndarray:
    """The Z_2 noise vectors of the standard Monte Carlo estimator (Sections 1.1.2, 5.2): entry i
    of vector m is -1 iff the top bit of SplitMix64 output number m V + i (seeded with ``seed``)
    is set.  Phases 0/1 of P = 2."""
    out = np.empty((count, V), dtype=np.int64)
    for t in range(count):
        m = first + t
        out[t] = [splitmix64_output(seed, m * V + i) >> 63 for i in range(V)]
    return out


# ------------------------------------------------------ correctly rounded values
def _pi_decimal(prec: int) -> Decimal:
    """pi by Machin's formula pi = 16 atan(1/5) - 4 atan(1/239), in Decimal."""
    getcontext().prec = prec + 10

    def atan_inv(n: int) -> Decimal:
        x = Decimal(1) / n
        x2 = x * x
        term, total, k = x, x, 1
        while True:
            term = -term * x2
            k += 2
            t = term / k
            if t == 0 or abs(t) < Decimal(10) ** (-(prec + 5)):
                break
            total += t
        return total

    return 16 * atan_inv(5) - 4 * atan_inv(239)


def _cos_sin_decimal(k: int, P: int, prec: int = 40) -> tuple[Decimal, Decimal]:
    getcontext().prec = prec + 10
    x = 2 * _pi_decimal(prec) * k / P
    c, s = Decimal(0), Decimal(0)
    term = Decimal(1)
    n = 0
    while abs(term) > Decimal(10) ** (-(prec + 5)) or n < 4:
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * x / n
    return c, s


def phase_values(P: int) -> np.ndarray:
    """Correctly rounded FP64 (cos, sin) of 2 pi k / P, k = 0..P-1 (Taylor series in
    40-digit decimal arithmetic, then one rounding to binary64)."""
    out = np.empty((P, 2), dtype=np.float64)
    for k in range(P):
        c, s = _cos_sin_decimal(k, P)
        # a true value of 0 comes out as ~1e-45; every non-zero value has |v| >= sin(2 pi / P)
        out[k, 0] = 0.0 if abs(c) < Decimal("1e-30") else float(c)
        out[k, 1] = 0.0 if abs(s) < Decimal("1e-30") else float(s)
    return out


def probe_values(phases: np.ndarray, P: int) -> np.ndarray:
    """Complex entries exp(2 pi i phase / P) from the correctly rounded table."""
    tab = phase_values(P)
    return tab[phases, 0] + 1j * tab[phases, 1]
