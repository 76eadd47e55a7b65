"""Pins of the oracle's probing vectors (Sections 2.2 and 4)."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import permutation as P
from oracle import probing as Pr


@pytest.mark.parametrize("n", [2, 4, 8, 16, 64, 256])
def test_hadamard_orthogonal_and_element_formula(n):
    H = Pr.hadamard(n)
    assert np.array_equal(H @ H.T, n * np.eye(n, dtype=np.int64))
    for i in range(1, n + 1, max(1, n // 16)):
        for j in range(1, n + 1):
            assert Pr.hadamard_element(i, j, n) == H[i - 1, j - 1]


def test_hperm_sequence_golden():
    for row in read_golden("hperm_sequence.txt"):
        N = int(row[0])
        listed = [int(v) for v in row[1:]]
        assert Pr.hperm_sequence(N)[:len(listed)] == listed


@pytest.mark.parametrize("K", range(1, 17))
def test_hperm_is_bit_reversal(K):
    seq = Pr.hperm_sequence(1 << K)
    for m in range(0, 1 << K, max(1, (1 << K) // 512)):
        assert seq[m] == int(format(m, "0%db" % K)[::-1], 2)


@pytest.mark.parametrize("K", range(1, 11))
def test_kronecker_recursion_permutes_hadamard_columns(K):
    # Eq. (Hperm-recursive) produces H_N(:, Hperm) (Eqs. HpermSequence, row-col-permutation)
    N = 1 << K
    Z = Pr.basis_kron([2] * K, 2)
    H = Pr.hadamard(N)
    seq = Pr.hperm_sequence(N)
    assert np.array_equal(np.where(Z == 0, 1, -1), H[:, seq])
    for m in range(0, N, max(1, N // 64)):
        assert np.array_equal(Pr.basis_column([2] * K, 2, m), Z[:, m])


@pytest.mark.parametrize("K", range(1, 10))
def test_nesting(K):
    # Z^(k-1) = Z^(k)(:, 1:2^{k-1}) with Z^(k) = Z~^(k) (x) 1_{N/2^k}  (Section 2.2)
    N = 1 << K
    prev = None
    for k in range(1, K + 1):
        Zk = np.repeat(Pr.basis_kron([2] * k, 2), N >> k, axis=0)
        if prev is not None:
            assert np.array_equal(Zk[:, :prev.shape[1]], prev)
        prev = Zk


def test_n8_worked_example():
    rows = read_golden("n8_example.txt")
    i1 = rows.index(["Z1"])
    i2 = rows.index(["Z2"])
    Z1 = np.array([[int(v) for v in r] for r in rows[i1 + 1:i2]])
    Z2 = np.array([[int(v) for v in r] for r in rows[i2 + 1:i2 + 9]])
    span1 = [int(v) for v in rows[i2 + 9][1:]]
    span2 = [int(v) for v in rows[i2 + 10][1:]]
    H8 = Pr.hadamard(8)
    h = [H8[:, j] for j in range(8)]
    # the first vectors of the hierarchical sequence are h0, h4 then h0, h4, h2, h6
    assert Pr.hperm_sequence(8)[:2] == span1 and Pr.hperm_sequence(8)[:4] == span2
    # Z1 = 1/2 [h0, h4] H_2.  The printed Z2 = 1/2 [h0, h2, h4, h6] H_4 holds with 1/4
    # (each column of H_4 sums four +-1 columns of H_8); read as 1/4.
    assert np.array_equal(2 * Z1, np.stack([h[0], h[4]], 1) @ Pr.hadamard(2))
    assert np.array_equal(4 * Z2, np.stack([h[0], h[2], h[4], h[6]], 1) @ Pr.hadamard(4))
    # [h0, h4] = H_2 (x) 1_4 ; [h0, h4, h2, h6] = [H_2 (x) H_2(:,1), H_2 (x) H_2(:,2)] (x) 1_2
    H2 = Pr.hadamard(2)
    assert np.array_equal(np.stack([h[0], h[4]], 1), np.kron(H2, np.ones((4, 1), dtype=int)))
    inner = np.concatenate([np.kron(H2, H2[:, :1]), np.kron(H2, H2[:, 1:])], axis=1)
    assert np.array_equal(np.stack([h[0], h[4], h[2], h[6]], 1), np.kron(inner, np.ones((2, 1), dtype=int)))


def test_fig2_red_black():
    rows = {r[0]: r[1:] for r in read_golden("fig2_red_black.txt")}
    dims = [int(v) for v in rows["dims"]]
    h8 = [int(v) for v in rows["h8_permuted"]]
    assert np.array_equal(np.where(Pr.basis_kron([2] * 4, 2)[:, 1] == 0, 1, -1), h8)
    ph, Pp = Pr.probe_phases(dims, 1, 1, 0)
    vals = np.where(ph[0] == 0, 1, -1)
    for site in range(16):
        x = P.coords_of(site, dims)
        assert vals[site] == (1 if sum(x) % 2 == 0 else -1)


@pytest.mark.parametrize("dims", [(4, 4), (2, 4, 8), (4, 4, 4, 4), (8, 2, 2, 4)])
def test_element_formula_matches_kronecker(dims):
    loc = P.hierarchical_loc(dims)
    V = len(loc)
    ph, Pp = Pr.probe_phases(dims, 0, V, 0, loc=loc)
    assert Pp == 2
    assert np.array_equal(ph, Pr.probe_phases_hadamard(dims, 0, V, loc))


def _values(ph, P):
    return Pr.probe_values(ph, P)


@pytest.mark.parametrize("dims,seed", [((4, 4, 4), 0), ((6, 6), 7), ((3, 3, 3, 3), 11), ((6, 2, 6, 2), 3),
                                       ((12, 6), 0), ((2, 2, 2, 4), 5)])
def test_orthogonality_full_basis(dims, seed):
    # Z^H Z = N I for the full nested basis (Hadamard and Fourier levels), with and without z_0
    basis = Pr.LatticeBasis(dims)
    assert basis.n_vectors == basis.V
    ph, Pp = Pr.probe_phases(dims, 0, basis.V, seed)
    Z = _values(ph, Pp)
    G = Z.conj() @ Z.T
    assert np.allclose(G, basis.V * np.eye(basis.V), atol=1e-9 * basis.V)


@pytest.mark.parametrize("dims", [(8, 8), (4, 4, 4, 4), (4, 8, 4), (2, 4, 2, 8)])
def test_probing_property_at_completion(dims):
    """Proposition 1 / Section 2.2: at a completion point s = 2^{dm+1} the
    average (1/s) sum z_m z_m^H is exactly the same-colour indicator matrix."""
    d = len(dims)
    order = P.LatticeOrder(dims)
    loc = np.array(order.all_loc())
    V = order.V
    for m in range(0, min(order.ks)):
        s = 2 ** (d * m + 1)
        ph, Pp = Pr.probe_phases(dims, 0, s, 0, loc=loc)
        Z = _values(ph, Pp)
        M = (Z.T @ Z.conj()) / s
        color = loc >> (order.K - (d * m + 1))
        ind = (color[:, None] == color[None, :]).astype(float)
        assert np.allclose(M, ind, atol=1e-12)


def test_bias_removal_identities():
    # Section 4: V^T V = Z^T Z and V V^T = (z0 z0^T) (.) Z Z^T
    dims = (4, 4, 2)
    s = 12
    ph, Pp = Pr.probe_phases(dims, 0, s, 0)
    phb, _ = Pr.probe_phases(dims, 0, s, 12345)
    Z = _values(ph, Pp).T
    Vv = _values(phb, Pp).T
    z0 = Pr.z0_signs(12345, Z.shape[0])
    assert set(z0.tolist()) == {-1, 1}
    assert np.allclose(Vv, z0[:, None] * Z)
    assert np.allclose(Vv.conj().T @ Vv, Z.conj().T @ Z)
    assert np.allclose(Vv @ Vv.conj().T, np.outer(z0, z0) * (Z @ Z.conj().T))


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 1234567: published first outputs of Vigna's generator
    outs = [Pr.splitmix64_output(1234567, i) for i in range(5)]
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]


@pytest.mark.parametrize("Pp", [2, 6, 54, 162, 4374])
def test_phase_values_correctly_rounded(Pp):
    tab = Pr.phase_values(Pp)
    k = np.arange(Pp)
    ref = np.stack([np.cos(2 * np.pi * k / Pp), np.sin(2 * np.pi * k / Pp)], 1)
    assert np.all(np.abs(tab - ref) <= 4e-16 * (1 + np.abs(ref)) + 1e-15)
    # exact special values
    for kk in range(Pp):
        if (4 * kk) % Pp == 0:
            c = [1.0, 0.0, -1.0, 0.0][(4 * kk) // Pp]
            s = [0.0, 1.0, 0.0, -1.0][(4 * kk) // Pp]
            assert tab[kk, 0] == c and tab[kk, 1] == s
        if (12 * kk) % Pp == 0 and (12 * kk // Pp) % 3 != 0:
            assert abs(tab[kk, 0]) == 0.5 or abs(tab[kk, 1]) == 0.5


@pytest.mark.parametrize("Pp", [2, 6, 54, 162, 1458, 4374, 65534])
def test_phase_values_are_the_nearest_binary64(Pp):
    """Every entry of the oracle's table is the binary64 number nearest to cos / sin(2 pi k / P):
    an independent 60-digit evaluation (mpmath) must be closer to it than to either neighbour
    (a 1-ulp error anywhere in the decimal series fails this)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    tab = Pr.phase_values(Pp)
    ks = range(Pp) if Pp <= 4374 else list(range(0, Pp, 97)) + [1, 2, Pp // 4 - 1, Pp // 2 + 1, Pp - 1]
    for k in ks:
        x = 2 * mp.pi * k / Pp
        for j, true in enumerate((mp.cos(x), mp.sin(x))):
            v = float(tab[k, j])
            if abs(true) < mp.mpf(10) ** -50:       # an exact zero
                assert v == 0.0, (k, j, v)
                continue
            err = abs(mp.mpf(v) - true)
            for nb in (np.nextafter(v, np.inf), np.nextafter(v, -np.inf)):
                assert err < abs(mp.mpf(float(nb)) - true), (Pp, k, j, v)


def test_basis_sizes_for_lattices():
    b = Pr.LatticeBasis((12, 12, 12, 12))
    assert b.radices == [2] * 8 + [3, 27] and b.P == 54 and b.n_vectors == 20736
    b = Pr.LatticeBasis((24, 24, 24, 48))
    assert b.K == 13 and b.radices[-2:] == [3, 27] and b.n_vectors == 663552
    b = Pr.LatticeBasis((5, 4))
    assert b.n_vectors == 4 and b.tail == 5          # unequal colour classes: binary part only
