"""Pins of the oracle's estimator: exactness, closed forms, unbiasedness, gradients."""
import itertools

import numpy as np
import pytest

from oracle import estimator as E
from oracle import operators as O
from oracle import permutation as P
from oracle import probing as Pr
from paper_1302_4018_gb300 import synth
from pins import (free_wilson_singular_values, free_wilson_trace_inverse, laplacian_eigenvalues,
                  laplacian_trace_inverse)


def test_prefix_sequential_vs_kahan():
    rng = np.random.default_rng(0)
    q = rng.standard_normal(1000) * 1e3 + 1j * rng.standard_normal(1000)
    a = E.trace_prefix(q)
    b = E.trace_prefix_kahan(q)
    assert np.allclose(a, b, rtol=1e-13)
    assert np.isclose(a[-1], np.mean(q))


@pytest.mark.parametrize("seed", [0, 1])
def test_laplacian_full_sequence_is_exact_4x4x4x4(seed):
    dims = (4, 4, 4, 4)
    q = E.laplacian_quadratures(dims, 0.05, 0, 256, seed, tol=1e-13)
    T = E.trace_prefix(q)
    assert np.isclose(T[-1].real, laplacian_trace_inverse(dims, 0.05), rtol=1e-11)


def test_laplacian_8x8x8x8_dense_full_sequence():
    # the 8^4, m = 0.05 control problem: T_N = Tr(A^-1) = closed form = dense LU
    dims = (8, 8, 8, 8)
    q = E.laplacian_quadratures(dims, 0.05, 0, 4096, 1, method="dense")
    T = E.trace_prefix(q)
    assert np.isclose(T[-1].real, laplacian_trace_inverse(dims, 0.05), rtol=1e-11)
    # first vector without bias removal: h_0 = 1 is the lowest eigenvector: T_1 = V / m
    q0 = E.laplacian_quadratures(dims, 0.05, 0, 2, 0, tol=1e-13)
    assert np.isclose(q0[0].real, 4096 / 0.05, rtol=1e-12)


@pytest.mark.parametrize("dims,seed", [((8, 8, 8, 8), 0), ((4, 8, 4, 8), 3)])
def test_powers_exact_at_completion(dims, seed):
    """Tr(A^k), k <= 2^{m+1} - 1, is exact at the completion point s = 2^{dm+1}
    (same-colour sites are >= 2^{m+1} apart, Section 3.3), matvec only."""
    d = 4
    lam = laplacian_eigenvalues(dims, 0.05)
    for m in (0, 1):
        s = 2 ** (d * m + 1)
        W = E.probe_vectors(dims, 0, s, seed).real
        for k in range(1, 2 ** (m + 1)):
            X = W.T.copy()
            for _ in range(k):
                X = O.laplacian_apply(X, dims, 0.05)
            est = np.sum(W.T * X) / s
            assert np.isclose(est, np.sum(lam ** k), rtol=1e-12)


def test_unbiased_over_all_z0_2x2x2x2():
    """Section 4: with v = z0 (.) z, E_{z0}[T_s] = Tr(A^-1) for every s (all 2^16 z0 on 2^4)."""
    dims = (2, 2, 2, 2)
    V = 16
    Ainv = np.linalg.inv(O.laplacian_dense(dims, 0.05))
    Z = np.where(Pr.LatticeBasis(dims).matrix()[np.array(P.hierarchical_loc(dims))] == 0, 1.0, -1.0)
    signs = np.array(list(itertools.product([1.0, -1.0], repeat=V)))      # all z0
    exact = np.trace(Ainv)
    for s in (1, 2, 3, 5, 16):
        Ts = np.zeros(len(signs))
        for m in range(s):
            Vm = signs * Z[:, m][None, :]
            Ts += np.einsum("ni,ij,nj->n", Vm, Ainv, Vm)
        assert np.isclose(Ts.mean() / s, exact, rtol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (3, 2, 2, 2)])
def test_wilson_full_sequence_equals_dense_trace(dims):
    U = synth.gauge_links(dims, 0.3, 11)
    V = int(np.prod(dims))
    q = E.wilson_quadratures(dims, U, 0.12, 0, V, 5, method="dense")
    T = E.trace_prefix(q)
    D = O.wilson_dense(U, dims, 0.12)
    assert np.isclose(T[-1], np.trace(np.linalg.inv(D)), rtol=1e-11)
    # gamma_5-hermiticity: every q_m (hence every T_s) is real
    assert np.max(np.abs(T.imag)) <= 1e-11 * np.max(np.abs(T.real))
    # BiCGStab oracle agrees with dense on a prefix
    qb = E.wilson_quadratures(dims, U, 0.12, 0, 3, 5, tol=1e-13)
    assert np.allclose(qb, q[:3], rtol=1e-11)


def test_wilson_free_field_full_sequence_4x4x4x4():
    dims = (4, 4, 4, 4)
    V = 256
    U = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    Ug, _ = synth.gauge_transform(U, dims, 5)
    q = E.wilson_quadratures(dims, Ug, 0.115, 0, V, 9, method="dense")
    T = E.trace_prefix(q)
    assert np.isclose(T[-1].real, free_wilson_trace_inverse(dims, 0.115), rtol=1e-10)


def test_laplacian_gradient_closed_form_and_fd():
    dims = (4, 4, 2, 2)
    V = 64
    m = 0.3
    # at s = N: dT/dm = sum_x dT/dmu(x) = -sum_k 1/lambda_k^2
    g = E.laplacian_grad_mass_field(dims, m, V, 2, tol=1e-14)
    lam = laplacian_eigenvalues(dims, m)
    assert np.isclose(np.sum(g).real, -np.sum(1.0 / lam ** 2), rtol=1e-10)
    # central differences of the estimate at s = 5 in a few site directions
    s = 5
    g5 = E.laplacian_grad_mass_field(dims, m, s, 2, method="dense").real
    h = 1e-5
    for site in (0, 7, 33):
        e = np.zeros(V)
        e[site] = h
        tp = E.trace_prefix(E.laplacian_quadratures(dims, m, 0, s, 2, mass_field=e, method="dense"))[-1]
        tm = E.trace_prefix(E.laplacian_quadratures(dims, m, 0, s, 2, mass_field=-e, method="dense"))[-1]
        assert np.isclose((tp - tm).real / (2 * h), g5[site], rtol=1e-6, atol=1e-9)


def test_wilson_gradient_fd():
    dims = (2, 2, 2, 4)
    V = 32
    U = synth.gauge_links(dims, 0.3, 21)
    mf = synth.mass_field(dims, 0.01, 5000)
    s = 3
    g = E.wilson_grad_mass_field(dims, U, 0.12, s, 7, mass_field=mf, method="dense")
    assert np.max(np.abs(g.imag)) < 1e-10 * np.max(np.abs(g.real))
    h = 1e-5
    for site in (0, 13, 31):
        e = mf.copy()
        e[site] += h
        tp = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, s, 7, mass_field=e, method="dense"))[-1]
        e[site] -= 2 * h
        tm = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, s, 7, mass_field=e, method="dense"))[-1]
        assert np.isclose(((tp - tm) / (2 * h)).real, g[site].real, rtol=1e-6, atol=1e-9)
    # uniform direction d/dm = sum_x dT/dmu(x)
    tp = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, s, 7, mass=h, mass_field=mf, method="dense"))[-1]
    tm = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, s, 7, mass=-h, mass_field=mf, method="dense"))[-1]
    assert np.isclose(((tp - tm) / (2 * h)).real, np.sum(g).real, rtol=1e-7)


# ------------------------------------------------------------------ the comparison sequences (NEXT-2)
def test_natural_hadamard_is_sylvester_in_natural_order():
    import scipy.linalg

    from oracle import probing as Pr

    V = 64
    ph = Pr.probe_phases_natural(V, 0, V, 0)
    H = scipy.linalg.hadamard(V)
    assert np.array_equal(1 - 2 * ph, H.T)               # row m of ph is column m of H
    z0 = Pr.z0_signs(99, V)
    assert np.array_equal((1 - 2 * Pr.probe_phases_natural(V, 3, 5, 99)), (H[:, 3:8] * z0[:, None]).T)


def test_z2_noise_is_splitmix64_counter_stream():
    from oracle import probing as Pr

    V = 10
    ph = Pr.probe_phases_z2(V, 2, 3, 1234567)
    for t in range(3):
        for i in range(V):
            assert ph[t, i] == Pr.splitmix64_output(1234567, (2 + t) * V + i) >> 63
    big = Pr.probe_phases_z2(64, 0, 64, 5)
    assert 0.4 < big.mean() < 0.6


@pytest.mark.parametrize("kind", ["hp", "natural"])
def test_z0_variance_formula_matches_enumeration_of_all_z0(kind):
    """Brute force over all 2^16 vectors z_0 on the 2^4 torus: the mean of T_s is Tr A^-1 exactly
    (bias removal, Section 4) and its variance is the closed form of z0_variance."""
    from oracle import probing as Pr

    dims = (2, 2, 2, 2)
    V = 16
    B = np.linalg.inv(O.laplacian_dense(dims, 0.3))
    if kind == "hp":
        ph, _ = Pr.probe_phases(dims, 0, V, 0)
    else:
        ph = Pr.probe_phases_natural(V, 0, V, 0)
    Z = 1 - 2 * ph
    bits = (np.arange(2 ** V)[:, None] >> np.arange(V)[None, :]) & 1
    Z0 = 1 - 2 * bits                                    # all 65536 z_0
    for s in (1, 2, 3, 4, 8, 16):
        C = Z[:s].T @ Z[:s]
        T = np.einsum("ki,ij,kj->k", Z0, B * C, Z0) / s  # T_s for every z_0
        assert abs(T.mean() - np.trace(B)) <= 1e-12 * np.trace(B)
        assert abs(T.var() - E.z0_variance(B, Z, s)) <= 1e-10 * max(T.var(), 1e-30) + 1e-24
    assert E.z0_variance(B, Z, 16) <= 1e-28              # s = N: exact for every z_0


def test_hierarchical_variance_at_completion_is_same_colour_sum():
    """At a completion point s = 2^{k}, sum_m z_m z_m^T = s [same colour] (Proposition of Section 2),
    so the variance reduces to 2 sum over same-colour pairs i != j of (A^-1)_ij^2: the elements the
    colouring could not remove."""
    from oracle import probing as Pr

    dims = (4, 4, 4, 4)
    V = 256
    B = np.linalg.inv(O.laplacian_dense(dims, 0.5))
    ph, _ = Pr.probe_phases(dims, 0, 32, 0)
    Z = 1 - 2 * ph
    for s in (2, 32):
        C = Z[:s].T @ Z[:s]
        same = (C == s)
        assert np.all((C == s) | (C == 0))
        direct = 2 * np.sum(np.where(same & ~np.eye(V, dtype=bool), B ** 2, 0.0))
        assert abs(E.z0_variance(B, Z, s) - direct) <= 1e-12 * direct
    assert E.z0_variance(B, Z, 32) < 0.2 * E.z0_variance(B, Z, 2)


# ------------------------------------------------------------------ deflated probing
def _lowest_eigvecs(dims, mass, k):
    A = O.laplacian_dense(dims, mass)
    lam, V = np.linalg.eigh(A)
    return lam[:k], V[:, :k]


@pytest.mark.parametrize("k", [1, 5, 17])
def test_deflated_full_sequence_is_exact(k):
    """At s = N the nested vectors form an orthogonal basis (W^H W = N I), so the probed part is
    Tr(P A^-1 P) = Tr(A^-1 P) and T_N = sum 1/lambda_j + Tr(A^-1 P) = Tr A^-1, the Fourier closed
    form of the periodic Laplacian, for any number k of deflated eigenvectors."""
    dims, mass = (4, 4, 2, 2), 0.3
    N = 64
    lam, V = _lowest_eigvecs(dims, mass, k)
    q = E.laplacian_deflated_quadratures(dims, mass, V, 0, N, z0_seed=5)
    T = E.deflated_trace_prefix(lam, q)
    exact = laplacian_trace_inverse(dims, mass)
    assert abs(T[-1] - exact) <= 1e-12 * exact
    assert abs(T[-1].imag) <= 1e-12 * exact


def test_deflating_every_eigenvector_leaves_nothing_to_probe():
    """k = N: P = 0, every quadrature vanishes and T_s = Tr A^-1 for every s."""
    dims, mass = (2, 2, 2, 4), 0.7
    lam, V = _lowest_eigvecs(dims, mass, 32)
    q = E.laplacian_deflated_quadratures(dims, mass, V, 0, 8, z0_seed=3)
    assert np.abs(q).max() <= 1e-12
    T = E.deflated_trace_prefix(lam, q)
    assert np.allclose(T, laplacian_trace_inverse(dims, mass), rtol=1e-12, atol=0)


def test_deflation_with_no_vectors_is_plain_probing():
    dims, mass = (4, 4, 4, 2), 0.2
    q0 = E.laplacian_quadratures(dims, mass, 0, 12, 9, method="dense")
    q = E.laplacian_deflated_quadratures(dims, mass, np.zeros((128, 0)), 0, 12, z0_seed=9)
    assert np.allclose(q, q0, rtol=1e-12, atol=0)


def test_deflating_the_lowest_modes_reduces_the_z0_variance():
    """The exact z_0-variance (1/s^2) sum_{i<j} |B_ij + B_ji|^2 C_ij^2 of the probed part falls
    when B = A^-1 is replaced by A^-1 P with the 7 lowest modes removed (cond ~ 100 Laplacian)."""
    from oracle import probing as Pr

    dims, mass = (8, 8, 8), 12.0 / 99.0
    A = O.laplacian_dense(dims, mass)
    lam, V = np.linalg.eigh(A)
    B = np.linalg.inv(A)
    Bd = B - (V[:, :7] / lam[:7]) @ V[:, :7].T
    ph, _ = Pr.probe_phases(dims, 0, 64, 0)
    Z = 1 - 2 * ph
    for s in (8, 16, 64):
        assert E.z0_variance(Bd, Z, s) < 0.5 * E.z0_variance(B, Z, s)


def test_speedup_ratio_of_all_z0_is_the_closed_form_ratio():
    """R_s over every one of the 2^16 vectors z_0 of the 2^4 torus (population variances) equals
    z0_variance(1) / (z0_variance(s) s) from the closed form; R_1 = 1; at s = N the estimate is
    exact for every z_0 (infinite ratio)."""
    from oracle import probing as Pr

    dims = (2, 2, 2, 2)
    V = 16
    B = np.linalg.inv(O.laplacian_dense(dims, 0.3))
    ph, _ = Pr.probe_phases(dims, 0, V, 0)
    Z = 1 - 2 * ph
    bits = (np.arange(2 ** V)[:, None] >> np.arange(V)[None, :]) & 1
    Z0 = 1 - 2 * bits
    svals = (1, 2, 3, 4, 8)
    T = np.stack([np.einsum("ki,ij,kj->k", Z0, B * (Z[:s].T @ Z[:s]), Z0) / s for s in svals], 1)
    # columns are s = 1, 2, 3, 4, 8: rescale the generic definition by the actual s
    v = [E.sample_variance(T[:, j], ddof=0) for j in range(len(svals))]
    for j, s in enumerate(svals):
        closed = E.z0_variance(B, Z, 1) / (E.z0_variance(B, Z, s) * s)
        assert abs(v[0] / (v[j] * s) - closed) <= 1e-9 * closed
    R = E.speedup_ratio(T[:, :2], ddof=0)
    assert R[0] == 1.0
    assert abs(R[1] - E.z0_variance(B, Z, 1) / (E.z0_variance(B, Z, 2) * 2)) <= 1e-9 * R[1]


def test_jackknife_of_the_mean_is_the_standard_error():
    """For the mean, the delete-one jackknife error equals the textbook standard error
    std(ddof = 1) / sqrt(n) exactly; for a constant statistic it is zero."""
    x = np.random.default_rng(3).normal(2.0, 0.7, 41)
    m, err = E.jackknife(x, lambda a: a.mean())
    assert abs(m - x.mean()) <= 1e-15 * abs(m)
    assert abs(err - x.std(ddof=1) / np.sqrt(41)) <= 1e-12 * err
    assert E.jackknife(x, lambda a: 5.0)[1] == 0.0
    # the variance statistic: its jackknife error shrinks like 1 / sqrt(n)
    y = np.random.default_rng(4).normal(0, 1, 4000)
    _, e_small = E.jackknife(y[:400], lambda a: a.var(ddof=1))
    _, e_big = E.jackknife(y, lambda a: a.var(ddof=1))
    assert 2.0 < e_small / e_big < 5.0


def test_lowest_eigenpairs_match_the_fourier_spectrum():
    """Without a mass field the Laplacian's spectrum is m + sum_j 4 sin^2(pi k_j / L_j) over all
    wave vectors; the oracle's k lowest pairs carry exactly those values, are orthonormal and
    satisfy A v = lambda v."""
    dims, mass = (6, 4, 4), 0.2
    lam, V = E.laplacian_lowest_eigenpairs(dims, mass, 9)
    k = [np.arange(L) for L in dims]
    spec = np.sort((mass + sum(4 * np.sin(np.pi * kk / L) ** 2
                               for kk, L in zip(np.meshgrid(*k, indexing="ij"), dims))).ravel())
    assert np.allclose(lam, spec[:9], rtol=0, atol=1e-12)
    assert np.allclose(V @ V.T, np.eye(9), atol=1e-12)
    A = O.laplacian_dense(dims, mass)
    assert np.abs(A @ V.T - V.T * lam[None, :]).max() <= 1e-12


# ------------------------------------------------------------------ Wilson deflation (gamma_5 D)
def test_gamma5_wilson_spectrum_is_the_free_field_closed_form():
    """U = 1: |lambda(gamma_5 D)| are the singular values sqrt(a^2 + b^2) of the plane waves."""
    dims, kappa, mass = (4, 2, 2, 4), 0.11, 0.05
    U = synth.gauge_links(dims, 0.0, 1)
    assert np.allclose(U, np.broadcast_to(np.eye(3), U.shape))
    Q = E.gamma5_hermitian_dense(dims, U, kappa, mass)
    assert np.abs(Q - np.conj(Q).T).max() <= 1e-14
    lam = np.linalg.eigvalsh(Q)
    assert np.allclose(np.sort(np.abs(lam)), np.sort(free_wilson_singular_values(dims, kappa, mass)), rtol=1e-12,
                       atol=0)


def test_wilson_eigenpairs_are_gamma5_eigenpairs():
    """Q w = lambda w with Q = gamma_5 D applied by the stencil (not the dense matrix), and the
    pairs come in increasing |lambda|."""
    dims, kappa = (2, 4, 2, 2), 0.12
    U = synth.gauge_links(dims, 0.4, 3)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, kappa, 10, mass=0.02)
    assert np.all(np.diff(np.abs(lam)) >= 0)
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None]
    for j in range(10):
        r = g5 * O.wilson_apply(W[j], U, dims, kappa, 0.02) - lam[j] * W[j]
        assert np.linalg.norm(r) <= 1e-12
        assert abs(np.vdot(W[j], W[j]) - 1) <= 1e-12


@pytest.mark.parametrize("k", [1, 7, 30])
def test_wilson_deflated_full_sequence_is_exact(k):
    """At s = N the diluted probe vectors span everything, so the probed part is
    Tr(D^-1 (I - U U^H)) and T_N = sum_j w_j^H g5 w_j / lambda_j + Tr(D^-1 (I - U U^H)) = Tr D^-1
    (dense inverse), for any k."""
    dims, kappa = (2, 2, 2, 4), 0.12
    U = synth.gauge_links(dims, 0.4, 5)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, kappa, k)
    q, exact = E.wilson_deflated_quadratures(dims, U, kappa, lam, W, 0, 32, z0_seed=4)
    T = exact + E.trace_prefix(q)
    ref = np.trace(np.linalg.inv(O.wilson_dense(U, dims, kappa)))
    assert abs(T[-1] - ref) <= 1e-11 * abs(ref)


def test_wilson_deflating_every_eigenvector_leaves_nothing_to_probe():
    """k = 12 V: U U^H = I, every quadrature vanishes and T_s = Tr D^-1 for every s; the trace is
    real (gamma_5-hermiticity)."""
    dims, kappa = (2, 2, 2, 2), 0.12
    U = synth.gauge_links(dims, 0.4, 6)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, kappa, 192)
    q, exact = E.wilson_deflated_quadratures(dims, U, kappa, lam, W, 0, 6, z0_seed=2)
    assert np.abs(q).max() <= 1e-11
    ref = np.trace(np.linalg.inv(O.wilson_dense(U, dims, kappa)))
    assert abs(exact - ref) <= 1e-11 * abs(ref) and abs(ref.imag) <= 1e-11 * abs(ref)


def test_wilson_deflated_quadrature_is_the_plain_one_minus_a_projection_sum():
    """q'_m = q_m - sum_a g5_a sum_j |v_{m,a}^H w_j|^2 / lambda_j: the correction that turns plain
    quadratures into deflated ones without changing the solves (D^-1 u_j = w_j / lambda_j and
    u_j^H v = g5_a conj(v^H w_j) for a vector supported on component a)."""
    dims, kappa = (2, 2, 4, 2), 0.115
    U = synth.gauge_links(dims, 0.3, 7)
    mf = synth.mass_field(dims, 0.01, 8)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, kappa, 9, mass_field=mf)
    qd, _ = E.wilson_deflated_quadratures(dims, U, kappa, lam, W, 0, 8, z0_seed=3, mass_field=mf)
    q0 = E.wilson_quadratures(dims, U, kappa, 0, 8, 3, mass_field=mf, method="dense")
    P = E.probe_vectors(dims, 0, 8, 3)
    g5 = np.repeat([1.0, 1.0, -1.0, -1.0], 3)
    Wf = W.reshape(9, -1, 12)
    corr = np.array([sum(g5[a] * np.abs(np.vdot(P[m], Wf[j, :, a])) ** 2 / lam[j] for a in range(12) for j in range(9))
                     for m in range(8)])
    assert np.allclose(qd, q0 - corr, rtol=0, atol=1e-11 * np.abs(q0).max())


def test_wilson_deflation_reduces_the_z0_variance():
    """The exact z_0-variance of T_s falls when D^-1 is replaced by D^-1 (I - U U^H) with the 24
    smallest |lambda(gamma_5 D)| removed (rough links near the critical kappa).  With full
    dilution sum_a (z (x) e_a)^H B (z (x) e_a) = z^T Bt z, Bt[x, y] the trace of the 12 x 12 block
    B[x, y], so the variance is z0_variance of the block traces."""
    from oracle import probing as Pr

    dims, kappa = (4, 4, 2, 2), 0.124
    U = synth.gauge_links(dims, 0.5, 9)
    D = O.wilson_dense(U, dims, kappa)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, kappa, 24)
    V = int(np.prod(dims))
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    Uv = g5[:, None] * W.reshape(24, -1).T
    B = np.linalg.inv(D)
    Bd = B @ (np.eye(12 * V) - Uv @ np.conj(Uv).T)
    def block_traces(M):
        return np.einsum("xaya->xy", M.reshape(V, 12, V, 12))

    ph, _ = Pr.probe_phases(dims, 0, 32, 0)
    Z = 1 - 2 * ph
    for s in (4, 8, 16):
        assert E.z0_variance(block_traces(Bd), Z, s) < 0.7 * E.z0_variance(block_traces(B), Z, s)


# ------------------------------------------------------------------ Wilson deflation with singular triplets
def test_wilson_singular_triplets_are_the_gamma5_eigenpairs():
    """D v = sigma u with v = w_j, u = sign(lambda_j) gamma_5 w_j, sigma = |lambda_j| for the
    eigenpairs of gamma_5 D: the same smallest singular values, and D v_j = sigma_j u_j."""
    dims, kappa = (2, 4, 2, 2), 0.12
    U = synth.gauge_links(dims, 0.4, 11)
    sig, R, L = E.wilson_smallest_singular_triplets(dims, U, kappa, 8, mass=0.02)
    lam, _ = E.wilson_lowest_eigenpairs(dims, U, kappa, 8, mass=0.02)
    assert np.allclose(sig, np.abs(lam), rtol=1e-12, atol=0)
    for j in range(8):
        assert np.linalg.norm(O.wilson_apply(R[j], U, dims, kappa, 0.02) - sig[j] * L[j]) <= 1e-12
        assert abs(np.vdot(R[j], R[j]) - 1) <= 1e-12 and abs(np.vdot(L[j], L[j]) - 1) <= 1e-12


@pytest.mark.parametrize("k", [1, 6, 25])
def test_wilson_svd_deflated_full_sequence_is_exact(k):
    """T_N = sum_j u_j^H v_j / sigma_j + Tr(D^-1 (I - U U^H)) = Tr D^-1 (dense inverse) for any k."""
    dims, kappa = (2, 2, 4, 2), 0.12
    U = synth.gauge_links(dims, 0.4, 12)
    sig, R, L = E.wilson_smallest_singular_triplets(dims, U, kappa, k)
    q, exact = E.wilson_deflated_quadratures_svd(dims, U, kappa, sig, R, L, 0, 32, z0_seed=6)
    T = exact + E.trace_prefix(q)
    ref = np.trace(np.linalg.inv(O.wilson_dense(U, dims, kappa)))
    assert abs(T[-1] - ref) <= 1e-11 * abs(ref)


def test_wilson_svd_deflated_quadrature_is_the_plain_one_minus_a_projection_sum():
    """q'_m = q_m - sum_{a,j} (v_{m,a}^H v_j)(u_j^H v_{m,a}) / sigma_j, and the gamma_5 eigenpair form
    gives the same deflated quadratures (its triplets are the same modes)."""
    dims, kappa = (2, 2, 2, 4), 0.115
    U = synth.gauge_links(dims, 0.3, 13)
    sig, R, L = E.wilson_smallest_singular_triplets(dims, U, kappa, 7)
    qd, ex = E.wilson_deflated_quadratures_svd(dims, U, kappa, sig, R, L, 0, 8, z0_seed=3)
    q0 = E.wilson_quadratures(dims, U, kappa, 0, 8, 3, method="dense")
    P = E.probe_vectors(dims, 0, 8, 3)
    Rf, Lf = R.reshape(7, -1, 12), L.reshape(7, -1, 12)
    corr = np.array([sum(np.vdot(P[m], Rf[j, :, a]) * np.vdot(Lf[j, :, a], P[m]) / sig[j]
                         for a in range(12) for j in range(7)) for m in range(8)])
    assert np.allclose(qd, q0 - corr, rtol=0, atol=1e-11 * np.abs(q0).max())
    lam, Wq = E.wilson_lowest_eigenpairs(dims, U, kappa, 7)
    qg, exg = E.wilson_deflated_quadratures(dims, U, kappa, lam, Wq, 0, 8, z0_seed=3)
    assert np.allclose(qd, qg, rtol=0, atol=1e-11 * np.abs(q0).max()) and abs(ex - exg) <= 1e-11 * abs(exg)


def test_wilson_deflation_with_unconverged_ritz_triplets_is_exact():
    """Rayleigh-Ritz triplets of Q^2 = D^H D on an arbitrary orthonormal block (v_j the Ritz vectors,
    sigma_j^2 the Ritz values, u_j = D v_j / sigma_j) are not singular triplets (D^H u_j differs from
    sigma_j v_j), but U is orthonormal and D^-1 u_j = v_j / sigma_j holds exactly, so the deflated
    sequence still reaches Tr D^-1 at s = N: an unconverged eigensolver leaves the estimate exact."""
    dims, kappa = (2, 2, 4, 2), 0.12
    U = synth.gauge_links(dims, 0.4, 14)
    D = O.wilson_dense(U, dims, kappa)
    n, b, k = D.shape[0], 12, 6
    rng = np.random.default_rng(5)
    X, _ = np.linalg.qr(rng.standard_normal((n, b)) + 1j * rng.standard_normal((n, b)))
    DX = D @ X
    th2, W = np.linalg.eigh(DX.conj().T @ DX)
    Vr = (X @ W)[:, :k]
    sig = np.sqrt(th2[:k])
    Ul = (DX @ W)[:, :k] / sig
    assert np.allclose(Ul.conj().T @ Ul, np.eye(k), rtol=0, atol=1e-12)
    assert np.linalg.norm(D.conj().T @ Ul - Vr * sig) > 1e-2
    V = int(np.prod(dims))
    R, L = Vr.T.reshape(k, V, 4, 3), Ul.T.reshape(k, V, 4, 3)
    q, exact = E.wilson_deflated_quadratures_svd(dims, U, kappa, sig, R, L, 0, 32, z0_seed=6)
    T = exact + E.trace_prefix(q)
    ref = np.trace(np.linalg.inv(D))
    assert abs(T[-1] - ref) <= 1e-11 * abs(ref)
