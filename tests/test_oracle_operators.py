"""Pins of the oracle's operators and solvers against closed forms and library routines."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import operators as O
from oracle import solvers as S
from paper_1302_4018_gb300 import synth
from pins import free_wilson_trace_inverse, laplacian_eigenvalues, laplacian_trace_inverse


def test_gamma_clifford_and_hermitian():
    g = O.gamma_matrices()
    for m in range(4):
        assert np.allclose(g[m].conj().T, g[m])
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))


def test_links_are_special_unitary():
    U = synth.gauge_links((4, 4, 2, 2), 0.4, 17).reshape(-1, 3, 3)
    assert np.allclose(U @ np.conj(np.swapaxes(U, -1, -2)), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
    # eps -> 0: links approach the identity like 1 + i eps H
    U0 = synth.gauge_links((2, 2, 2, 2), 1e-8, 3).reshape(-1, 3, 3)
    assert np.allclose(U0, np.eye(3), atol=1e-6)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 5), (8, 1, 2, 4)])
def test_laplacian_apply_equals_dense(dims):
    A = O.laplacian_dense(dims, 0.05)
    x = synth.random_real_fields(dims, 1, 3)[0]
    assert np.allclose(A @ x, O.laplacian_apply(x, dims, 0.05), atol=1e-12)
    assert np.allclose(A, A.T)
    # the constant vector (h_0) is the lowest eigenvector with eigenvalue m (Section 5.1 remark)
    assert np.allclose(O.laplacian_apply(np.ones(A.shape[0]), dims, 0.05), 0.05)


@pytest.mark.parametrize("dims,m", [((4, 4, 4, 4), 0.05), ((8, 8, 8, 8), 0.05), ((6, 4, 3, 2), 0.3)])
def test_laplacian_trace_closed_form(dims, m):
    A = O.laplacian_dense(dims, m)
    assert np.isclose(np.trace(np.linalg.inv(A)), laplacian_trace_inverse(dims, m), rtol=1e-11)
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(laplacian_eigenvalues(dims, m)), atol=1e-10)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 2, 2), (3, 2, 2, 2)])
def test_wilson_apply_equals_dense_and_adjoint(dims):
    U = synth.gauge_links(dims, 0.3, 5)
    mf = synth.mass_field(dims, 0.01, 9)
    D = O.wilson_dense(U, dims, 0.12, 0.02, mf)
    psi = synth.random_spinors(dims, 1, 3)[0]
    assert np.allclose(D @ psi.reshape(-1), O.wilson_apply(psi, U, dims, 0.12, 0.02, mf).reshape(-1))
    assert np.allclose(D.conj().T @ psi.reshape(-1),
                       O.wilson_apply(psi, U, dims, 0.12, 0.02, mf, dagger=True).reshape(-1))
    # gamma_5-hermiticity D^H = g5 D g5
    g5 = np.kron(np.eye(int(np.prod(dims))), np.kron(O.gamma_matrices()[4], np.eye(3)))
    assert np.allclose(D.conj().T, g5 @ D @ g5)


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.115), ((2, 4, 2, 4), 0.12), ((3, 3, 2, 4), 0.1)])
def test_free_wilson_trace_closed_form(dims, kappa):
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    D = O.wilson_dense(U, dims, kappa)
    assert np.isclose(np.trace(np.linalg.inv(D)), free_wilson_trace_inverse(dims, kappa), rtol=1e-11)
    # a random gauge transformation of the free field leaves the trace unchanged
    Ug, _ = synth.gauge_transform(U, dims, 77)
    Dg = O.wilson_dense(Ug, dims, kappa)
    assert np.isclose(np.trace(np.linalg.inv(Dg)), free_wilson_trace_inverse(dims, kappa), rtol=1e-11)


def test_solvers_match_dense():
    dims = (4, 4, 2, 2)
    b = synth.random_real_fields(dims, 1, 1)[0]
    x, _ = S.cg(lambda v: O.laplacian_apply(v, dims, 0.05), b, tol=1e-13)
    A = O.laplacian_dense(dims, 0.05)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)
    dims = (2, 2, 2, 4)
    U = synth.gauge_links(dims, 0.3, 2)
    psi = synth.random_spinors(dims, 1, 4)[0]
    y, _ = S.bicgstab(lambda v: O.wilson_apply(v, U, dims, 0.12), psi, tol=1e-13)
    D = O.wilson_dense(U, dims, 0.12)
    ref = np.linalg.solve(D, psi.reshape(-1))
    assert np.linalg.norm(y.reshape(-1) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_problem_size_golden():
    rows = {r[0]: int(r[1]) for r in read_golden("problem_size.txt")}
    n = 3 * 4 * rows["Ls"] ** 3 * rows["Lt"]
    assert n == 25165824 and round(n / 2 ** 20) == rows["approx_millions"]


# ------------------------------------------------------------------ clover term
def test_sigma_munu_closed_forms():
    """sigma_{mu nu} = (i/2)[g_mu, g_nu] in the chiral basis, worked out by hand from the gammas:
    sigma_jk = -eps_jkl diag(s_l, s_l) and sigma_k4 = diag(s_k, -s_k) (k, j, l spatial)."""
    s = O.pauli()
    Z = np.zeros((2, 2), dtype=complex)
    blk = lambda a, b: np.block([[a, Z], [Z, b]])
    eps = {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (1, 0, 2): -1, (2, 1, 0): -1, (0, 2, 1): -1}
    for (j, k, l), e in eps.items():
        assert np.allclose(O.sigma_munu(j, k), -e * blk(s[l], s[l]), atol=1e-15)
    for k in range(3):
        assert np.allclose(O.sigma_munu(k, 3), blk(s[k], -s[k]), atol=1e-15)
        assert np.allclose(O.sigma_munu(3, k), -blk(s[k], -s[k]), atol=1e-15)
    g5 = O.gamma_matrices()[4]
    for mu in range(4):
        for nu in range(4):
            sm = O.sigma_munu(mu, nu)
            assert np.allclose(sm, np.conj(sm).T) and np.allclose(sm @ g5, g5 @ sm)


def test_clover_field_of_constant_abelian_field():
    """U_1(x) = exp(i b x_2 lam), lam = diag(1, -1, 0), b = 2 pi / L_2, all other links 1: every
    plaquette of the 1-2 plane is exp(-i b lam), so F_12 = -sin(b lam) everywhere, F_21 = -F_12,
    and the other planes carry no field."""
    dims = (3, 6, 2, 2)
    V = int(np.prod(dims))
    b = 2 * np.pi / dims[1]
    lam = np.array([1.0, -1.0, 0.0])
    U = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    for i in range(V):
        x2 = (i // dims[0]) % dims[1]
        U[i, 0] = np.diag(np.exp(1j * b * x2 * lam))
    F = O.clover_field(U, dims, 0, 1)
    assert np.allclose(F, np.diag(-np.sin(b * lam))[None], atol=1e-14)
    assert np.allclose(O.clover_field(U, dims, 1, 0), -F, atol=1e-14)
    for mu, nu in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        assert np.allclose(O.clover_field(U, dims, mu, nu), 0, atol=1e-14)
    C = O.clover_term(U, dims, 0.12, 1.5)
    assert np.allclose(C, -1.5 * 0.12 * np.kron(O.sigma_munu(0, 1), np.diag(-np.sin(b * lam)))[None], atol=1e-14)


def test_clover_field_is_gauge_covariant_and_hermitian():
    """Under U'_mu(x) = g(x) U_mu(x) g(x+mu)^H every closed leaf turns into g(x) Q g(x)^H: a leaf
    that is not a closed path through x breaks this."""
    dims = (2, 4, 3, 2)
    U = synth.gauge_links(dims, 0.5, 61)
    Ug, g = synth.gauge_transform(U, dims, 62)
    for mu, nu in [(0, 1), (0, 3), (1, 2), (2, 3)]:
        F = O.clover_field(U, dims, mu, nu)
        Fg = O.clover_field(Ug, dims, mu, nu)
        assert np.allclose(Fg, g @ F @ np.conj(np.swapaxes(g, -1, -2)), atol=1e-13)
        assert np.allclose(F, np.conj(np.swapaxes(F, -1, -2)), atol=1e-14)
        assert np.allclose(np.trace(F, axis1=1, axis2=2), 0, atol=1e-14)
        assert np.max(np.abs(F)) > 1e-3


def test_clover_wilson_dense_apply_adjoint_and_gauge_invariant_trace():
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    U = synth.gauge_links(dims, 0.6, 63)
    C = O.clover_term(U, dims, 0.12, 1.3)
    D = O.wilson_dense(U, dims, 0.12, 0.02, clover=C)
    psi = synth.random_spinors(dims, 1, 64)[0]
    assert np.allclose(D @ psi.reshape(-1), O.wilson_apply(psi, U, dims, 0.12, 0.02, clover=C).reshape(-1),
                       atol=1e-13)
    assert np.allclose(np.conj(D).T @ psi.reshape(-1),
                       O.wilson_apply(psi, U, dims, 0.12, 0.02, dagger=True, clover=C).reshape(-1), atol=1e-13)
    G5 = np.kron(np.eye(V), np.kron(O.gamma_matrices()[4], np.eye(3)))
    assert np.allclose(np.conj(D).T, G5 @ D @ G5, atol=1e-14)          # gamma_5-hermiticity survives
    Ug, _ = synth.gauge_transform(U, dims, 65)
    Dg = O.wilson_dense(Ug, dims, 0.12, 0.02, clover=O.clover_term(Ug, dims, 0.12, 1.3))
    t, tg = np.trace(np.linalg.inv(D)), np.trace(np.linalg.inv(Dg))
    assert abs(t - tg) <= 1e-11 * abs(t)
    assert abs(t - np.trace(np.linalg.inv(O.wilson_dense(U, dims, 0.12, 0.02)))) > 1e-6 * abs(t)


def test_clover_vanishes_on_pure_gauge_links():
    """A gauge transform of the free field has unit plaquettes: F = 0, and the clover-Wilson
    trace keeps the free-field closed form."""
    dims = (4, 2, 2, 4)
    V = int(np.prod(dims))
    Ufree = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    Ug, _ = synth.gauge_transform(Ufree, dims, 66)
    assert np.allclose(O.clover_term(Ug, dims, 0.12, 1.7), 0, atol=1e-14)
    D = O.wilson_dense(Ug, dims, 0.12, 0.0, clover=O.clover_term(Ug, dims, 0.12, 1.7))
    exact = free_wilson_trace_inverse(dims, 0.12)
    assert abs(np.trace(np.linalg.inv(D)).real - exact) <= 1e-10 * exact


# ------------------------------------------------------------------ quadrature bounds (Section 1.1.2)
@pytest.mark.parametrize("case", ["laplacian", "random_spd"])
def test_cg_quadrature_bounds_bracket_the_exact_quadrature(case):
    """Gauss (lower) and Gauss-Radau (upper) bounds from the CG coefficients: every step brackets
    b^T A^-1 b, the lower bound is b^T x_k, and the bracket closes to the tolerance."""
    rng = np.random.default_rng(3)
    if case == "laplacian":
        dims = (4, 4, 2, 4)
        A = O.laplacian_dense(dims, 0.2)
        mu = 0.2                                        # lambda_min of the shifted Laplacian
    else:
        n = 80
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.sort(rng.uniform(0.1, 5.0, n))
        A = (Q * lam) @ Q.T
        mu = 0.9 * lam[0]
    b = rng.standard_normal(A.shape[0])
    exact = b @ np.linalg.solve(A, b)
    x, hist = S.cg_quadrature_bounds(lambda v: A @ v, b, mu, 1e-12)
    for lo, hi in hist:
        assert lo <= exact * (1 + 1e-12) and hi >= exact * (1 - 1e-12)
    assert abs(hist[-1][0] - b @ x) <= 1e-12 * exact
    assert hist[-1][1] - hist[-1][0] <= 1e-12 * hist[-1][0]
    widths = [hi - lo for lo, hi in hist]
    assert widths[-1] < 1e-9 * widths[0]


def test_cg_quadrature_bounds_needs_mu_below_spectrum():
    """A node above lambda_min loses the guarantee: the 'upper bound' falls below the exact value
    at some step (the property the bound rests on is real)."""
    dims = (4, 4, 2, 4)
    A = O.laplacian_dense(dims, 0.2)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    exact = b @ np.linalg.solve(A, b)
    _, hist = S.cg_quadrature_bounds(lambda v: A @ v, b, 3.0, 1e-12)
    assert any(hi < exact * (1 - 1e-9) for _, hi in hist)


@pytest.mark.parametrize("dims,csw,with_mf", [((4, 2, 2, 2), 0.0, True), ((2, 4, 2, 4), 0.0, False),
                                              ((4, 2, 2, 2), 1.3, True), ((2, 2, 4, 2), 0.7, False)])
def test_schur_complement_matches_dense_partition(dims, csw, with_mf):
    """wilson_schur_apply against the Schur complement of the dense matrix: rows and columns
    of D split by site parity, S = D_oo - D_oe D_ee^-1 D_eo (numpy's inverse), applied to a
    random odd-site vector; the even sites of the result are zero."""
    from paper_1302_4018_gb300 import synth

    U = synth.gauge_links(dims, 0.5, 21)
    V = int(np.prod(dims))
    mf = synth.mass_field(dims, 0.05, 22) if with_mf else None
    C = O.clover_term(U, dims, 0.13, csw) if csw else None
    D = O.wilson_dense(U, dims, 0.13, 0.02, mf, clover=C)
    par = np.repeat(O.site_parity(dims), 12)
    e, o = np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]
    S = D[np.ix_(o, o)] - D[np.ix_(o, e)] @ np.linalg.inv(D[np.ix_(e, e)]) @ D[np.ix_(e, o)]
    x = synth.random_spinors(dims, 1, 23)[0]
    got = O.wilson_schur_apply(x, U, dims, 0.13, 0.02, mf, clover=C).reshape(-1)
    assert np.allclose(got[o], S @ x.reshape(-1)[o], rtol=0, atol=1e-12 * np.abs(S @ x.reshape(-1)[o]).max())
    assert not np.any(got[e])
    # and the parity split itself: every hop of D connects sites of opposite parity, so D_ee and
    # D_oo are block diagonal over sites
    site = np.repeat(np.arange(V), 12)
    for idx in (e, o):
        blk = D[np.ix_(idx, idx)]
        assert not np.any(blk[site[idx][:, None] != site[idx][None, :]])


def test_schur_complement_needs_even_extents():
    from paper_1302_4018_gb300 import synth

    U = synth.gauge_links((4, 3, 2, 2), 0.3, 1)
    with pytest.raises(ValueError):
        O.wilson_schur_apply(np.zeros((48, 4, 3), complex), U, (4, 3, 2, 2), 0.12)
