"""The hierarchical-probing trace estimator (oracle, test infrastructure only).

Section 1 of arXiv:1302.4018 writes the estimator as (1/s) sum_k z_k^T f(A) z_k;
Section 2.2 makes the vectors nested so that every prefix s reuses the
quadratures of the shorter prefixes; Section 4 multiplies every vector by one
Z_2 vector z_0 (Eq. removebias); Section 5.3 dilutes the 12 spin-colour
components fully, so probe m of the space-time sequence stands for 12 right
hand sides  v_{m,a} = (z_0 (.) z_m) (x) e_a,  a = 0..11, and
    q_m = sum_a v_{m,a}^H A^-1 v_{m,a},     T_s = (1/s) sum_{m<s} q_m.
For the (scalar) Laplacian there is one right-hand side per probe.

The derivative of T_s with respect to a real per-site mass mu(x) (the
diagonal term) follows from d(A^-1) = -A^-1 (dA) A^-1:
    dT_s / dmu(x) = -(1/s) sum_{m,a} sum_c conj(y_{m,a}(x, c)) x_{m,a}(x, c),
with x = A^-1 v and y = A^-H v.  This oracle solves the adjoint system
explicitly (it does not use gamma_5-hermiticity).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import operators as ops
from . import solvers
from . import probing as Pr
from .probing import probe_phases, probe_values


def probe_vectors(dims: Sequence[int], first: int, count: int, z0_seed: int,
                  loc: Sequence[int] | None = None, kind: str = "hp") -> np.ndarray:
    """v_m = z_0 (.) z_m as complex [count, V] (correctly rounded entries).  kind: "hp"
    (hierarchical probing), "natural" (Hadamard vectors in natural order, bias removed), "z2"
    (independent Z_2 noise vectors, seeded by z0_seed)."""
    if kind == "natural":
        return probe_values(Pr.probe_phases_natural(int(np.prod(dims)), first, count, z0_seed), 2)
    if kind == "z2":
        return probe_values(Pr.probe_phases_z2(int(np.prod(dims)), first, count, z0_seed), 2)
    ph, P = probe_phases(dims, first, count, z0_seed, loc=loc)
    return probe_values(ph, P)


def z0_variance(B: np.ndarray, Z: np.ndarray, s: int) -> float:
    """Exact variance over the Z_2 vector z_0 of T_s = (1/s) sum_{m<s} (z_0 (.) z_m)^H B (z_0 (.) z_m)
    for real +-1 probing vectors z_m (rows of Z): writing C = sum_{m<s} z_m z_m^T,
    T_s = (1/s) sum_{i,j} z0_i z0_j B_ij C_ij, whose diagonal part is Tr B for every z_0 and whose
    pairs i < j are uncorrelated with unit variance, so
        Var(T_s) = (1/s^2) sum_{i<j} |B_ij + B_ji|^2 C_ij^2
    (Section 1.1.2's variance of the Z_2 estimator, 2 sum_{i!=j} B_ij^2 for s = 1 and symmetric B)."""
    Zs = np.asarray(Z[:s], dtype=float)
    C = Zs.T @ Zs
    W = np.abs(B + B.T) ** 2 * C ** 2
    return float(np.sum(np.triu(W, 1))) / s ** 2


# ------------------------------------------------------------------ Section 5.3 statistics
def sample_variance(x: np.ndarray, ddof: int = 1) -> float:
    """(1/(n - ddof)) sum_i |x_i - mean|^2 over the n entries of x, written out."""
    x = np.asarray(x)
    n = x.shape[0]
    m = sum(x) / n
    return float(sum(abs(v - m) ** 2 for v in x) / (n - ddof))


def speedup_ratio(T: np.ndarray, V_stoc: float | None = None, ddof: int = 1) -> np.ndarray:
    """Section 5.3: R_s = V_stoc / (V_hp(s) s) for s = 1..S, from the estimates T[i, s-1] of n runs
    (one row per bias-removal vector z_0^(i), one column per s).  V_hp(s) is the variance over the
    runs of T_s; V_stoc, the variance of the standard Z_2 estimator with one vector, defaults to
    V_hp(1): the first probing vector is z_0 (.) h_0 = z_0, a Z_2 noise vector itself.  The factor s
    compares equal work: n s noise vectors would divide V_stoc by s."""
    T = np.asarray(T)
    S = T.shape[1]
    v_hp = np.array([sample_variance(T[:, s], ddof) for s in range(S)])
    v0 = v_hp[0] if V_stoc is None else V_stoc
    return np.array([v0 / (v_hp[s] * (s + 1)) for s in range(S)])


def jackknife(samples: np.ndarray, stat) -> tuple[float, float]:
    """Delete-one jackknife (the error estimate of Section 5.3): stat over all n samples, and
    err = sqrt((n - 1)/n sum_i (stat_(i) - mean_i stat_(i))^2) with stat_(i) computed without
    sample i."""
    samples = np.asarray(samples)
    n = samples.shape[0]
    full = stat(samples)
    loo = [stat(np.concatenate([samples[:i], samples[i + 1:]])) for i in range(n)]
    m = sum(loo) / n
    err = np.sqrt((n - 1) / n * sum((v - m) ** 2 for v in loo))
    return full, err


# ------------------------------------------------------------------ prefix
def trace_prefix(q: Sequence[complex]) -> np.ndarray:
    """T_s = (1/s) sum_{m<s} q_m, s = 1..len(q), plain sequential FP64 sums."""
    out = np.empty(len(q), dtype=complex)
    acc = 0.0 + 0.0j
    for s in range(1, len(q) + 1):
        acc = acc + q[s - 1]
        out[s - 1] = acc / s
    return out


def trace_prefix_kahan(q: Sequence[complex]) -> np.ndarray:
    """The same prefix with Kahan-compensated sums (cross-check of rounding)."""
    out = np.empty(len(q), dtype=complex)
    sr = cr = si = ci = 0.0
    for s in range(1, len(q) + 1):
        for part in (0, 1):
            v = q[s - 1].real if part == 0 else q[s - 1].imag
            if part == 0:
                y = v - cr
                t = sr + y
                cr = (t - sr) - y
                sr = t
            else:
                y = v - ci
                t = si + y
                ci = (t - si) - y
                si = t
        out[s - 1] = complex(sr, si) / s
    return out


# ------------------------------------------------------------------ Laplacian
def laplacian_solutions(dims, mass, W, tol=1e-13, mass_field=None, method="cg"):
    """x_m = A^-1 v_m for the rows v_m of W."""
    if method == "dense":
        A = ops.laplacian_dense(dims, mass, mass_field)
        return solvers.dense_solve(A, W.T).T
    X = np.empty_like(W)
    for m in range(W.shape[0]):
        X[m], _ = solvers.cg(lambda v: ops.laplacian_apply(v, dims, mass, mass_field), W[m], tol=tol)
    return X


def laplacian_quadratures(dims, mass, first, count, z0_seed, tol=1e-13, mass_field=None,
                          method="cg", loc=None, kind="hp"):
    """q_m = v_m^H A^-1 v_m, m = first..first+count-1 (kind: the probing sequence, see probe_vectors)."""
    W = probe_vectors(dims, first, count, z0_seed, loc=loc, kind=kind)
    if np.all(W.imag == 0):
        W = W.real
    X = laplacian_solutions(dims, mass, W, tol, mass_field, method)
    return np.array([np.vdot(W[m], X[m]) for m in range(count)])


def laplacian_deflated_quadratures(dims, mass, evecs, first, count, z0_seed, mass_field=None):
    """Deflated probing (the variance reduction the conclusions pair with probing): with k
    orthonormal real eigenvectors V (columns of evecs, n x k) of the real symmetric A and
    P = I - V V^T, A^-1 = V diag(1/lambda) V^T + A^-1 P, so
        Tr A^-1 = sum_j 1/lambda_j + Tr(A^-1 P),
    and the probed part uses the projected vectors:  q_m = (P v_m)^H A^-1 (P v_m)  (dense solve)."""
    W = probe_vectors(dims, first, count, z0_seed)
    if np.all(W.imag == 0):
        W = W.real
    V = np.asarray(evecs, dtype=float)
    Wp = W - (W @ V) @ V.T
    A = ops.laplacian_dense(dims, mass, mass_field)
    X = solvers.dense_solve(A, Wp.T).T
    return np.array([np.vdot(Wp[m], X[m]) for m in range(count)])


def laplacian_lowest_eigenpairs(dims, mass, k, mass_field=None):
    """The k lowest eigenpairs of the shifted Laplacian (the modes deflation removes): the dense
    matrix of laplacian_dense diagonalised by numpy's symmetric eigensolver; returns (evals [k]
    ascending, evecs [k][V] orthonormal rows)."""
    lam, V = np.linalg.eigh(ops.laplacian_dense(dims, mass, mass_field))
    return lam[:k], np.ascontiguousarray(V[:, :k].T)


def deflated_trace_prefix(evals, q) -> np.ndarray:
    """T_s = sum_j 1/lambda_j + (1/s) sum_{m<s} q_m."""
    return float(np.sum(1.0 / np.asarray(evals, dtype=float))) + trace_prefix(q)


def laplacian_grad_mass_field(dims, mass, s, z0_seed, tol=1e-13, mass_field=None, method="cg"):
    """dT_s/dmu(x); A is real symmetric (its stencil is symmetric), so A^-H v = A^-1 v = x."""
    W = probe_vectors(dims, 0, s, z0_seed)
    if np.all(W.imag == 0):
        W = W.real
    X = laplacian_solutions(dims, mass, W, tol, mass_field, method)
    Y = X
    return -(np.sum(np.conj(Y) * X, axis=0)) / s


# ------------------------------------------------------------------ Wilson
def _dilute(w: np.ndarray, a: int) -> np.ndarray:
    V = w.shape[0]
    b = np.zeros((V, 12), dtype=complex)
    b[:, a] = w
    return b.reshape(V, 4, 3)


def wilson_solutions(dims, U, kappa, W, tol=1e-13, mass=0.0, mass_field=None, method="bicgstab",
                     dagger=False, csw=0.0):
    """x_{m,a} = D^-1 v_{m,a} (or D^-H v_{m,a}); returns complex [count, 12, V, 4, 3].
    csw != 0 adds the clover term C(x) of operators.clover_term."""
    count, V = W.shape
    X = np.empty((count, 12, V, 4, 3), dtype=complex)
    clover = ops.clover_term(U, dims, kappa, csw) if csw else None
    if method == "dense":
        D = ops.wilson_dense(U, dims, kappa, mass, mass_field, clover=clover)
        if dagger:
            D = np.conj(D).T
        B = np.zeros((12 * V, 12 * count), dtype=complex)
        for m in range(count):
            for a in range(12):
                B[:, 12 * m + a] = _dilute(W[m], a).reshape(-1)
        Xs = solvers.dense_solve(D, B)
        for m in range(count):
            for a in range(12):
                X[m, a] = Xs[:, 12 * m + a].reshape(V, 4, 3)
        return X

    def apply(v):
        return ops.wilson_apply(v, U, dims, kappa, mass, mass_field, dagger=dagger, clover=clover)

    for m in range(count):
        for a in range(12):
            X[m, a], _ = solvers.bicgstab(apply, _dilute(W[m], a), tol=tol)
    return X


def wilson_quadratures(dims, U, kappa, first, count, z0_seed, tol=1e-13, mass=0.0,
                       mass_field=None, method="bicgstab", loc=None, csw=0.0):
    """q_m = sum_a v_{m,a}^H D^-1 v_{m,a} with full spin-colour dilution."""
    W = probe_vectors(dims, first, count, z0_seed, loc=loc)
    X = wilson_solutions(dims, U, kappa, W, tol, mass, mass_field, method, csw=csw)
    V = W.shape[1]
    q = np.zeros(count, dtype=complex)
    for m in range(count):
        for a in range(12):
            q[m] += np.vdot(_dilute(W[m], a), X[m, a])
    return q


def gamma5_hermitian_dense(dims, U, kappa, mass=0.0, mass_field=None, csw=0.0):
    """Q = gamma_5 D as a dense matrix: gamma_5-hermiticity (D^H = gamma_5 D gamma_5) makes Q
    Hermitian, so its eigenvalues are real and |lambda| runs over the singular values of D.
    gamma_5 = diag(1, 1, -1, -1) on the spins (chiral basis of operators.gamma_matrices)."""
    clover = ops.clover_term(U, dims, kappa, csw) if csw else None
    D = ops.wilson_dense(U, dims, kappa, mass, mass_field, clover=clover)
    V = int(np.prod(dims))
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    return g5[:, None] * D


def wilson_lowest_eigenpairs(dims, U, kappa, k, mass=0.0, mass_field=None, csw=0.0):
    """The k eigenpairs of Q = gamma_5 D with the smallest |lambda| (numpy's Hermitian
    eigensolver on the dense Q): returns (evals [k] ordered by |lambda|, evecs [k][V][4][3])."""
    Q = gamma5_hermitian_dense(dims, U, kappa, mass, mass_field, csw)
    Q = 0.5 * (Q + np.conj(Q).T)   # Hermitian up to the rounding of its assembly
    lam, W = np.linalg.eigh(Q)
    order = np.argsort(np.abs(lam), kind="stable")[:k]
    V = int(np.prod(dims))
    return lam[order], np.ascontiguousarray(W[:, order].T.reshape(k, V, 4, 3))


def wilson_deflated_quadratures(dims, U, kappa, evals, evecs, first, count, z0_seed, mass=0.0,
                                mass_field=None, csw=0.0):
    """Deflated probing of the Wilson matrix, written out literally.  With eigenpairs
    Q w_j = lambda_j w_j of Q = gamma_5 D (evecs [k][V][4][3], orthonormal) and the left vectors
    u_j = gamma_5 w_j (D^-1 u_j = Q^-1 w_j = w_j / lambda_j; U = [u_j] is orthonormal),
        D^-1 = D^-1 U U^H + D^-1 (I - U U^H),  Tr D^-1 = sum_j (w_j^H gamma_5 w_j) / lambda_j + Tr(D^-1 (I - U U^H)),
    and the second term is probed with the diluted vectors:
        q_m = sum_a v_{m,a}^H D^-1 (I - U U^H) v_{m,a}    (dense solves).
    Returns (q [count], the exact part sum_j (w_j^H gamma_5 w_j) / lambda_j)."""
    W = probe_vectors(dims, first, count, z0_seed)
    V = W.shape[1]
    clover = ops.clover_term(U, dims, kappa, csw) if csw else None
    D = ops.wilson_dense(U, dims, kappa, mass, mass_field, clover=clover)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    Wv = np.asarray(evecs).reshape(len(evals), 12 * V).T          # columns w_j
    Uv = g5[:, None] * Wv                                           # columns u_j = gamma_5 w_j
    B = np.zeros((12 * V, 12 * count), dtype=complex)
    for m in range(count):
        for a in range(12):
            B[:, 12 * m + a] = _dilute(W[m], a).reshape(-1)
    Bp = B - Uv @ (np.conj(Uv).T @ B)
    X = solvers.dense_solve(D, Bp)
    q = np.array([sum(np.vdot(B[:, 12 * m + a], X[:, 12 * m + a]) for a in range(12)) for m in range(count)])
    exact = sum(np.vdot(Wv[:, j], g5 * Wv[:, j]) / evals[j] for j in range(len(evals)))
    return q, complex(exact)


def wilson_smallest_singular_triplets(dims, U, kappa, k, mass=0.0, mass_field=None, csw=0.0):
    """The k smallest singular triplets D v_j = sigma_j u_j of the Wilson matrix (numpy's dense SVD):
    returns (sigma [k] ascending, right [k][V][4][3], left [k][V][4][3]), both sets orthonormal."""
    clover = ops.clover_term(U, dims, kappa, csw) if csw else None
    D = ops.wilson_dense(U, dims, kappa, mass, mass_field, clover=clover)
    Ul, s, Vh = np.linalg.svd(D)
    order = np.argsort(s, kind="stable")[:k]
    V = int(np.prod(dims))
    right = np.conj(Vh[order]).reshape(k, V, 4, 3)
    left = Ul[:, order].T.reshape(k, V, 4, 3)
    return s[order], np.ascontiguousarray(right), np.ascontiguousarray(left)


def wilson_deflated_quadratures_svd(dims, U, kappa, sigma, right, left, first, count, z0_seed, mass=0.0,
                                    mass_field=None, csw=0.0):
    """Deflated probing of the Wilson matrix with singular triplets D v_j = sigma_j u_j (right
    vectors v_j, left vectors u_j, each set orthonormal), written out literally:
        D^-1 u_j = v_j / sigma_j,  D^-1 = sum_j v_j u_j^H / sigma_j + D^-1 (I - U U^H),
        Tr D^-1 = sum_j (u_j^H v_j) / sigma_j + Tr(D^-1 (I - U U^H)),
    the second term probed: q_m = sum_a v_{m,a}^H D^-1 (I - U U^H) v_{m,a} (dense solves).
    Returns (q [count], the exact part)."""
    W = probe_vectors(dims, first, count, z0_seed)
    V = W.shape[1]
    k = len(sigma)
    clover = ops.clover_term(U, dims, kappa, csw) if csw else None
    D = ops.wilson_dense(U, dims, kappa, mass, mass_field, clover=clover)
    Rv = np.asarray(right).reshape(k, 12 * V).T
    Lv = np.asarray(left).reshape(k, 12 * V).T
    B = np.zeros((12 * V, 12 * count), dtype=complex)
    for m in range(count):
        for a in range(12):
            B[:, 12 * m + a] = _dilute(W[m], a).reshape(-1)
    Bp = B - Lv @ (np.conj(Lv).T @ B)
    X = solvers.dense_solve(D, Bp)
    q = np.array([sum(np.vdot(B[:, 12 * m + a], X[:, 12 * m + a]) for a in range(12)) for m in range(count)])
    exact = sum(np.vdot(Lv[:, j], Rv[:, j]) / sigma[j] for j in range(k))
    return q, complex(exact)


def wilson_grad_mass_field(dims, U, kappa, s, z0_seed, tol=1e-13, mass=0.0, mass_field=None,
                           method="bicgstab", csw=0.0):
    """dT_s/dmu(x) = -(1/s) sum_{m<s,a} sum_c conj(y(x,c)) x(x,c), y = D^-H v solved explicitly."""
    W = probe_vectors(dims, 0, s, z0_seed)
    X = wilson_solutions(dims, U, kappa, W, tol, mass, mass_field, method, csw=csw)
    Y = wilson_solutions(dims, U, kappa, W, tol, mass, mass_field, method, dagger=True, csw=csw)
    g = np.sum(np.conj(Y) * X, axis=(0, 1, 3, 4))
    return -g / s
