"""Lattice operators of arXiv:1302.4018, written out plainly in FP64.

Oracle (test infrastructure only).

* Shifted periodic Laplacian (Section 5 control problem, written for
  d = 4):  A = (2d + m) I - sum_mu (S_mu + S_mu^T), plus an optional
  per-site mass field mu(x) on the diagonal.
* Wilson-Dirac matrix (Section 1.1.1: a sparse matrix on a periodic 4-D
  lattice with 12 = 4 spin x 3 colour unknowns per site; Section 5.3 uses its
  clover variant).  Wilson form in kappa normalisation:
      (D psi)(x) = (1 + m + mu(x)) psi(x) + C(x) psi(x)
                   - kappa sum_mu [ (1 - g_mu) U_mu(x)        psi(x + mu)
                                  + (1 + g_mu) U_mu(x - mu)^H psi(x - mu) ]
  with explicit 4x4 gamma matrices (chiral basis, gamma_5 diagonal) and full
  3x3 link products: no spin projection, no link reconstruction.  C(x) is the
  Sheikholeslami-Wohlert (clover) term the paper's Section 5.3 operator
  carries (it only names the discretisation; the form used is the standard
  clover-leaf one):
      C(x) = -c_sw kappa sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
      sigma_{mu nu} = (i/2) [g_mu, g_nu],
      F_{mu nu}(x) = traceless part of (Q_{mu nu}(x) - Q_{mu nu}(x)^H) / (8 i),
  Q_{mu nu}(x) the sum of the four plaquettes of the mu-nu plane that start and
  end at x, each run mu-then-nu (counter-clockwise).  c_sw = 0 is plain Wilson.

Field layout: arrays indexed by the lexicographic site (x_1 fastest); a spinor
is complex128 [V, 4, 3] (spin, colour); a gauge field is complex128
[V, 4, 3, 3] (site, direction mu = 1..4 along x_1..x_4, row, column).
Unknown number (spin s, colour c) of site x is 12 x + 3 s + c.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def _shape(dims: Sequence[int]) -> tuple:
    return tuple(reversed([int(v) for v in dims]))


def _axis(dims: Sequence[int], mu: int) -> int:
    """numpy axis of lattice direction mu (0-based) in the reversed-dims shape."""
    return len(dims) - 1 - mu


def shift_field(f: np.ndarray, dims: Sequence[int], mu: int, sign: int) -> np.ndarray:
    """g(x) = f(x + sign * mu_hat) on the torus (f indexed by site first)."""
    V = f.shape[0]
    g = f.reshape(_shape(dims) + f.shape[1:])
    g = np.roll(g, -sign, axis=_axis(dims, mu))
    return g.reshape((V,) + f.shape[1:])


# ------------------------------------------------------------------ Laplacian
def laplacian_apply(x: np.ndarray, dims: Sequence[int], mass: float,
                    mass_field: np.ndarray | None = None) -> np.ndarray:
    """A x for x of shape [V] or [V, n] (real or complex)."""
    d = len(dims)
    diag = 2 * d + mass
    y = diag * x
    if mass_field is not None:
        y = y + (mass_field.reshape((-1,) + (1,) * (x.ndim - 1))) * x
    for mu in range(d):
        y = y - shift_field(x, dims, mu, +1) - shift_field(x, dims, mu, -1)
    return y


def laplacian_dense(dims: Sequence[int], mass: float, mass_field: np.ndarray | None = None) -> np.ndarray:
    """The Laplacian as a dense matrix, row by row from the stencil definition."""
    d = len(dims)
    V = int(np.prod(dims))
    A = np.zeros((V, V))
    strides = [int(np.prod(dims[:j])) for j in range(d)]
    for i in range(V):
        A[i, i] += 2 * d + mass + (0.0 if mass_field is None else mass_field[i])
        x = [(i // strides[j]) % dims[j] for j in range(d)]
        for mu in range(d):
            for sgn in (+1, -1):
                y = list(x)
                y[mu] = (y[mu] + sgn) % dims[mu]
                A[i, sum(y[j] * strides[j] for j in range(d))] -= 1.0
    return A


# ------------------------------------------------------------------ gammas
def pauli() -> list:
    return [np.array([[0, 1], [1, 0]], dtype=complex),
            np.array([[0, -1j], [1j, 0]], dtype=complex),
            np.array([[1, 0], [0, -1]], dtype=complex)]


def gamma_matrices() -> list:
    """Euclidean chiral basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = 1..3), g_4 = [[0, 1], [1, 0]],
    g_5 = g_1 g_2 g_3 g_4 = diag(1, 1, -1, -1).  Returns [g_1, g_2, g_3, g_4, g_5]."""
    Z = np.zeros((2, 2), dtype=complex)
    I2 = np.eye(2, dtype=complex)
    g = []
    for s in pauli():
        g.append(np.block([[Z, -1j * s], [1j * s, Z]]))
    g.append(np.block([[Z, I2], [I2, Z]]))
    g.append(g[0] @ g[1] @ g[2] @ g[3])
    return g


# ------------------------------------------------------------------ clover term
def sigma_munu(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2) [g_mu, g_nu], a Hermitian 4x4 matrix (mu, nu 0-based)."""
    g = gamma_matrices()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _site_index(x: Sequence[int], dims: Sequence[int]) -> int:
    i, stride = 0, 1
    for j in range(len(dims)):
        i += (x[j] % dims[j]) * stride
        stride *= dims[j]
    return i


def clover_leaves(U: np.ndarray, dims: Sequence[int], mu: int, nu: int) -> np.ndarray:
    """Q_{mu nu}(x) for every site: the four plaquettes of the mu-nu plane starting and ending at
    x, each run mu-then-nu, as products of 3x3 links, site by site; complex [V, 3, 3]."""
    V = int(np.prod(dims))
    strides = [int(np.prod(dims[:j])) for j in range(len(dims))]
    Q = np.zeros((V, 3, 3), dtype=complex)

    def link(x, d):
        return U[_site_index(x, dims), d]

    def step(x, d, n):
        y = list(x)
        y[d] += n
        return y

    H = lambda A: np.conj(A).T
    for i in range(V):
        x = [(i // strides[j]) % dims[j] for j in range(len(dims))]
        xm, xn = step(x, mu, -1), step(x, nu, -1)
        xmn = step(xm, nu, -1)
        # x -> x+mu -> x+mu+nu -> x+nu -> x
        Q[i] += link(x, mu) @ link(step(x, mu, 1), nu) @ H(link(step(x, nu, 1), mu)) @ H(link(x, nu))
        # x -> x+nu -> x+nu-mu -> x-mu -> x
        Q[i] += link(x, nu) @ H(link(step(xm, nu, 1), mu)) @ H(link(xm, nu)) @ link(xm, mu)
        # x -> x-mu -> x-mu-nu -> x-nu -> x
        Q[i] += H(link(xm, mu)) @ H(link(xmn, nu)) @ link(xmn, mu) @ link(xn, nu)
        # x -> x-nu -> x-nu+mu -> x+mu -> x
        Q[i] += H(link(xn, nu)) @ link(xn, mu) @ link(step(xn, mu, 1), nu) @ H(link(x, mu))
    return Q


def clover_field(U: np.ndarray, dims: Sequence[int], mu: int, nu: int) -> np.ndarray:
    """F_{mu nu}(x) = traceless part of (Q - Q^H) / (8 i); Hermitian, complex [V, 3, 3]."""
    Q = clover_leaves(U, dims, mu, nu)
    F = (Q - np.conj(np.transpose(Q, (0, 2, 1)))) / 8j
    tr = np.trace(F, axis1=1, axis2=2)
    return F - tr[:, None, None] * np.eye(3)[None] / 3.0


def clover_term(U: np.ndarray, dims: Sequence[int], kappa: float, csw: float) -> np.ndarray:
    """C(x) = -c_sw kappa sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x) as 12x12 matrices indexed
    (3 s + c, 3 t + d); complex [V, 12, 12]."""
    V = int(np.prod(dims))
    C = np.zeros((V, 12, 12), dtype=complex)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = clover_field(U, dims, mu, nu)
            s = sigma_munu(mu, nu)
            for i in range(V):
                C[i] += np.kron(s, F[i])
    return -csw * kappa * C


# ------------------------------------------------------------------ Wilson
def wilson_apply(psi: np.ndarray, U: np.ndarray, dims: Sequence[int], kappa: float,
                 mass: float = 0.0, mass_field: np.ndarray | None = None,
                 dagger: bool = False, clover: np.ndarray | None = None) -> np.ndarray:
    """D psi (or D^H psi when ``dagger``) for psi [V, 4, 3] complex; ``clover`` = the site
    matrices C(x) of clover_term (None: plain Wilson).

    D^H follows from transposing the blocks of D: the hopping term to x + mu
    becomes (1 + g_mu) U_mu(x) and the one to x - mu becomes
    (1 - g_mu) U_mu(x - mu)^H (the projectors are Hermitian); C(x) is Hermitian.
    """
    g = gamma_matrices()
    I4 = np.eye(4, dtype=complex)
    diag = 1.0 + mass
    out = diag * psi
    if mass_field is not None:
        out = out + mass_field[:, None, None] * psi
    if clover is not None:
        Cx = np.conj(np.transpose(clover, (0, 2, 1))) if dagger else clover
        out = out + np.einsum("xij,xj->xi", Cx, psi.reshape(-1, 12)).reshape(psi.shape)
    hop = np.zeros_like(psi)
    for mu in range(4):
        P_fwd = I4 - g[mu] if not dagger else I4 + g[mu]
        P_bwd = I4 + g[mu] if not dagger else I4 - g[mu]
        U_mu = U[:, mu]
        psi_f = shift_field(psi, dims, mu, +1)
        col = np.einsum("xab,xsb->xsa", U_mu, psi_f)
        hop = hop + np.einsum("st,xta->xsa", P_fwd, col)
        psi_b = shift_field(psi, dims, mu, -1)
        U_b = shift_field(U_mu, dims, mu, -1)
        col = np.einsum("xba,xsb->xsa", np.conj(U_b), psi_b)
        hop = hop + np.einsum("st,xta->xsa", P_bwd, col)
    return out - kappa * hop


def site_parity(dims: Sequence[int]) -> np.ndarray:
    """(x_1 + ... + x_d) mod 2 for every lexicographic site (the red-black split of the lattice)."""
    V = int(np.prod(dims))
    strides = [int(np.prod(dims[:j])) for j in range(len(dims))]
    i = np.arange(V)
    return sum((i // strides[j]) % dims[j] for j in range(len(dims))) % 2


def wilson_schur_apply(x: np.ndarray, U: np.ndarray, dims: Sequence[int], kappa: float,
                       mass: float = 0.0, mass_field: np.ndarray | None = None,
                       clover: np.ndarray | None = None) -> np.ndarray:
    """The odd-site Schur complement of D (even-odd preconditioning of the Section 1.1.1 matrix,
    the operator a red-black ordered solve iterates on):  ordering the sites even then odd,
        D = [[A_e, -kappa H_eo], [-kappa H_oe, A_o]],   A = 1 + m + mu(x) + C(x) (site-diagonal),
        S = A_o - kappa^2 H_oe A_e^-1 H_eo.
    Returns S x_o on the odd sites and 0 on the even ones (x [V, 4, 3]; its even sites are
    ignored), from two applications of D and the diagonal blocks A_e solved site by site:
    y = D x_o has y_o = A_o x_o and y_e = -kappa H_eo x_o; w = A_e^-1 y_e on the even sites;
    z = D w has z_o = -kappa H_oe w = kappa^2 H_oe A_e^-1 H_eo x_o; so S x_o = y_o - z_o.
    The split needs every extent even: an odd extent wraps around between sites of one parity."""
    if any(int(L) % 2 for L in dims):
        raise ValueError("the even-odd split needs every lattice extent even: %s" % (tuple(dims),))
    par = site_parity(dims)
    odd = (par == 1)[:, None, None]
    y = wilson_apply(np.where(odd, x, 0), U, dims, kappa, mass, mass_field, clover=clover)
    ye = np.where(odd, 0, y)
    d = 1.0 + mass + (np.zeros(y.shape[0]) if mass_field is None else mass_field)
    if clover is None:
        w = ye / d[:, None, None]
    else:
        ev = np.nonzero(par == 0)[0]
        A = clover[ev] + d[ev, None, None] * np.eye(12)[None]
        w = np.zeros_like(ye)
        w[ev] = np.linalg.solve(A, ye[ev].reshape(-1, 12, 1)).reshape(-1, 4, 3)
    z = wilson_apply(w, U, dims, kappa, mass, mass_field, clover=clover)
    return np.where(odd, y - z, 0)


def wilson_dense(U: np.ndarray, dims: Sequence[int], kappa: float, mass: float = 0.0,
                 mass_field: np.ndarray | None = None, clover: np.ndarray | None = None) -> np.ndarray:
    """D as a dense 12V x 12V matrix, block by block from its definition."""
    g = gamma_matrices()
    I4 = np.eye(4, dtype=complex)
    d = 4
    V = int(np.prod(dims))
    D = np.zeros((12 * V, 12 * V), dtype=complex)
    strides = [int(np.prod(dims[:j])) for j in range(d)]
    for i in range(V):
        m_i = mass + (0.0 if mass_field is None else mass_field[i])
        D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += (1.0 + m_i) * np.eye(12)
        if clover is not None:
            D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += clover[i]
        x = [(i // strides[j]) % dims[j] for j in range(d)]
        for mu in range(d):
            y = list(x)
            y[mu] = (y[mu] + 1) % dims[mu]
            jf = sum(y[k] * strides[k] for k in range(d))
            D[12 * i:12 * i + 12, 12 * jf:12 * jf + 12] += -kappa * np.kron(I4 - g[mu], U[i, mu])
            y = list(x)
            y[mu] = (y[mu] - 1) % dims[mu]
            jb = sum(y[k] * strides[k] for k in range(d))
            D[12 * i:12 * i + 12, 12 * jb:12 * jb + 12] += -kappa * np.kron(I4 + g[mu], np.conj(U[jb, mu]).T)
    return D
