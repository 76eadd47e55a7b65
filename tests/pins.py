"""Closed forms that pin the oracle (not part of it).

Each is an independent mathematical statement of a quantity the oracle
computes another way.
"""
import numpy as np


def laplacian_eigenvalues(dims, mass):
    """Eigenvalues m + sum_mu 4 sin^2(pi k_mu / L_mu) of the shifted periodic Laplacian (Section 5)."""
    grids = np.meshgrid(*[4.0 * np.sin(np.pi * np.arange(L) / L) ** 2 for L in dims], indexing="ij")
    return (mass + sum(grids)).reshape(-1)


def laplacian_trace_inverse(dims, mass):
    return float(np.sum(1.0 / laplacian_eigenvalues(dims, mass)))


def free_wilson_trace_inverse(dims, kappa, mass=0.0):
    """Tr D^-1 for U = 1.  A plane wave e^{ip.x} u sees
    D(p) = a + i sum_mu g_mu b_mu, a = 1 + m - 2 kappa sum cos p_mu, b_mu = 2 kappa sin p_mu,
    so D(p)^-1 = (a - i g.b)/(a^2 + b^2) and its 12-dimensional trace is 12 a/(a^2 + b^2)."""
    ps = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    a = 1.0 + mass - 2 * kappa * sum(np.cos(p) for p in ps)
    b2 = sum((2 * kappa * np.sin(p)) ** 2 for p in ps)
    return float(np.sum(12.0 * a / (a * a + b2)))


def free_wilson_singular_values(dims, kappa, mass=0.0):
    """Singular values of D for U = 1, each of multiplicity 12: with D(p) = a + i g.b as above
    (the g_mu Hermitian and anticommuting), D(p)^H D(p) = (a - i g.b)(a + i g.b) = a^2 + b^2."""
    ps = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    a = 1.0 + mass - 2 * kappa * sum(np.cos(p) for p in ps)
    b2 = sum((2 * kappa * np.sin(p)) ** 2 for p in ps)
    return np.repeat(np.sqrt(a * a + b2).reshape(-1), 12)


def torus_distance(x, y, dims):
    return sum(min(abs(a - b), L - abs(a - b)) for a, b, L in zip(x, y, dims))
