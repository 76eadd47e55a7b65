"""Textbook Krylov solvers in FP64 (oracle, test infrastructure only).

Section 1.1.2 of arXiv:1302.4018 computes each quadrature z^H A^-1 z by
solving A x = z and forming z^H x.  These are the plain textbook methods:
CG (Hestenes-Stiefel) for the Hermitian positive definite Laplacian and
BiCGStab (van der Vorst) for the non-Hermitian Wilson matrix, x_0 = 0,
shadow residual r^ = b, restart r^ = r on breakdown, stopped on the TRUE
relative residual ||b - A x|| / ||b|| (the recursive residual only proposes
a stop; it is then recomputed from x).
"""
from __future__ import annotations

from typing import Callable

import numpy as np

Apply = Callable[[np.ndarray], np.ndarray]


def _norm(v: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(v, v).real))


def cg(apply: Apply, b: np.ndarray, tol: float = 1e-13, maxiter: int = 10000) -> tuple[np.ndarray, int]:
    bn = _norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    for it in range(1, maxiter + 1):
        Ap = apply(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        if np.sqrt(rr_new) <= tol * bn:
            r = b - apply(x)                     # true residual decides
            rr_new = np.vdot(r, r).real
            if np.sqrt(rr_new) <= tol * bn:
                return x, it
            p = r.copy()
            rr = rr_new
            continue
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError("oracle CG did not converge")


def cg_quadrature_bounds(apply: Apply, b: np.ndarray, mu: float, tol: float,
                         maxiter: int = 10000) -> tuple[np.ndarray, list]:
    """CG on a Hermitian positive definite A with bounds on the quadrature b^H A^-1 b (Section 1.1.2:
    the Lanczos/Gauss quadrature of z^H A^-1 z comes with lower and upper bounds).

    With x_0 = 0, step lengths gamma_k = ||r_k||^2 / (p_k, A p_k) and delta_{k+1} = ||r_{k+1}||^2 /
    ||r_k||^2, the Gauss rule after k steps is G_k = sum_{j<k} gamma_j ||r_j||^2 = b^H x_k (a lower
    bound), and for 0 < mu <= lambda_min(A) the Gauss-Radau rule with the node mu adds
    gt_k ||r_k||^2 (an upper bound), gt_0 = 1/mu,
        gt_{k+1} = (gt_k - gamma_k) / (mu (gt_k - gamma_k) + delta_{k+1})
    (the CG form of the Gauss-Radau recurrence of Golub and Meurant).  Stops when the bracket
    is at most tol times the lower bound; returns x and the list of (lower, upper) per step."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    G, gt = 0.0, 1.0 / mu
    hist = [(G, G + gt * rr)]
    if rr == 0.0:
        return x, hist
    for _ in range(maxiter):
        Ap = apply(p)
        gamma = rr / np.vdot(p, Ap).real
        x = x + gamma * p
        r = r - gamma * Ap
        rr_new = np.vdot(r, r).real
        delta = rr_new / rr
        G += gamma * rr
        gt = (gt - gamma) / (mu * (gt - gamma) + delta)
        hist.append((G, G + gt * rr_new))
        if gt * rr_new <= tol * G:
            return x, hist
        p = r + delta * p
        rr = rr_new
    raise RuntimeError("oracle CG did not reach the quadrature tolerance")


def bicgstab(apply: Apply, b: np.ndarray, tol: float = 1e-13, maxiter: int = 10000) -> tuple[np.ndarray, int]:
    bn = _norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0
    r = b.copy()
    rhat = b.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxiter + 1):
        rho_new = np.vdot(rhat, r)
        if abs(rho_new) < 1e-30 * _norm(r) * _norm(rhat):
            rhat = r.copy()                      # breakdown: new shadow residual
            rho_new = np.vdot(rhat, r)
            p = np.zeros_like(b)
            v = np.zeros_like(b)
            rho = alpha = omega = 1.0 + 0j
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho_new / np.vdot(rhat, v)
        s = r - alpha * v
        t = apply(s)
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0 + 0j
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        if _norm(r) <= tol * bn:
            r = b - apply(x)                     # true residual decides
            if _norm(r) <= tol * bn:
                return x, it
            rhat = r.copy()
            rho = alpha = omega = 1.0 + 0j
            p = np.zeros_like(b)
            v = np.zeros_like(b)
    raise RuntimeError("oracle BiCGStab did not converge")


def dense_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """LU solve (LAPACK) for tiny lattices."""
    return np.linalg.solve(A, B)
