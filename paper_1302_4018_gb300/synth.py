"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the probing method: it only draws the
inputs the method is applied to (gauge links, mass fields, random spinors,
the uneven batch of lattices).  It imports nothing else from this package,
so the oracle can use it without touching the CUDA library.

Gauge links (stand-in for the missing 32^3x64 ensemble of Section 5.3):
  U_mu(x) = exp(i eps H),  H = (G + G^H)/2 - tr(...)/3 I,
  G_ij = (a + i b)/sqrt(2),  a, b ~ N(0, 1) from numpy PCG64(seed), drawn in
  the order (site, mu, i, j, re/im).  The exponential is evaluated by
  scaling and squaring: a degree-10 Taylor series of (i eps H)/8 (norm below
  0.5 for every config used, truncation < 1e-13) squared three times,
  followed by re-unitarisation: Gram-Schmidt on rows 1-2 and
  row 3 = conj(row1 x row2), which makes every link special unitary to
  rounding.  The matrix algebra runs in torch on the requested device (the
  CPU by default); the random draws are always numpy PCG64 on the host.
  Layout complex128 [V, 4, 3, 3].
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def volume(dims: Sequence[int]) -> int:
    v = 1
    for L in dims:
        v *= int(L)
    return v


def _expm_i(H, eps: float, degree: int = 10, squarings: int = 3):
    import torch

    n = H.shape[-1]
    X = (1j * eps / (1 << squarings)) * H
    eye = torch.eye(n, dtype=H.dtype, device=H.device)
    out = eye.expand_as(H).clone()
    term = out.clone()
    for k in range(1, degree + 1):
        term = torch.matmul(term, X) / k
        out += term
    for _ in range(squarings):
        out = torch.matmul(out, out)
    return out


def reunitarize(U):
    """Gram-Schmidt on rows 1-2, row 3 = conj(row1 x row2) (numpy or torch input)."""
    import torch

    T = torch.as_tensor(U)
    r1 = T[..., 0, :]
    r1 = r1 / torch.sqrt(torch.sum(torch.abs(r1) ** 2, dim=-1, keepdim=True))
    r2 = T[..., 1, :]
    r2 = r2 - torch.sum(torch.conj(r1) * r2, dim=-1, keepdim=True) * r1
    r2 = r2 / torch.sqrt(torch.sum(torch.abs(r2) ** 2, dim=-1, keepdim=True))
    r3 = torch.conj(torch.linalg.cross(r1, r2, dim=-1))
    out = torch.stack([r1, r2, r3], dim=-2)
    return out.numpy() if isinstance(U, np.ndarray) else out


def gauge_links(dims: Sequence[int], eps: float, seed: int, device: str = "cpu",
                chunk_sites: int = 1 << 18) -> np.ndarray:
    """SU(3) links U = exp(i eps H) on every site and direction; complex128 numpy [V, 4, 3, 3]."""
    import torch

    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((V, 4, 3, 3), dtype=complex)
    eye = None
    for s0 in range(0, V, chunk_sites):
        n = min(chunk_sites, V - s0)
        ab = torch.from_numpy(rng.standard_normal((n, 4, 3, 3, 2))).to(device)
        G = torch.complex(ab[..., 0], ab[..., 1]) / math.sqrt(2.0)
        H = 0.5 * (G + torch.conj(G.transpose(-1, -2)))
        if eye is None:
            eye = torch.eye(3, dtype=H.dtype, device=H.device)
        tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1).real
        H = H - (tr / 3.0)[..., None, None] * eye
        if eps == 0.0:
            U = eye.expand(n, 4, 3, 3)
        else:
            U = reunitarize(_expm_i(H, eps))
        out[s0:s0 + n] = U.cpu().numpy()
    return out


def gauge_transform(U: np.ndarray, dims: Sequence[int], seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Random SU(3) gauge transformation g(x); returns (U', g) with
    U'_mu(x) = g(x) U_mu(x) g(x + mu)^H."""
    V = volume(dims)
    g = gauge_links([V], 1.0, seed)[:, 0]
    shape = tuple(reversed([int(v) for v in dims]))
    Up = np.empty_like(U)
    for mu in range(4):
        axis = len(dims) - 1 - mu
        gf = np.roll(g.reshape(shape + (3, 3)), -1, axis=axis).reshape(V, 3, 3)
        Up[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(gf, -1, -2))
    return Up, g


def mass_field(dims: Sequence[int], sigma: float, seed: int) -> np.ndarray:
    """Per-site additive mass mu(x) ~ N(0, sigma^2) (sigma is the standard deviation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return sigma * rng.standard_normal(volume(dims))


def random_spinors(dims: Sequence[int], nrhs: int, seed: int) -> np.ndarray:
    """Gaussian complex spinor fields, complex128 [nrhs, V, 4, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    V = volume(dims)
    a = rng.standard_normal((nrhs, V, 4, 3, 2))
    return a[..., 0] + 1j * a[..., 1]


def random_real_fields(dims: Sequence[int], nrhs: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((nrhs, volume(dims)))


BATCH_LATTICES = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 48)]


def batch_config(seed: int = 3000, lattices=BATCH_LATTICES) -> list[dict]:
    """The uneven batch: per lattice kappa ~ U[0.10, 0.12], eps ~ U[0.2, 0.4],
    s uniform in {64, 128, 256, 512}, link seed 1100 + i, all from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i, dims in enumerate(lattices):
        kappa = float(rng.uniform(0.10, 0.12))
        eps = float(rng.uniform(0.2, 0.4))
        s = int(rng.choice([64, 128, 256, 512]))
        out.append({"dims": tuple(dims), "kappa": kappa, "eps": eps, "s": s, "link_seed": 1100 + i})
    return out


# ------------------------------------------------------------ general sparse matrices
# Stand-ins for the general sparse matrices of Section 2.1 (the paper fixes none): a
# periodic grid whose rows are renumbered by a seeded permutation (so the natural order
# carries no lattice structure), and random graphs.  CSR arrays: row_ptr int32[n+1],
# col_idx int32[nnz] (sorted within each row, duplicates merged), values float64[nnz].

def csr_from_entries(n: int, rows, cols, vals=None):
    """CSR of the entries (rows, cols, vals); repeated (row, col) pairs are merged (values summed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * n + cols
    uniq, inv = np.unique(key, return_inverse=True)
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    if vals is None:
        return row_ptr, c
    v = np.zeros(len(uniq), dtype=np.float64)
    np.add.at(v, inv, np.asarray(vals, dtype=np.float64))
    return row_ptr, c, v


def _weighted_laplacian(n: int, ei, ej, w, shift: float):
    """A = D - W + shift I for the undirected weighted edges (ei, ej, w): symmetric positive definite."""
    rows = np.concatenate([ei, ej, np.arange(n), ei, ej])
    cols = np.concatenate([ej, ei, np.arange(n), ei, ej])
    vals = np.concatenate([-w, -w, np.full(n, shift), w, w])
    return csr_from_entries(n, rows, cols, vals)


def grid_matrix(dims: Sequence[int], seed: int, shift: float = 0.1, renumber: bool = True):
    """Weighted graph Laplacian plus shift of the periodic grid dims (nearest neighbours), edge
    weights U[0.5, 1.5] and the row renumbering permutation from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = volume(dims)
    idx = np.arange(n)
    coords = []
    r = idx.copy()
    for L in dims:
        coords.append(r % L)
        r //= L
    ei, ej = [], []
    stride = 1
    for j, L in enumerate(dims):
        if L > 1:
            fw = idx + np.where(coords[j] == L - 1, -(L - 1) * stride, stride)
            ei.append(idx)
            ej.append(fw)
        stride *= L
    ei = np.concatenate(ei)
    ej = np.concatenate(ej)
    keep = ei != ej
    ei, ej = ei[keep], ej[keep]
    w = rng.uniform(0.5, 1.5, len(ei))
    if renumber:
        perm = rng.permutation(n)
        ei, ej = perm[ei], perm[ej]
    return _weighted_laplacian(n, ei, ej, w, shift)


def random_graph_matrix(n: int, degree: int, seed: int, shift: float = 0.1):
    """Weighted graph Laplacian plus shift of a random graph: every row draws `degree` partners
    uniformly (self pairs dropped), weights U[0.5, 1.5], all from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ei = np.repeat(np.arange(n), degree)
    ej = rng.integers(0, n, n * degree)
    keep = ei != ej
    ei, ej = ei[keep], ej[keep]
    w = rng.uniform(0.5, 1.5, len(ei))
    return _weighted_laplacian(n, ei, ej, w, shift)


def random_pattern(n: int, degree: int, seed: int, symmetric: bool = True, diagonal: bool = True):
    """A sparsity pattern only: `degree` uniform partners per row from PCG64(seed) (self pairs
    dropped), mirrored when symmetric, the diagonal stored when asked."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ei = np.repeat(np.arange(n), degree)
    ej = rng.integers(0, n, n * degree)
    keep = ei != ej
    ei, ej = ei[keep], ej[keep]
    if symmetric:
        ei, ej = np.concatenate([ei, ej]), np.concatenate([ej, ei])
    if diagonal:
        ei, ej = np.concatenate([ei, np.arange(n)]), np.concatenate([ej, np.arange(n)])
    return csr_from_entries(n, ei, ej)
