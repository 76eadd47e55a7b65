"""Python binding of libhprobe.so (include/hprobe.h): argument marshalling only.

Every computation happens in the CUDA library; this module only converts
Python / torch arguments to the C structs and pointers of the ABI and turns
error codes into exceptions.  Importing it loads the library and raises
``HProbeLibraryMissing`` when it is absent: there is no fallback path.

Device buffers are torch CUDA tensors (their ``data_ptr``); host buffers are
numpy arrays.  Names follow the C ABI: ``permutation``, ``probe_vectors``,
``trace_inv``, ``trace_inv_grad``, ``trace_inv_batch``, ``operator_apply``,
``dslash_bench``.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhprobe.so")


class HProbeLibraryMissing(RuntimeError):
    pass


class HProbeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("hprobe status %d: %s" % (status, msg))
        self.status = status


HP_OK, HP_EINVAL, HP_EUNSUPPORTED, HP_ENOMEM, HP_ECUDA, HP_ENOCONV, HP_ETIMEOUT = range(7)
OP_LAPLACIAN, OP_WILSON = 0, 1
PROBE_KINDS = {"hp": 0, "natural": 1, "z2": 2}
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}

EXPORTED = ["hp_ctx_create", "hp_ctx_destroy", "hp_last_error", "hp_ctx_synchronize", "hp_basis_info",
            "hp_phase_values",
            "hp_permutation", "hp_probe_vectors", "hp_trace_inv", "hp_trace_inv_grad", "hp_trace_inv_batch",
            "hp_operator_apply", "hp_dslash_bench", "hp_profile_enable", "hp_profile_report",
            "hp_launch_count", "hp_operator_apply_noalloc", "hp_probe_sequence", "hp_trace_inv_bounds",
            "hp_sparse_coloring", "hp_sparse_ordering", "hp_sparse_probe_vectors", "hp_trace_inv_sparse", "hp_trace_inv_deflated",
            "hp_trace_inv_solutions", "hp_trace_prefix", "hp_schur_apply", "hp_laplacian_eigs", "hp_wilson_eigs", "hp_wilson_svd",
            "hp_trace_inv_deflated_svd"]


class Lattice(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dims", C.c_int64 * 8)]


class Basis(C.Structure):
    _fields_ = [("volume", C.c_int64), ("n_vectors", C.c_int64), ("K", C.c_int32), ("Q", C.c_int32),
                ("R", C.c_int32), ("period", C.c_int32), ("kmax", C.c_int32), ("ks", C.c_int32 * 8),
                ("ps", C.c_int32 * 8)]


class Operator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mass", C.c_double), ("kappa", C.c_double),
                ("links", C.c_void_p), ("mass_field", C.c_void_p), ("csw", C.c_double)]


class SolverOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rhs_block", C.c_int32), ("maxiter", C.c_int32),
                ("dilution", C.c_int32), ("z0_seed", C.c_uint64), ("first", C.c_int64), ("delta", C.c_double),
                ("check_every", C.c_int32), ("use_graph", C.c_int32), ("block_threads", C.c_int32),
                ("rhs_per_thread", C.c_int32), ("even_odd", C.c_int32), ("probe_kind", C.c_int32),
                ("eo_kernel", C.c_int32), ("reserved", C.c_int32 * 1)]


class SolveStats(C.Structure):
    _fields_ = [("rhs_solved", C.c_int64), ("iterations_total", C.c_int64), ("iterations_max", C.c_int32),
                ("iterations_min", C.c_int32), ("reliable_updates", C.c_int64), ("sloppy_matvecs", C.c_int64),
                ("fp64_matvecs", C.c_int64), ("max_true_residual", C.c_double), ("seconds", C.c_double),
                ("n_unconverged", C.c_int32), ("group_updates", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise HProbeLibraryMissing("libhprobe.so not built (run __graft_entry__.build()): %s" % path)
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "hp_ctx_create": (C.c_int, [C.c_int, P, C.POINTER(P)]),
        "hp_ctx_destroy": (None, [P]),
        "hp_last_error": (C.c_char_p, []),
        "hp_ctx_synchronize": (C.c_int, [P]),
        "hp_basis_info": (C.c_int, [C.POINTER(Lattice), C.POINTER(Basis)]),
        "hp_phase_values": (C.c_int, [I32, P]),
        "hp_permutation": (C.c_int, [P, C.POINTER(Lattice), P]),
        "hp_probe_vectors": (C.c_int, [P, C.POINTER(Lattice), I64, I64, C.c_uint64, P, C.POINTER(I32)]),
        "hp_probe_sequence": (C.c_int, [P, C.POINTER(Lattice), I32, I64, I64, C.c_uint64, P, C.POINTER(I32)]),
        "hp_trace_inv": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, D, C.POINTER(SolverOpts),
                                   P, P, C.POINTER(SolveStats)]),
        "hp_trace_inv_bounds": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, D, D,
                                          C.POINTER(SolverOpts), P, P, P, C.POINTER(SolveStats)]),
        "hp_trace_inv_grad": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, D,
                                        C.POINTER(SolverOpts), P, P, P, C.POINTER(SolveStats)]),
        "hp_trace_inv_batch": (C.c_int, [P, I32, P, P, P, D, C.POINTER(SolverOpts), P, C.POINTER(SolveStats)]),
        "hp_operator_apply": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, I32, P, P]),
        "hp_dslash_bench": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, I32, I32,
                                      C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
        "hp_profile_enable": (C.c_int, [P, I32]),
        "hp_launch_count": (C.c_int, [P, C.POINTER(I64)]),
        "hp_operator_apply_noalloc": (C.c_int, [C.POINTER(Operator), C.POINTER(Lattice), I64, P, P, P]),
        "hp_profile_report": (C.c_int, [P, C.c_char_p, I64]),
        "hp_sparse_coloring": (C.c_int, [P, I32, P, P, I32, P, P, C.POINTER(I32)]),
        "hp_sparse_ordering": (C.c_int, [P, I32, P, I32, P, P, I64, C.POINTER(I64)]),
        "hp_sparse_probe_vectors": (C.c_int, [P, I32, P, P, I32, I64, I64, C.c_uint64, P, C.POINTER(I32)]),
        "hp_trace_inv_sparse": (C.c_int, [P, I32, P, P, P, P, P, I32, I64, D, C.POINTER(SolverOpts), P, P,
                                          C.POINTER(SolveStats)]),
        "hp_trace_inv_deflated": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, P, P, I64, D,
                                            C.POINTER(SolverOpts), P, P, C.POINTER(SolveStats)]),
        "hp_trace_inv_solutions": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, D,
                                             C.POINTER(SolverOpts), I64, P, P, P, C.POINTER(SolveStats)]),
        "hp_trace_prefix": (C.c_int, [P, I64, P, P]),
        "hp_schur_apply": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I64, I32, I32, P, P]),
        "hp_laplacian_eigs": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, D, I32, P, P, P]),
        "hp_wilson_eigs": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, D, I32, P, P, P]),
        "hp_wilson_svd": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, D, I32, P, P, P, P]),
        "hp_trace_inv_deflated_svd": (C.c_int, [P, C.POINTER(Operator), C.POINTER(Lattice), I32, P, P, P, I64, D,
                                                C.POINTER(SolverOpts), P, P, C.POINTER(SolveStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(status: int):
    if status != HP_OK:
        raise HProbeError(status, lib().hp_last_error().decode())


def make_lattice(dims: Sequence[int]) -> Lattice:
    lat = Lattice()
    lat.ndim = len(dims)
    for j, v in enumerate(dims):
        lat.dims[j] = int(v)
    return lat


def basis_info(dims: Sequence[int]) -> dict:
    b = Basis()
    _check(lib().hp_basis_info(C.byref(make_lattice(dims)), C.byref(b)))
    return {"volume": b.volume, "n_vectors": b.n_vectors, "K": b.K, "Q": b.Q, "R": b.R, "period": b.period,
            "kmax": b.kmax, "ks": list(b.ks)[:len(dims)], "ps": list(b.ps)[:len(dims)]}


def phase_values(period: int) -> np.ndarray:
    """(cos, sin) table of 2 pi k / P from the library (host code)."""
    out = np.zeros((period, 2), dtype=np.float64)
    _check(lib().hp_phase_values(int(period), out.ctypes.data))
    return out


def _ptr(x) -> Optional[int]:
    """data pointer of a torch tensor or numpy array (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


class Context:
    """hp_ctx on one CUDA device.

    ``stream`` is a cudaStream_t handle (int); by default the context runs on
    torch's current stream of that device, so its work is ordered with the
    torch operations that produce its inputs and consume its outputs.
    """

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            try:
                import torch

                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                pass
        h = C.c_void_p()
        _check(lib().hp_ctx_create(int(device), C.c_void_p(stream) if stream else None, C.byref(h)))
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().hp_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        _check(lib().hp_ctx_synchronize(self._h))

    # ---------------------------------------------------------------- integer path
    def permutation(self, dims: Sequence[int], out):
        """loc into ``out`` (device int32/uint32 tensor of V entries)."""
        _check(lib().hp_permutation(self._h, C.byref(make_lattice(dims)), _ptr(out)))
        return out

    def probe_vectors(self, dims: Sequence[int], first: int, count: int, z0_seed: int, out, kind=0) -> int:
        """uint16 phases into ``out`` (device int16/uint16 tensor of count*V); returns the period.
        kind: the probing sequence (0 / "hp", 1 / "natural", 2 / "z2")."""
        per = C.c_int32()
        k = PROBE_KINDS[kind] if isinstance(kind, str) else int(kind)
        if k == 0:
            _check(lib().hp_probe_vectors(self._h, C.byref(make_lattice(dims)), int(first), int(count),
                                          C.c_uint64(z0_seed), _ptr(out), C.byref(per)))
        else:
            _check(lib().hp_probe_sequence(self._h, C.byref(make_lattice(dims)), k, int(first), int(count),
                                           C.c_uint64(z0_seed), _ptr(out), C.byref(per)))
        return per.value

    # ---------------------------------------------------------------- operators
    @staticmethod
    def make_operator(kind: int, mass: float = 0.0, kappa: float = 0.0, links=None, mass_field=None,
                      csw: float = 0.0) -> Operator:
        """The operator struct; it keeps the link and mass-field arrays alive (the C struct only
        holds their addresses).  csw != 0 adds the clover term (Wilson only)."""
        op = Operator()
        op.kind = kind
        op.mass = float(mass)
        op.kappa = float(kappa)
        op.links = _ptr(links)
        op.mass_field = _ptr(mass_field)
        op.csw = float(csw)
        op._keep = (links, mass_field)
        return op

    @staticmethod
    def make_opts(precision="fp64", rhs_block=0, maxiter=0, z0_seed=0, first=0, delta=0.0, check_every=0,
                  use_graph=0, block_threads=0, dilution=0, rhs_per_thread=0, even_odd=0,
                  probe_kind=0, eo_kernel=0) -> SolverOpts:
        """probe_kind: 0 / "hp" hierarchical probing, 1 / "natural" Hadamard vectors in natural
        order, 2 / "z2" Z_2 noise vectors (seeded by z0_seed).  eo_kernel: the even-odd V / T step
        kernels (1 one right-hand side per thread, 3 / 4 pair kernels, 0 autotuned)."""
        o = SolverOpts()
        o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        o.rhs_block = rhs_block
        o.maxiter = maxiter
        o.dilution = dilution
        o.z0_seed = z0_seed
        o.first = first
        o.delta = delta
        o.check_every = check_every
        o.use_graph = use_graph
        o.block_threads = block_threads
        o.rhs_per_thread = rhs_per_thread
        o.even_odd = even_odd
        o.probe_kind = PROBE_KINDS[probe_kind] if isinstance(probe_kind, str) else int(probe_kind)
        o.eo_kernel = eo_kernel
        return o

    def operator_apply(self, op: Operator, dims, nrhs: int, precision, inp, out):
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        _check(lib().hp_operator_apply(self._h, C.byref(op), C.byref(make_lattice(dims)), int(nrhs), prec,
                                       _ptr(inp), _ptr(out)))
        return out

    def schur_apply(self, op: Operator, dims, nrhs: int, precision, inp, out, eo_kernel: int = 0):
        """out = S inp on the odd sites (the even-odd iteration's Schur complement), canonical layout;
        eo_kernel as in make_opts (0: the autotuner's choice)."""
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        _check(lib().hp_schur_apply(self._h, C.byref(op), C.byref(make_lattice(dims)), int(nrhs), prec,
                                    int(eo_kernel), _ptr(inp), _ptr(out)))
        return out

    def laplacian_eigs(self, op: Operator, dims, k: int, tol: float = 1e-10, max_sweeps: int = 0, evecs=None):
        """The k lowest eigenpairs of the Laplacian operator: (evals [k], evecs, resid [k]); evecs is
        written into the given float64 array / tensor of k * V values (host array by default)."""
        V = int(np.prod(dims))
        if evecs is None:
            evecs = np.zeros((k, V))
        evals = np.zeros(k)
        resid = np.zeros(k)
        _check(lib().hp_laplacian_eigs(self._h, C.byref(op), C.byref(make_lattice(dims)), int(k), float(tol),
                                       int(max_sweeps), _ptr(evecs), _ptr(evals), _ptr(resid)))
        return evals, evecs, resid

    def wilson_eigs(self, op: Operator, dims, k: int, tol: float = 1e-10, max_sweeps: int = 0, evecs=None):
        """The k eigenpairs of gamma_5 D (Hermitian) with the smallest |lambda|: (evals [k] signed,
        ordered by |lambda|, evecs complex [k, V, 4, 3] (host array by default, or the given
        complex128 array / tensor), resid [k])."""
        V = int(np.prod(dims))
        if evecs is None:
            evecs = np.zeros((k, V, 4, 3), dtype=np.complex128)
        evals = np.zeros(k)
        resid = np.zeros(k)
        _check(lib().hp_wilson_eigs(self._h, C.byref(op), C.byref(make_lattice(dims)), int(k), float(tol),
                                    int(max_sweeps), _ptr(evecs), _ptr(evals), _ptr(resid)))
        return evals, evecs, resid

    def wilson_svd(self, op: Operator, dims, k: int, tol: float = 1e-10, max_sweeps: int = 0, right=None, left=None,
                   check: bool = True):
        """The k smallest singular triplets D v = sigma u: (sigma [k] ascending, right, left complex
        [k, V, 4, 3] (host arrays by default, or the given complex128 arrays / tensors), resid [k]).
        check=False returns the last Rayleigh-Ritz triplets when max_sweeps ends the iteration before
        tol (HP_ENOCONV): D v_j = sigma_j u_j still holds, so deflation with them stays exact."""
        V = int(np.prod(dims))
        if right is None:
            right = np.zeros((k, V, 4, 3), dtype=np.complex128)
        if left is None:
            left = np.zeros((k, V, 4, 3), dtype=np.complex128)
        sigma = np.zeros(k)
        resid = np.zeros(k)
        st = lib().hp_wilson_svd(self._h, C.byref(op), C.byref(make_lattice(dims)), int(k), float(tol),
                                 int(max_sweeps), _ptr(right), _ptr(left), _ptr(sigma), _ptr(resid))
        if check or st != HP_ENOCONV:
            _check(st)
        return sigma, right, left, resid

    def trace_inv_deflated_svd(self, op: Operator, dims, right, left, sigma, s_max: int, tol: float,
                               opts: SolverOpts, q_inout=None):
        """Wilson deflation with singular triplets D v_j = sigma_j u_j: right, left complex128
        [k, V, 4, 3] (host arrays or device tensors), sigma float64 [k] (host).  Returns (T, q, stats)."""
        sg = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
        k = int(sg.shape[0])
        V = int(np.prod(dims))
        for a in (right, left):
            if not (str(a.dtype).endswith("complex128") and int(np.prod(a.shape)) == 12 * k * V):
                raise ValueError("singular vectors must be complex of %d x %d values" % (k, 12 * V))
        T = np.zeros(s_max, dtype=np.complex128)
        st = SolveStats()
        if q_inout is not None:
            assert q_inout.dtype == np.complex128 and q_inout.shape == (s_max,)
        _check(lib().hp_trace_inv_deflated_svd(self._h, C.byref(op), C.byref(make_lattice(dims)), k, _ptr(right),
                                               _ptr(left), _ptr(sg), int(s_max), float(tol), C.byref(opts),
                                               _ptr(q_inout), _ptr(T), C.byref(st)))
        return T, q_inout, st.as_dict()

    def trace_inv(self, op: Operator, dims, s_max: int, tol: float, opts: SolverOpts, q_inout=None):
        """Returns (T [s_max] complex, q [s_max] complex or None, stats dict).  ``q_inout``: host
        complex128 array of s_max (entries < opts.first are inputs)."""
        T = np.zeros(s_max, dtype=np.complex128)
        st = SolveStats()
        if q_inout is not None:
            assert q_inout.dtype == np.complex128 and q_inout.shape == (s_max,)
        _check(lib().hp_trace_inv(self._h, C.byref(op), C.byref(make_lattice(dims)), int(s_max), float(tol),
                                  C.byref(opts), _ptr(q_inout), _ptr(T), C.byref(st)))
        return T, q_inout, st.as_dict()

    def trace_inv_solutions(self, op: Operator, dims, s_max: int, tol: float, opts: SolverOpts, x_out,
                            q_inout=None):
        """hp_trace_inv that also writes the solutions of the first right-hand sides into x_out
        (device float64 tensor of n_keep * V * 24 values, canonical layout).  Returns as trace_inv."""
        V = int(np.prod(dims))
        n_keep = x_out.numel() // (24 * V)
        assert x_out.numel() == n_keep * 24 * V
        T = np.zeros(s_max, dtype=np.complex128)
        st = SolveStats()
        if q_inout is not None:
            assert q_inout.dtype == np.complex128 and q_inout.shape == (s_max,)
        _check(lib().hp_trace_inv_solutions(self._h, C.byref(op), C.byref(make_lattice(dims)), int(s_max),
                                            float(tol), C.byref(opts), n_keep, _ptr(x_out), _ptr(q_inout), _ptr(T),
                                            C.byref(st)))
        return T, q_inout, st.as_dict()

    def trace_prefix(self, q):
        """T_s = (1/s) sum_{m<s} q_m for a host complex128 sequence q, by the library's prefix kernel."""
        q = np.ascontiguousarray(q, dtype=np.complex128)
        T = np.zeros(q.shape[0], dtype=np.complex128)
        _check(lib().hp_trace_prefix(self._h, int(q.shape[0]), _ptr(q), _ptr(T)))
        return T

    def trace_inv_bounds(self, op: Operator, dims, s_max: int, quad_tol: float, opts: SolverOpts,
                         lambda_min: float = 0.0):
        """Laplacian: (T [s_max] complex, T_lower [s_max], T_upper [s_max], stats dict) with every
        quadrature bracketed by Gauss / Gauss-Radau rules to quad_tol (relative)."""
        T = np.zeros(s_max, dtype=np.complex128)
        lo = np.zeros(s_max)
        hi = np.zeros(s_max)
        st = SolveStats()
        _check(lib().hp_trace_inv_bounds(self._h, C.byref(op), C.byref(make_lattice(dims)), int(s_max),
                                         float(quad_tol), float(lambda_min), C.byref(opts), _ptr(T), _ptr(lo),
                                         _ptr(hi), C.byref(st)))
        return T, lo, hi, st.as_dict()

    # ---------------------------------------------------------------- general sparse matrices
    @staticmethod
    def _csr(row_ptr, col_idx, values=None):
        """int32 row_ptr / col_idx (and float64 values): numpy arrays or torch tensors, either side."""
        for a, dt in ((row_ptr, "int32"), (col_idx, "int32"), (values, "float64")):
            if a is not None:
                assert str(a.dtype).endswith(dt), "CSR arrays must be %s" % dt
        return _ptr(row_ptr), _ptr(col_idx), _ptr(values)

    def sparse_coloring(self, row_ptr, col_idx, max_levels: int = 32, paths_out=None):
        """Hierarchical colouring of the pattern of an n x n CSR matrix (Algorithm 1).  Returns
        (paths [n_levels, n] int32, radices list): paths[l, i] = colour of row i at level l + 1.
        ``paths_out`` (optional, int32 [max_levels, n], host or device) receives all levels."""
        n = int(row_ptr.shape[0]) - 1
        if paths_out is None:
            paths_out = np.zeros((max_levels, max(n, 0)), dtype=np.int32)
        rad = np.zeros(max_levels, dtype=np.int32)
        nl = C.c_int32()
        rp, ci, _ = self._csr(row_ptr, col_idx)
        _check(lib().hp_sparse_coloring(self._h, n, rp, ci, int(max_levels), _ptr(paths_out), _ptr(rad),
                                        C.byref(nl)))
        return paths_out[:nl.value], [int(r) for r in rad[:nl.value]]

    def sparse_ordering(self, paths, perm_out=None, offsets_out=None):
        """Algorithm 1's perm and colorOffsets from colour paths [n_levels, n] (int32, host or device):
        (perm [n], offsets [n_blocks, 3] of (start, end, level)).  Without ``perm_out`` /
        ``offsets_out`` (host or device int32 arrays of n and of (2n - 1) x 3) host arrays are returned."""
        n_levels, n = int(paths.shape[0]), int(paths.shape[1])
        perm = np.zeros(n, dtype=np.int32) if perm_out is None else perm_out
        offs = np.zeros((max(2 * n - 1, 1), 3), dtype=np.int32) if offsets_out is None else offsets_out
        cnt = C.c_int64()
        _check(lib().hp_sparse_ordering(self._h, n, _ptr(paths), n_levels, _ptr(perm), _ptr(offs),
                                        int(offs.shape[0]), C.byref(cnt)))
        return perm, offs[:cnt.value]

    def sparse_probe_vectors(self, paths, radices: Sequence[int], first: int, count: int, z0_seed: int, out) -> int:
        """uint16 phases of the path probing vectors into ``out`` (device tensor of count*n);
        returns the period."""
        n = int(paths.shape[1])
        rad = np.ascontiguousarray(np.asarray(radices, dtype=np.int32))
        per = C.c_int32()
        _check(lib().hp_sparse_probe_vectors(self._h, n, _ptr(paths), _ptr(rad), len(rad), int(first), int(count),
                                             C.c_uint64(z0_seed), _ptr(out), C.byref(per)))
        return per.value

    def trace_inv_sparse(self, row_ptr, col_idx, values, paths, radices: Sequence[int], s_max: int, tol: float,
                         opts: SolverOpts, q_inout=None):
        """Tr(A^-1) estimates of a real symmetric positive definite CSR matrix with the path probing
        vectors (or opts.probe_kind's sequence): (T [s_max] complex, q, stats)."""
        n = int(row_ptr.shape[0]) - 1
        rad = np.ascontiguousarray(np.asarray(radices, dtype=np.int32))
        T = np.zeros(s_max, dtype=np.complex128)
        st = SolveStats()
        if q_inout is not None:
            assert q_inout.dtype == np.complex128 and q_inout.shape == (s_max,)
        rp, ci, va = self._csr(row_ptr, col_idx, values)
        _check(lib().hp_trace_inv_sparse(self._h, n, rp, ci, va, _ptr(paths), _ptr(rad), len(rad), int(s_max),
                                         float(tol), C.byref(opts), _ptr(q_inout), _ptr(T), C.byref(st)))
        return T, q_inout, st.as_dict()

    def trace_inv_deflated(self, op: Operator, dims, evecs, evals, s_max: int, tol: float, opts: SolverOpts,
                           q_inout=None):
        """Deflated probing.  Laplacian: evecs float64 [k, V] orthonormal eigenvectors; Wilson: evecs
        complex128 [k, V, 4, 3] eigenvectors of gamma_5 D (host array or device tensor); evals float64
        [k] (host) their eigenvalues.  Returns (T [s_max] complex, q (deflated), stats)."""
        ev = np.ascontiguousarray(np.asarray(evals, dtype=np.float64))
        k = int(ev.shape[0])
        V = int(np.prod(dims))
        wilson = op.kind == OP_WILSON
        n_el = int(np.prod(evecs.shape))
        dt = str(evecs.dtype)   # numpy or torch dtype name
        if (wilson and not (dt.endswith("complex128") and n_el == 12 * k * V)) or \
                (not wilson and not (dt.endswith("float64") and n_el == k * V)):
            raise ValueError("eigenvectors must be %s of %d x %d values" % ("complex" if wilson else "real", k,
                                                                            (12 if wilson else 1) * V))
        T = np.zeros(s_max, dtype=np.complex128)
        st = SolveStats()
        if q_inout is not None:
            assert q_inout.dtype == np.complex128 and q_inout.shape == (s_max,)
        _check(lib().hp_trace_inv_deflated(self._h, C.byref(op), C.byref(make_lattice(dims)), k, _ptr(evecs),
                                           _ptr(ev), int(s_max), float(tol), C.byref(opts), _ptr(q_inout), _ptr(T),
                                           C.byref(st)))
        return T, q_inout, st.as_dict()

    def trace_inv_grad(self, op: Operator, dims, s_max: int, tol: float, opts: SolverOpts, grad_out):
        """Returns (T, dT/dm, stats); dT/dmu(x) is written into ``grad_out`` (host float64 array or
        device float64 tensor of V)."""
        T = np.zeros(s_max, dtype=np.complex128)
        dm = C.c_double()
        st = SolveStats()
        _check(lib().hp_trace_inv_grad(self._h, C.byref(op), C.byref(make_lattice(dims)), int(s_max), float(tol),
                                       C.byref(opts), _ptr(T), _ptr(grad_out), C.byref(dm), C.byref(st)))
        return T, dm.value, st.as_dict()

    def trace_inv_batch(self, ops: Sequence[Operator], dims_list, s_max: Sequence[int], tol: float,
                        opts: SolverOpts):
        n = len(ops)
        ops_arr = (Operator * n)(*ops)
        lats = (Lattice * n)(*[make_lattice(d) for d in dims_list])
        smax = (C.c_int64 * n)(*[int(s) for s in s_max])
        outs = [np.zeros(int(s), dtype=np.complex128) for s in s_max]
        ptrs = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
        st = SolveStats()
        _check(lib().hp_trace_inv_batch(self._h, n, C.cast(ops_arr, C.c_void_p), C.cast(lats, C.c_void_p),
                                        C.cast(smax, C.c_void_p), float(tol), C.byref(opts),
                                        C.cast(ptrs, C.c_void_p), C.byref(st)))
        return outs, st.as_dict()

    def dslash_bench(self, op: Operator, dims, precision, nrhs: int, iters: int) -> dict:
        ms, by, fl = C.c_double(), C.c_double(), C.c_double()
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        _check(lib().hp_dslash_bench(self._h, C.byref(op), C.byref(make_lattice(dims)), prec, int(nrhs),
                                     int(iters), C.byref(ms), C.byref(by), C.byref(fl)))
        return {"ms": ms.value, "bytes": by.value, "flops": fl.value}

    # ---------------------------------------------------------------- profiling
    def launch_count(self) -> int:
        n = C.c_int64()
        _check(lib().hp_launch_count(self._h, C.byref(n)))
        return n.value

    def profile_enable(self, on: bool = True):
        _check(lib().hp_profile_enable(self._h, 1 if on else 0))

    def profile_report(self) -> dict:
        buf = C.create_string_buffer(1 << 16)
        _check(lib().hp_profile_report(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())
