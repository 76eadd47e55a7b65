"""The C-ABI library builds, loads and exports every symbol include/hprobe.h declares;
host-only entry points agree with the oracle.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import permutation as P
from oracle import probing as Pr


@pytest.fixture(scope="module")
def lib():
    from paper_1302_4018_gb300 import build as b

    b.build()
    from paper_1302_4018_gb300 import hprobe

    return hprobe


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hprobe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hp_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    handle = lib.lib()
    for n in names:
        assert hasattr(handle, n)
    assert sorted(lib.EXPORTED) == names


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (12, 12, 12, 12), (24, 24, 24, 48), (32, 32, 32, 64), (5, 4),
                                  (3, 3, 3, 3), (6, 10), (1, 1, 1, 1), (7,), (2, 2, 2, 2, 2, 2, 2, 2)])
def test_basis_info_matches_oracle(lib, dims):
    info = lib.basis_info(dims)
    b = Pr.LatticeBasis(dims)
    assert info["volume"] == b.V and info["n_vectors"] == b.n_vectors
    assert info["K"] == b.K and info["Q"] == b.Q and info["period"] == b.P
    assert info["R"] == (b.Q // 3 if (b.Q > 1 and b.order.odd.equal) else 0)


@pytest.mark.parametrize("period", [2, 4, 6, 8, 54, 162, 1458, 4374])
def test_phase_table_bit_exact_with_oracle(lib, period):
    ours = lib.phase_values(period)
    ref = Pr.phase_values(period)
    assert np.array_equal(ours, ref), np.argwhere(ours != ref)[:5]


def test_errors_without_gpu_are_reported(lib):
    h = ctypes.c_void_p()
    st = lib.lib().hp_ctx_create(0, None, ctypes.byref(h))
    if st == lib.HP_OK:
        lib.lib().hp_ctx_destroy(h)
        pytest.skip("a GPU is present")
    assert st in (lib.HP_ECUDA, lib.HP_EINVAL)
    assert len(lib.lib().hp_last_error()) > 0


def test_host_argument_validation(lib):
    b = lib.Basis()
    lat = lib.make_lattice([4, 0])
    assert lib.lib().hp_basis_info(ctypes.byref(lat), ctypes.byref(b)) == lib.HP_EINVAL
    lat = lib.make_lattice([1 << 16, 1 << 16])
    assert lib.lib().hp_basis_info(ctypes.byref(lat), ctypes.byref(b)) == lib.HP_EINVAL
    lat = lib.Lattice()
    lat.ndim = 9
    assert lib.lib().hp_basis_info(ctypes.byref(lat), ctypes.byref(b)) == lib.HP_EINVAL
    assert lib.lib().hp_phase_values(0, None) == lib.HP_EINVAL


def test_no_oracle_in_product_path():
    pkg = os.path.join(ROOT, "paper_1302_4018_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_noalloc_rejects_clover_without_gpu():
    """The allocation-free stencil is plain Wilson: a clover coefficient is an argument error,
    reported before any device work."""
    from paper_1302_4018_gb300 import hprobe

    lib = hprobe.lib()
    op = hprobe.Context.make_operator(hprobe.OP_WILSON, 0.0, 0.12, np.zeros(72 * 16), None, csw=1.0)
    lat = hprobe.make_lattice((2, 2, 2, 2))
    buf = np.zeros(24 * 16)
    st = lib.hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(lat), 1, buf.ctypes.data, buf.ctypes.data,
                                       None)
    assert st == hprobe.HP_EINVAL
    assert "csw" in lib.hp_last_error().decode()


def test_noalloc_rejects_host_buffers_without_gpu():
    """Links, input and output of the allocation-free stencil must be device memory of the current
    device: host arrays are an argument error, found before any launch."""
    from paper_1302_4018_gb300 import hprobe

    lib = hprobe.lib()
    links = np.zeros(72 * 16)
    op = hprobe.Context.make_operator(hprobe.OP_WILSON, 0.0, 0.12, links, None)
    lat = hprobe.make_lattice((2, 2, 2, 2))
    a, b = np.zeros(24 * 16), np.zeros(24 * 16)
    st = lib.hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(lat), 1, a.ctypes.data, b.ctypes.data, None)
    assert st == hprobe.HP_EINVAL
    assert "device memory" in lib.hp_last_error().decode()
    st = lib.hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(lat), 1 << 31, a.ctypes.data, b.ctypes.data,
                                       None)
    assert st == hprobe.HP_EINVAL
    assert "2^31" in lib.hp_last_error().decode()


def test_sparse_entry_points_reject_a_missing_context_without_gpu():
    """The general-sparse calls validate their context and arguments before any device work."""
    from paper_1302_4018_gb300 import hprobe

    lib = hprobe.lib()
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    paths = np.zeros(4, dtype=np.int32)
    rad = np.array([1], dtype=np.int32)
    nl = ctypes.c_int32()
    assert lib.hp_sparse_coloring(None, 2, rp.ctypes.data, ci.ctypes.data, 2, paths.ctypes.data, rad.ctypes.data,
                                  ctypes.byref(nl)) == hprobe.HP_EINVAL
    perm = np.zeros(2, dtype=np.int32)
    nb = ctypes.c_int64()
    assert lib.hp_sparse_ordering(None, 2, paths.ctypes.data, 1, perm.ctypes.data, None, 0,
                                  ctypes.byref(nb)) == hprobe.HP_EINVAL
    per = ctypes.c_int32()
    assert lib.hp_sparse_probe_vectors(None, 2, paths.ctypes.data, rad.ctypes.data, 1, 0, 1, 0, None,
                                       ctypes.byref(per)) == hprobe.HP_EINVAL
    opts = hprobe.Context.make_opts("fp64")
    T = np.zeros(2, dtype=np.complex128)
    vals = np.ones(2)
    assert lib.hp_trace_inv_sparse(None, 2, rp.ctypes.data, ci.ctypes.data, vals.ctypes.data, paths.ctypes.data,
                                   rad.ctypes.data, 1, 1, 1e-10, ctypes.byref(opts), None, T.ctypes.data,
                                   None) == hprobe.HP_EINVAL
    assert "context" in lib.hp_last_error().decode().lower()


def test_eigensolvers_reject_a_missing_context_without_gpu():
    from paper_1302_4018_gb300 import hprobe

    lib = hprobe.lib()
    lat = hprobe.make_lattice((4, 4, 4, 4))
    op = hprobe.Operator(kind=hprobe.OP_WILSON, kappa=0.12)
    ev = np.zeros(8)
    for fn in (lib.hp_wilson_eigs, lib.hp_laplacian_eigs):
        assert fn(None, ctypes.byref(op), ctypes.byref(lat), 2, 1e-10, 0, ev.ctypes.data, ev.ctypes.data,
                  None) == hprobe.HP_EINVAL
    assert lib.hp_wilson_svd(None, ctypes.byref(op), ctypes.byref(lat), 2, 1e-10, 0, ev.ctypes.data, ev.ctypes.data,
                             ev.ctypes.data, None) == hprobe.HP_EINVAL
