"""hp_operator_apply_noalloc: the Wilson stencil for callers that cannot let a library allocate
GPU memory (device memory reserved up front by another framework's allocator, or no
synchronising cudaMalloc / cudaFree allowed on their stream).  Its output must equal
hp_operator_apply's FP64 output, on calls in a row with different lattices and inputs (the
fixed scratch array is shared by all calls and keeps the previous call's contents), and the
oracle's Wilson operator.  Collected last so that a run stopping at the first failure has run
every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as O
from paper_1302_4018_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hp():
    from paper_1302_4018_gb300 import build as b

    b.build()
    from paper_1302_4018_gb300 import hprobe

    return hprobe


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_noalloc_apply_matches_operator_apply_on_two_calls(hp):
    assert torch.cuda.is_available()
    ctx = hp.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    # the last case has no mass field and three dimensions (the fourth padded with L = 1, where the
    # forward and backward neighbours of a site are the site itself)
    cases = [((12, 12, 12, 12), 0.4, 7, 3, 0.12, True), ((4, 6, 2, 8), 0.3, 8, 2, 0.11, True),
             ((6, 4, 3), 0.35, 9, 2, 0.13, False)]
    for dims, eps, seed, nrhs, kappa, with_mf in cases:
        U = synth.gauge_links(dims, eps, seed, device="cuda:0")
        links = _dev(U.view(np.float64).reshape(-1))
        mf_h = synth.mass_field(dims, 0.01, seed + 1) if with_mf else None
        mf = _dev(mf_h) if with_mf else None
        psi_h = synth.random_spinors(dims, nrhs, seed + 2)
        psi = _dev(psi_h.view(np.float64).reshape(-1))
        op = ctx.make_operator(hp.OP_WILSON, 0.02, kappa, links, mf)
        ref = torch.empty_like(psi)
        ctx.operator_apply(op, dims, nrhs, "fp64", psi, ref)
        out = torch.full_like(psi, float("nan"))
        st = hp.lib().hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(hp.make_lattice(dims)), nrhs,
                                               psi.data_ptr(), out.data_ptr(), ctypes.c_void_p(stream))
        assert st == hp.HP_OK, hp.lib().hp_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-13, (dims, err)
        # and against the oracle's operator (explicit gammas, full 3x3 products), site by site
        got = out.cpu().numpy().view(np.complex128).reshape(nrhs, -1, 4, 3)
        d4 = tuple(dims) + (1,) * (4 - len(dims))
        for r in range(nrhs):
            want = O.wilson_apply(psi_h[r], U, d4, kappa, mass=0.02, mass_field=mf_h)
            site_err = np.abs(got[r] - want).max(axis=(1, 2)) / np.abs(want).max()
            assert site_err.max() <= 1e-13, (dims, r, site_err.max())
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(hp):
    ctx = hp.Context(0)
    dims = (16, 16, 16, 16)
    x = torch.zeros(24, dtype=torch.float64, device="cuda:0")
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.1, x, None)
    st = hp.lib().hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(hp.make_lattice(dims)), 1,
                                           x.data_ptr(), x.data_ptr(), None)
    assert st == hp.HP_EINVAL
    assert b"exceed the fixed scratch" in hp.lib().hp_last_error()
    # an in-place call (output = input) would read neighbours already overwritten: rejected
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 5, device="cuda:0")
    links = _dev(U.view(np.float64).reshape(-1))
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.1, links, None)
    psi = _dev(synth.random_spinors(dims, 1, 6).view(np.float64).reshape(-1))
    st = hp.lib().hp_operator_apply_noalloc(ctypes.byref(op), ctypes.byref(hp.make_lattice(dims)), 1,
                                           psi.data_ptr(), psi.data_ptr(), None)
    assert st == hp.HP_EINVAL
    assert b"overlaps" in hp.lib().hp_last_error()
    ctx.close()
