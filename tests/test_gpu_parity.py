"""GPU path vs the CPU oracle, element by element, through the C ABI.

Integer work (permutation, probe phases) is compared bit for bit; stencils
within the rounding of their storage precision; trace estimates within
1e-9 relative (the tolerance the solver residual 1e-10 supports: the error
of q is |v^H D^-1 r| <= ||v|| ||D^-1|| ||r||, and ||D^-1|| < 10 here).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import operators as O
from oracle import permutation as P
from oracle import probing as Pr
from paper_1302_4018_gb300 import synth

pytestmark = pytest.mark.gpu

TRACE_RTOL = 1e-9


@pytest.fixture(scope="module")
def hp():
    from paper_1302_4018_gb300 import build as b

    b.build()
    from paper_1302_4018_gb300 import hprobe

    return hprobe


@pytest.fixture(scope="module")
def ctx(hp):
    assert torch.cuda.is_available()
    c = hp.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def links_dev(U):
    return dev(U.view(np.float64).reshape(-1))


# ------------------------------------------------------------------ integer path
@pytest.mark.parametrize("dims", [(4, 4), (2, 4, 8), (8, 8, 8, 8), (4, 4, 4, 8), (12, 12), (6, 6, 6, 6),
                                  (3, 3, 3, 3), (5, 4), (1, 4, 2, 8), (7,), (1024,), (2, 2, 2, 2, 2, 2, 2, 2),
                                  (12, 6, 4, 2), (10, 6, 2)])
def test_permutation_bit_exact(ctx, dims):
    V = int(np.prod(dims))
    loc = torch.empty(V, dtype=torch.int32, device="cuda:0")
    ctx.permutation(dims, loc)
    assert np.array_equal(loc.cpu().numpy(), np.array(P.hierarchical_loc(dims)))


@pytest.mark.parametrize("dims", [(32, 32, 32, 64), (24, 24, 24, 48), (16, 16, 16, 32), (12, 12, 12, 12)])
def test_permutation_full_size_sampled(ctx, dims):
    V = int(np.prod(dims))
    loc = torch.empty(V, dtype=torch.int32, device="cuda:0")
    ctx.permutation(dims, loc)
    l = loc.cpu().numpy()
    assert np.array_equal(np.sort(l), np.arange(V))           # bijection at full size
    rng = np.random.default_rng(1)
    sites = rng.integers(0, V, 400)
    assert np.array_equal(l[sites], np.array(P.hierarchical_loc(dims, sites)))


@pytest.mark.parametrize("dims,seed", [((4, 4), 0), ((2, 4, 8), 5), ((4, 4, 4, 4), 2003), ((6, 6, 6, 6), 9),
                                       ((3, 3, 3, 3), 1), ((12, 6), 0), ((5, 4), 3), ((6, 2, 6, 2), 4)])
def test_probe_phases_bit_exact(ctx, hp, dims, seed):
    V = int(np.prod(dims))
    nvec = hp.basis_info(dims)["n_vectors"]
    for first, count in [(0, min(nvec, 64)), (max(0, nvec - 7), min(7, nvec))]:
        out = torch.empty(count * V, dtype=torch.int16, device="cuda:0")
        per = ctx.probe_vectors(dims, first, count, seed, out)
        ref, Pref = Pr.probe_phases(dims, first, count, seed)
        got = out.cpu().numpy().astype(np.int64).reshape(count, V) & 0xFFFF
        assert per == Pref
        assert np.array_equal(got, ref)


def test_probe_phases_full_size_sampled(ctx):
    dims = (32, 32, 32, 64)
    V = int(np.prod(dims))
    for first in (0, 255, 1 << 20):
        out = torch.empty(V, dtype=torch.int16, device="cuda:0")
        ctx.probe_vectors(dims, first, 1, 2003, out)
        got = out.cpu().numpy().astype(np.int64) & 0xFFFF
        basis = Pr.LatticeBasis(dims)
        col = basis.column(first)
        sites = np.random.default_rng(first).integers(0, V, 300)
        locs = np.array(P.hierarchical_loc(dims, sites))
        z0 = np.array([1 - 2 * (Pr.splitmix64_output(2003, int(s)) >> 63) for s in sites])
        ref = (col[locs] + np.where(z0 < 0, 1, 0)) % 2
        assert np.array_equal(got[sites], ref)


def test_probe_errors(ctx, hp):
    out = torch.empty(64, dtype=torch.int16, device="cuda:0")
    with pytest.raises(hp.HProbeError) as e:
        ctx.probe_vectors((5, 4), 0, 5, 0, out)        # only 4 nested vectors exist
    assert e.value.status == hp.HP_EUNSUPPORTED
    with pytest.raises(hp.HProbeError) as e:
        ctx.probe_vectors((4, 4), 10, 7, 0, out)
    assert e.value.status == hp.HP_EINVAL


# ------------------------------------------------------------------ stencils
WILSON_TOL = {"fp64": 1e-13, "fp32": 3e-6, "fp16": 4e-3, "bf16": 3e-2}


APPLY_CASES = [(d, n) for d in [(4, 4, 4, 4), (3, 5, 4, 6), (1, 4, 1, 3)] for n in (1, 2, 3, 4, 5, 6)] + \
              [(d, 3) for d in [(2, 2, 2, 2), (8, 4, 6, 2)]]


@pytest.mark.parametrize("dims,nrhs", APPLY_CASES)   # nrhs 1..6 select every stencil variant
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_wilson_apply_parity(ctx, hp, dims, prec, nrhs):
    U = synth.gauge_links(dims, 0.4, 7)
    mf = synth.mass_field(dims, 0.01, 8)
    psi = synth.random_spinors(dims, nrhs, 9)
    op = ctx.make_operator(hp.OP_WILSON, 0.03, 0.12, links_dev(U), dev(mf))
    out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda:0")
    ctx.operator_apply(op, dims, nrhs, prec, dev(psi.view(np.float64).reshape(-1)), out)
    got = out.cpu().numpy().view(np.complex128).reshape(psi.shape)
    for r in range(nrhs):   # per site: the largest component error of any site, relative to max |ref|
        ref = O.wilson_apply(psi[r], U, dims, 0.12, 0.03, mf)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()
        assert err <= WILSON_TOL[prec], err


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 4, 6), (8, 8, 8, 8), (16, 1, 1, 1)])
def test_laplacian_apply_parity(ctx, hp, dims):
    x = synth.random_real_fields(dims, 2, 3)
    mf = synth.mass_field(dims, 0.1, 4)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.05, 0.0, None, dev(mf))
    out = torch.empty(x.size, dtype=torch.float64, device="cuda:0")
    ctx.operator_apply(op, dims, 2, "fp64", dev(x.reshape(-1)), out)
    got = out.cpu().numpy().reshape(x.shape)
    pad = list(dims) + [1] * (4 - len(dims))
    for r in range(2):
        ref = O.laplacian_apply(x[r], pad, 0.05, mf)
        assert np.allclose(got[r], ref, rtol=1e-14, atol=1e-13)


# ------------------------------------------------------------------ trace estimates
def rel(a, b):
    return np.abs(a - b) / np.abs(b)


@pytest.mark.parametrize("seed", [0, 1])
def test_laplacian_trace_config_8x8x8x8(ctx, hp, seed):
    """8^4 Laplacian, m = 0.05, s = 1..256, CG to 1e-12."""
    dims = (8, 8, 8, 8)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.05)
    T, _, st = ctx.trace_inv(op, dims, 256, 1e-12, ctx.make_opts("fp64", z0_seed=seed))
    q_ref = E.laplacian_quadratures(dims, 0.05, 0, 256, seed, method="dense")
    T_ref = E.trace_prefix(q_ref)
    assert np.all(rel(T, T_ref) <= TRACE_RTOL)
    assert st["max_true_residual"] <= 1e-12
    if seed == 0:   # h_0 = 1 is an eigenvector: CG converges in one step, T_1 = V / m
        assert abs(T[0] - 4096 / 0.05) <= 1e-9 * 4096 / 0.05


def test_laplacian_full_sequence_is_exact(ctx, hp):
    from pins import laplacian_trace_inverse

    dims = (4, 4, 4, 8)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.1)
    T, _, _ = ctx.trace_inv(op, dims, 512, 1e-13, ctx.make_opts("fp64", z0_seed=3))
    assert abs(T[-1].real - laplacian_trace_inverse(dims, 0.1)) <= 1e-10 * laplacian_trace_inverse(dims, 0.1)


def test_laplacian_complex_probes(ctx, hp):
    dims = (6, 6, 2, 3)
    V = 216
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.2)
    T, _, _ = ctx.trace_inv(op, dims, V, 1e-13, ctx.make_opts("fp64", z0_seed=5))
    T_ref = E.trace_prefix(E.laplacian_quadratures(dims, 0.2, 0, V, 5, method="dense"))
    assert np.all(np.abs(T - T_ref) <= 1e-9 * np.abs(T_ref).max())
    from pins import laplacian_trace_inverse
    assert abs(T[-1].real - laplacian_trace_inverse(dims, 0.2)) <= 1e-9 * laplacian_trace_inverse(dims, 0.2)


@pytest.mark.parametrize("prec,rpt", [("fp64", 0), ("fp64", 1), ("fp32", 1), ("fp32", 2), ("fp32", 4), ("fp32", 101),
                                      ("fp32", 104), ("fp16", 1), ("fp16", 2), ("fp16", 4), ("fp16", 101),
                                      ("fp16", 102), ("bf16", 0), ("bf16", 2), ("bf16", 104),
                                      ("fp16", 4101), ("fp32", 2002), ("fp16", 8121)])
def test_wilson_trace_parity(ctx, hp, prec, rpt):
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 1002)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.115, links_dev(U), None)
    s = 6
    T, _, st = ctx.trace_inv(op, dims, s, 1e-10, ctx.make_opts(prec, z0_seed=2002, rhs_block=24,
                                                                rhs_per_thread=rpt))
    T_ref = E.trace_prefix(E.wilson_quadratures(dims, U, 0.115, 0, s, 2002, method="dense"))
    assert np.all(rel(T, T_ref) <= TRACE_RTOL), (T, T_ref)
    assert st["max_true_residual"] <= 1e-10
    assert st["rhs_solved"] == 12 * s


def test_wilson_full_sequence_exact_and_gauge_invariant(ctx, hp):
    from pins import free_wilson_trace_inverse

    dims = (4, 4, 2, 4)
    V = 128
    Ufree = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    Ug, _ = synth.gauge_transform(Ufree, dims, 77)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(Ug), None)
    T, _, _ = ctx.trace_inv(op, dims, V, 1e-11, ctx.make_opts("fp32", z0_seed=5))
    exact = free_wilson_trace_inverse(dims, 0.12)
    assert abs(T[-1].real - exact) <= 1e-9 * exact
    assert np.max(np.abs(T.imag)) <= 1e-8 * np.max(np.abs(T.real))


def test_wilson_config2_16x16x16x16_properties(ctx, hp):
    """16^4, kappa 0.115, eps 0.3, BiCGStab 1e-10: FP64 and mixed agree, Im T = 0."""
    dims = (16, 16, 16, 16)
    U = synth.gauge_links(dims, 0.3, 1002, device="cuda:0")
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.115, links_dev(U), None)
    T64, _, s64 = ctx.trace_inv(op, dims, 2, 1e-10, ctx.make_opts("fp64", z0_seed=2002))
    T32, _, s32 = ctx.trace_inv(op, dims, 2, 1e-10, ctx.make_opts("fp32", z0_seed=2002))
    T16, _, _ = ctx.trace_inv(op, dims, 2, 1e-10, ctx.make_opts("fp16", z0_seed=2002))
    assert np.all(rel(T32, T64) <= TRACE_RTOL) and np.all(rel(T16, T64) <= TRACE_RTOL)
    assert np.max(np.abs(T64.imag)) <= 1e-9 * np.max(np.abs(T64.real))
    assert s64["max_true_residual"] <= 1e-10 and s32["max_true_residual"] <= 1e-10


def test_resume_gives_identical_prefix(ctx, hp):
    """Checkpoint/resume: q of an earlier run plus first = 2 reproduces one long run bit for bit."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 3)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.11, links_dev(U), None)
    q_full = np.zeros(5, dtype=np.complex128)
    T_full, _, _ = ctx.trace_inv(op, dims, 5, 1e-10, ctx.make_opts("fp64", z0_seed=9, rhs_block=12), q_inout=q_full)
    q_part = np.zeros(2, dtype=np.complex128)
    ctx.trace_inv(op, dims, 2, 1e-10, ctx.make_opts("fp64", z0_seed=9, rhs_block=12), q_inout=q_part)
    q2 = np.zeros(5, dtype=np.complex128)
    q2[:2] = q_part
    T_res, _, _ = ctx.trace_inv(op, dims, 5, 1e-10, ctx.make_opts("fp64", z0_seed=9, first=2, rhs_block=12),
                                q_inout=q2)
    assert np.array_equal(q2, q_full) and np.array_equal(T_res, T_full)


def test_nonconvergence_and_argument_errors(ctx, hp):
    dims = (4, 4, 4, 4)
    U = synth.gauge_links(dims, 0.3, 3)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(U), None)
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv(op, dims, 1, 1e-10, ctx.make_opts("fp64", maxiter=2))
    assert e.value.status == hp.HP_ENOCONV
    for bad in [dict(s_max=0), dict(tol=-1.0), dict(s_max=257)]:
        kw = dict(s_max=2, tol=1e-10)
        kw.update(bad)
        with pytest.raises(hp.HProbeError) as e:
            ctx.trace_inv(op, dims, kw["s_max"], kw["tol"], ctx.make_opts("fp64"))
        assert e.value.status == hp.HP_EINVAL
    op5 = ctx.make_operator(hp.OP_LAPLACIAN, 0.1)
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv(op5, (5, 4), 5, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EUNSUPPORTED


# ------------------------------------------------------------------ gradient
def test_laplacian_gradient(ctx, hp):
    from pins import laplacian_eigenvalues

    dims = (4, 4, 2, 2)
    V = 64
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.3)
    g = np.zeros(V)
    T, dTdm, _ = ctx.trace_inv_grad(op, dims, V, 1e-13, ctx.make_opts("fp64", z0_seed=2), g)
    lam = laplacian_eigenvalues(dims, 0.3)
    assert abs(dTdm + np.sum(1.0 / lam ** 2)) <= 1e-9 * np.sum(1.0 / lam ** 2)
    g_ref = E.laplacian_grad_mass_field(dims, 0.3, 5, 2, method="dense").real
    g5 = np.zeros(V)
    ctx.trace_inv_grad(op, dims, 5, 1e-13, ctx.make_opts("fp64", z0_seed=2), g5)
    assert np.allclose(g5, g_ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_wilson_gradient_vs_oracle(ctx, hp, prec):
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 21)
    mf = synth.mass_field(dims, 0.01, 5000)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(mf))
    V = 128
    g = torch.zeros(V, dtype=torch.float64, device="cuda:0")
    T, dTdm, _ = ctx.trace_inv_grad(op, dims, 3, 1e-12, ctx.make_opts(prec, z0_seed=7), g)
    g_ref = E.wilson_grad_mass_field(dims, U, 0.118, 3, 7, mass_field=mf, method="dense").real
    assert np.allclose(g.cpu().numpy(), g_ref, rtol=1e-7, atol=1e-9)
    assert abs(dTdm - g_ref.sum()) <= 1e-7 * abs(g_ref.sum())


def test_autograd_function_and_finite_differences(ctx, hp):
    from paper_1302_4018_gb300.autograd import trace_inv_estimate

    dims = (4, 4, 4, 4)
    V = 256
    U = synth.gauge_links(dims, 0.3, 5)
    mf = torch.tensor(synth.mass_field(dims, 0.01, 5000), device="cuda:0", requires_grad=True)
    opts = ctx.make_opts("fp64", z0_seed=3)
    links = links_dev(U)
    T = trace_inv_estimate(mf, ctx, dims, 2, 1e-13, opts, kind=hp.OP_WILSON, kappa=0.118, links=links)
    T.backward()
    grad = mf.grad.cpu().numpy()
    h = 1e-4
    base = mf.detach().clone()
    for site in (0, 77, 255):
        e = torch.zeros(V, dtype=torch.float64, device="cuda:0")
        e[site] = h
        tp = trace_inv_estimate(base + e, ctx, dims, 2, 1e-13, opts, kind=hp.OP_WILSON, kappa=0.118, links=links)
        tm = trace_inv_estimate(base - e, ctx, dims, 2, 1e-13, opts, kind=hp.OP_WILSON, kappa=0.118, links=links)
        fd = (tp - tm).item() / (2 * h)
        assert abs(fd - grad[site]) <= 1e-4 * max(1.0, abs(grad[site])), (site, fd, grad[site])
    # uniform direction: dT/dm = sum_x dT/dmu(x)
    one = torch.ones(V, dtype=torch.float64, device="cuda:0") * h
    tp = trace_inv_estimate(base + one, ctx, dims, 2, 1e-13, opts, kind=hp.OP_WILSON, kappa=0.118, links=links)
    tm = trace_inv_estimate(base - one, ctx, dims, 2, 1e-13, opts, kind=hp.OP_WILSON, kappa=0.118, links=links)
    assert abs((tp - tm).item() / (2 * h) - grad.sum()) <= 1e-5 * abs(grad.sum())


# ------------------------------------------------------------------ batching
def test_batch_matches_single_lattice_oracle(ctx, hp):
    cases = [((4, 4, 4, 4), 0.11, 0.2, 6), ((2, 2, 2, 4), 0.12, 0.4, 8), ((6, 2, 2, 2), 0.10, 0.3, 5)]
    ops, dims_list, smax, refs, keep = [], [], [], [], []
    for i, (dims, kappa, eps, s) in enumerate(cases):
        U = synth.gauge_links(dims, eps, 1100 + i)
        L = links_dev(U)
        keep.append(L)
        ops.append(ctx.make_operator(hp.OP_WILSON, 0.0, kappa, L, None))
        dims_list.append(dims)
        smax.append(s)
        refs.append(E.trace_prefix(E.wilson_quadratures(dims, U, kappa, 0, s, 31, method="dense")))
    for prec in ("fp64", "fp16"):
        outs, st = ctx.trace_inv_batch(ops, dims_list, smax, 1e-10, ctx.make_opts(prec, z0_seed=31, rhs_block=16,
                                                                                    use_graph=1))
        for T, T_ref in zip(outs, refs):
            assert np.all(rel(T, T_ref) <= TRACE_RTOL)
        assert st["rhs_solved"] == 12 * sum(smax)


# ------------------------------------------------------------------ uneven batch at full lattice sizes
def test_batch_uneven_lattices_full_size(ctx, hp):
    """8^4, 12^4, 16^3x32, 24^3x48 with kappa, eps from PCG64(3000) in one schedule (truncated s):
    each lattice's prefix equals its own single-lattice solve.  12^4 runs past 256 vectors
    into the three-colour / Fourier level."""
    cfg = synth.batch_config()
    s_list = [4, 260, 2, 2]          # 12^4: probes 0..259 include 256..259 of the F_3 level
    ops, dims_list, keep = [], [], []
    for c in cfg:
        U = synth.gauge_links(c["dims"], c["eps"], c["link_seed"], device="cuda:0")
        L = links_dev(U)
        keep.append(L)
        ops.append(ctx.make_operator(hp.OP_WILSON, 0.0, c["kappa"], L, None))
        dims_list.append(c["dims"])
    outs, st = ctx.trace_inv_batch(ops, dims_list, s_list, 1e-10, ctx.make_opts("fp16", z0_seed=3000,
                                                                                rhs_block=48, use_graph=1))
    assert st["rhs_solved"] == 12 * sum(s_list) and st["max_true_residual"] <= 1e-10
    for op, dims, s, T in zip(ops, dims_list, s_list, outs):
        T1, _, _ = ctx.trace_inv(op, dims, s, 1e-10, ctx.make_opts("fp64", z0_seed=3000))
        assert np.all(rel(T, T1) <= TRACE_RTOL), (dims, T[:3], T1[:3])
        assert np.max(np.abs(T.imag)) <= 1e-8 * np.max(np.abs(T.real))


# ------------------------------------------------------------------ differentiation config
def test_gradient_config_8x8x8x8_copy_vs_oracle_and_fd(ctx, hp):
    """kappa 0.118, eps 0.3, mu(x) ~ N(0, 0.01) from PCG64(5000) on the 8^4 copy: the adjoint
    (gamma_5) gradient equals the oracle's explicit-adjoint gradient and central differences."""
    dims = (8, 8, 8, 8)
    V = 4096
    U = synth.gauge_links(dims, 0.3, 1005)
    mf = synth.mass_field(dims, 0.01, 5000)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(mf))
    s = 2
    g = np.zeros(V)
    T, dTdm, st = ctx.trace_inv_grad(op, dims, s, 1e-12, ctx.make_opts("fp64", z0_seed=5001), g)
    g_ref = E.wilson_grad_mass_field(dims, U, 0.118, s, 5001, tol=1e-13, mass_field=mf).real
    assert np.allclose(g, g_ref, rtol=1e-7, atol=1e-9 * np.abs(g_ref).max())
    h = 1e-5
    for site in (0, 1234, 4095):
        e = mf.copy()
        e[site] += h
        tp, _, _ = ctx.trace_inv(ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(e)), dims, s, 1e-13,
                                 ctx.make_opts("fp64", z0_seed=5001))
        e[site] -= 2 * h
        tm, _, _ = ctx.trace_inv(ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(e)), dims, s, 1e-13,
                                 ctx.make_opts("fp64", z0_seed=5001))
        fd = (tp[-1] - tm[-1]).real / (2 * h)
        assert abs(fd - g[site]) <= 1e-4 * max(1.0, abs(g[site])), (site, fd, g[site])


def test_gradient_config_24x24x24x48_properties(ctx, hp):
    """24^3x48, kappa 0.118, eps 0.3 (truncated to s = 2): mixed and FP64 gradients agree, the
    uniform-mass derivative equals the sum of the per-site one, and it matches central
    differences of the uniform mass."""
    dims = (24, 24, 24, 48)
    V = 663552
    U = synth.gauge_links(dims, 0.3, 1005, device="cuda:0")
    mf = dev(synth.mass_field(dims, 0.01, 5000))
    L = links_dev(U)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, L, mf)
    g64 = torch.zeros(V, dtype=torch.float64, device="cuda:0")
    g16 = torch.zeros(V, dtype=torch.float64, device="cuda:0")
    T64, dm64, _ = ctx.trace_inv_grad(op, dims, 2, 1e-10, ctx.make_opts("fp64", z0_seed=5001), g64)
    T16, dm16, _ = ctx.trace_inv_grad(op, dims, 2, 1e-10, ctx.make_opts("fp16", z0_seed=5001), g16)
    assert abs(dm64 - g64.sum().item()) <= 1e-10 * abs(dm64)
    assert abs(dm16 - dm64) <= 1e-7 * abs(dm64)
    assert torch.allclose(g16, g64, rtol=1e-6, atol=1e-8 * g64.abs().max().item())
    h = 1e-5
    tp, _, _ = ctx.trace_inv(ctx.make_operator(hp.OP_WILSON, h, 0.118, L, mf), dims, 2, 1e-12,
                             ctx.make_opts("fp64", z0_seed=5001))
    tm, _, _ = ctx.trace_inv(ctx.make_operator(hp.OP_WILSON, -h, 0.118, L, mf), dims, 2, 1e-12,
                             ctx.make_opts("fp64", z0_seed=5001))
    fd = (tp[-1] - tm[-1]).real / (2 * h)
    assert abs(fd - dm64) <= 1e-5 * abs(dm64), (fd, dm64)


@pytest.mark.parametrize("prec", ["fp16", "fp32", "bf16"])
def test_mixed_precision_true_residual_reaches_1e12(ctx, hp, prec):
    """The mixed solvers certify their solutions with a float-float true residual b - D x: driving
    them to 1e-12 (100x below the configs' tolerance) must still reproduce the dense-LU trace."""
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.4, 44)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(U), None)
    T, _, st = ctx.trace_inv(op, dims, 3, 1e-12, ctx.make_opts(prec, z0_seed=4))
    T_ref = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, 3, 4, method="dense"))
    assert st["max_true_residual"] <= 1e-12
    assert np.all(rel(T, T_ref) <= 1e-11), (T, T_ref)


# ------------------------------------------------------------------ even-odd (Schur complement) iteration
_ORACLE_CACHE = {}


# variant 0: the default (slot groups of 4, 18-real links); 4001: 12-real links (row 3 rebuilt);
# 2101: slot groups of 2; kernel: the V / T step kernels (0 autotuned, 1 one right-hand side per
# thread, 4 the pair kernels, 6 the tensor-core even-site kernel)
@pytest.mark.parametrize("prec,variant,kernel", [("fp64", 0, 0), ("fp32", 0, 0), ("fp16", 0, 0), ("bf16", 0, 0),
                                                 ("fp16", 4001, 0), ("fp32", 4001, 0), ("bf16", 2101, 0),
                                                 ("fp16", 0, 1), ("fp16", 0, 4), ("fp16", 0, 6), ("bf16", 0, 6)])
def test_even_odd_trace_parity(ctx, hp, prec, variant, kernel):
    dims = (4, 4, 6, 4)   # 384 sites, 192 per parity: the second 128-site tile is ragged
    U = synth.gauge_links(dims, 0.3, 1002)
    mf = synth.mass_field(dims, 0.01, 77)
    op = ctx.make_operator(hp.OP_WILSON, 0.01, 0.115, links_dev(U), dev(mf))
    s = 6
    T, _, st = ctx.trace_inv(op, dims, s, 1e-10, ctx.make_opts(prec, z0_seed=2002, rhs_block=24, even_odd=1,
                                                               rhs_per_thread=variant, eo_kernel=kernel))
    if "eo_parity" not in _ORACLE_CACHE:
        _ORACLE_CACHE["eo_parity"] = E.trace_prefix(E.wilson_quadratures(dims, U, 0.115, 0, s, 2002, mass=0.01,
                                                                         mass_field=mf, method="dense"))
    T_ref = _ORACLE_CACHE["eo_parity"]
    assert np.all(rel(T, T_ref) <= TRACE_RTOL), (T, T_ref)
    assert st["max_true_residual"] <= 1e-10 and st["rhs_solved"] == 12 * s


def test_even_odd_full_sequence_and_fallback(ctx, hp):
    from pins import free_wilson_trace_inverse

    dims = (4, 4, 2, 4)
    V = 128
    Ufree = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    Ug, _ = synth.gauge_transform(Ufree, dims, 78)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(Ug), None)
    T, _, _ = ctx.trace_inv(op, dims, V, 1e-11, ctx.make_opts("fp16", z0_seed=5, even_odd=1))
    exact = free_wilson_trace_inverse(dims, 0.12)
    assert abs(T[-1].real - exact) <= 1e-9 * exact
    # odd L_1: the even-odd request falls back to the full iteration and stays exact
    dims = (3, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 79)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(U), None)
    T, _, _ = ctx.trace_inv(op, dims, 4, 1e-10, ctx.make_opts("fp16", z0_seed=5, even_odd=1))
    T_ref = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, 4, 5, method="dense"))
    assert np.all(rel(T, T_ref) <= TRACE_RTOL)


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_even_odd_gradient_and_tight_residual(ctx, hp, prec):
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 21)
    mf = synth.mass_field(dims, 0.01, 5000)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(mf))
    g = np.zeros(128)
    T, dTdm, st = ctx.trace_inv_grad(op, dims, 3, 1e-12, ctx.make_opts(prec, z0_seed=7, even_odd=1), g)
    g_ref = E.wilson_grad_mass_field(dims, U, 0.118, 3, 7, mass_field=mf, method="dense").real
    assert st["max_true_residual"] <= 1e-12
    assert np.allclose(g, g_ref, rtol=1e-7, atol=1e-9)
    T_ref = E.trace_prefix(E.wilson_quadratures(dims, U, 0.118, 0, 3, 7, mass_field=mf, method="dense"))
    assert np.all(rel(T, T_ref) <= 1e-11)


def test_even_odd_batch_and_config_sizes(ctx, hp):
    """Uneven batch at full lattice sizes with the Schur iteration equals the full iteration."""
    cfg = synth.batch_config()
    s_list = [3, 2, 2, 2]
    ops, dims_list, keep = [], [], []
    for c in cfg:
        U = synth.gauge_links(c["dims"], c["eps"], c["link_seed"], device="cuda:0")
        L = links_dev(U)
        keep.append(L)
        ops.append(ctx.make_operator(hp.OP_WILSON, 0.0, c["kappa"], L, None))
        dims_list.append(c["dims"])
    eo, st = ctx.trace_inv_batch(ops, dims_list, s_list, 1e-10, ctx.make_opts("fp16", z0_seed=3000, even_odd=1,
                                                                              use_graph=1))
    full, _ = ctx.trace_inv_batch(ops, dims_list, s_list, 1e-10, ctx.make_opts("fp64", z0_seed=3000))
    for a_, b_ in zip(eo, full):
        assert np.all(rel(a_, b_) <= TRACE_RTOL)
    assert st["max_true_residual"] <= 1e-10


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_even_odd_start_at_tolerance(ctx, hp, prec):
    """A loose tolerance that the first residual already meets: the mixed solver hands its FP32
    start to the exact steps, which certify it with no iteration -- the same estimate as the FP64
    solver, whose start is exact."""
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 91)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.05, links_dev(U), None)
    T, _, st = ctx.trace_inv(op, dims, 2, 0.9, ctx.make_opts(prec, z0_seed=8, even_odd=1))
    T64, _, st64 = ctx.trace_inv(op, dims, 2, 0.9, ctx.make_opts("fp64", z0_seed=8, even_odd=1))
    assert st["iterations_total"] == 0 and st64["iterations_total"] == 0
    assert st["max_true_residual"] <= 0.9
    assert np.all(rel(T, T64) <= 1e-12), (T, T64)


# ------------------------------------------------------------------ clover term (Section 5.3 operator)
CSW = 1.3


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 2, 6), 1), ((3, 4, 2, 2), 5), ((2, 2, 2, 2), 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_clover_apply_parity(ctx, hp, dims, prec, nrhs):
    U = synth.gauge_links(dims, 0.5, 17)
    mf = synth.mass_field(dims, 0.01, 18)
    psi = synth.random_spinors(dims, nrhs, 19)
    op = ctx.make_operator(hp.OP_WILSON, 0.02, 0.12, links_dev(U), dev(mf), csw=CSW)
    out = torch.empty(psi.size * 2, dtype=torch.float64, device="cuda:0")
    ctx.operator_apply(op, dims, nrhs, prec, dev(psi.view(np.float64).reshape(-1)), out)
    got = out.cpu().numpy().view(np.complex128).reshape(psi.shape)
    C = O.clover_term(U, dims, 0.12, CSW)
    for r in range(nrhs):
        ref = O.wilson_apply(psi[r], U, dims, 0.12, 0.02, mf, clover=C)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()   # per site
        assert err <= WILSON_TOL[prec], err
    if prec in ("fp64", "fp32"):   # the clover term is far above the comparison tolerance
        plain = O.wilson_apply(psi[0], U, dims, 0.12, 0.02, mf)
        assert np.linalg.norm(got[0] - plain) > 100 * WILSON_TOL[prec] * np.linalg.norm(plain)


@pytest.mark.parametrize("prec,eo", [("fp64", 0), ("fp64", 1), ("fp16", 1), ("fp32", 1), ("bf16", 1), ("fp16", 0)])
def test_clover_trace_parity(ctx, hp, prec, eo):
    dims = (4, 4, 2, 6)
    U = synth.gauge_links(dims, 0.4, 1004)
    mf = synth.mass_field(dims, 0.01, 78)
    op = ctx.make_operator(hp.OP_WILSON, 0.01, 0.115, links_dev(U), dev(mf), csw=CSW)
    s = 4
    T, _, st = ctx.trace_inv(op, dims, s, 1e-10, ctx.make_opts(prec, z0_seed=2004, rhs_block=24, even_odd=eo))
    if "clover_trace" not in _ORACLE_CACHE:
        _ORACLE_CACHE["clover_trace"] = E.trace_prefix(E.wilson_quadratures(dims, U, 0.115, 0, s, 2004, mass=0.01,
                                                                            mass_field=mf, method="dense", csw=CSW))
    T_ref = _ORACLE_CACHE["clover_trace"]
    assert np.all(rel(T, T_ref) <= TRACE_RTOL), (T, T_ref)
    assert st["max_true_residual"] <= 1e-10 and st["rhs_solved"] == 12 * s


def test_clover_full_sequence_on_pure_gauge_links_is_free_closed_form(ctx, hp):
    """Pure-gauge links have unit plaquettes, so the clover term vanishes and the full probing
    sequence (s = V) must give the free-field trace in closed form."""
    from pins import free_wilson_trace_inverse

    dims = (4, 4, 2, 4)
    V = int(np.prod(dims))
    Ufree = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    Ug, _ = synth.gauge_transform(Ufree, dims, 79)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(Ug), None, csw=1.7)
    T, _, _ = ctx.trace_inv(op, dims, V, 1e-11, ctx.make_opts("fp16", z0_seed=6, even_odd=1))
    exact = free_wilson_trace_inverse(dims, 0.12)
    assert abs(T[-1].real - exact) <= 1e-9 * exact


def test_clover_gradient_vs_oracle(ctx, hp):
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 23)
    mf = synth.mass_field(dims, 0.01, 5001)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.118, links_dev(U), dev(mf), csw=CSW)
    g = np.zeros(128)
    T, dTdm, st = ctx.trace_inv_grad(op, dims, 3, 1e-12, ctx.make_opts("fp16", z0_seed=7, even_odd=1), g)
    g_ref = E.wilson_grad_mass_field(dims, U, 0.118, 3, 7, mass_field=mf, method="dense", csw=CSW).real
    assert st["max_true_residual"] <= 1e-12
    assert np.allclose(g, g_ref, rtol=1e-7, atol=1e-9)


# ------------------------------------------------------------------ the comparison sequences (Section 5.2)
@pytest.mark.parametrize("kind,dims,seed", [("natural", (8, 8, 8, 8), 0), ("natural", (2, 4, 8), 11),
                                            ("natural", (1024,), 3), ("z2", (4, 4, 4, 4), 12345),
                                            ("z2", (12, 12), 7), ("z2", (3, 5, 4, 6), 1)])
def test_probe_sequence_bit_exact(ctx, hp, kind, dims, seed):
    V = int(np.prod(dims))
    for first, count in [(0, min(V, 40)), (V - 5, 5)]:
        out = torch.empty(count * V, dtype=torch.int16, device="cuda:0")
        per = ctx.probe_vectors(dims, first, count, seed, out, kind=kind)
        ref = (Pr.probe_phases_natural(V, first, count, seed) if kind == "natural"
               else Pr.probe_phases_z2(V, first, count, seed))
        got = out.cpu().numpy().astype(np.int64).reshape(count, V) & 0xFFFF
        assert np.array_equal(got, ref * (per // 2))


def test_natural_order_rejects_non_power_of_two(ctx, hp):
    out = torch.empty(12 * 12, dtype=torch.int16, device="cuda:0")
    with pytest.raises(hp.HProbeError) as e:
        ctx.probe_vectors((12, 12), 0, 1, 0, out, kind="natural")
    assert e.value.status == hp.HP_EUNSUPPORTED


@pytest.mark.parametrize("kind", ["natural", "z2"])
def test_laplacian_trace_comparison_sequences(ctx, hp, kind):
    dims = (8, 8, 8, 8)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.05)
    s = 24
    T, _, st = ctx.trace_inv(op, dims, s, 1e-12, ctx.make_opts("fp64", z0_seed=21, probe_kind=kind))
    T_ref = E.trace_prefix(E.laplacian_quadratures(dims, 0.05, 0, s, 21, method="dense", kind=kind))
    assert np.all(rel(T, T_ref) <= TRACE_RTOL)
    assert st["max_true_residual"] <= 1e-12


def test_wilson_trace_z2_noise(ctx, hp):
    dims = (4, 4, 2, 4)
    U = synth.gauge_links(dims, 0.3, 31)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(U), None)
    T, _, st = ctx.trace_inv(op, dims, 3, 1e-10, ctx.make_opts("fp16", z0_seed=8, even_odd=1, probe_kind="z2"))
    W = E.probe_vectors(dims, 0, 3, 8, kind="z2")
    X = E.wilson_solutions(dims, U, 0.12, W, method="dense")
    q = [sum(np.vdot(E._dilute(W[m], a), X[m, a]) for a in range(12)) for m in range(3)]
    assert np.all(rel(T, E.trace_prefix(q)) <= TRACE_RTOL)


def test_variance_of_hierarchical_probing_over_z0_matches_closed_form(ctx, hp):
    """The GPU's T_s over many z_0 (4^4 Laplacian): its sample variance agrees with the exact
    z_0-variance within the sampling error, and the hierarchical sequence has a smaller variance
    than natural order at the completion point s = 32."""
    from oracle import probing as Pr

    dims = (4, 4, 4, 4)
    V = 256
    B = np.linalg.inv(O.laplacian_dense(dims, 0.5))
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.5)
    seeds = range(1, 201)
    Ts = np.array([ctx.trace_inv(op, dims, 32, 1e-13, ctx.make_opts("fp64", z0_seed=z, rhs_block=64))[0][31].real
                   for z in seeds])
    ph, _ = Pr.probe_phases(dims, 0, 32, 0)
    var = E.z0_variance(B, 1 - 2 * ph, 32)
    n = len(Ts)
    assert abs(Ts.mean() - np.trace(B)) <= 4 * np.sqrt(var / n)
    assert abs(Ts.var(ddof=1) / var - 1) <= 4 * np.sqrt(2.0 / (n - 1)) + 0.1
    var_nat = E.z0_variance(B, 1 - 2 * Pr.probe_phases_natural(V, 0, 32, 0), 32)
    assert var < var_nat


# ------------------------------------------------------------------ quadrature bounds (Section 1.1.2)
@pytest.mark.parametrize("dims,mass,seed,mf", [((8, 8, 8, 8), 0.05, 1, False), ((6, 6, 2, 3), 0.2, 5, False),
                                               ((4, 4, 4, 8), 0.1, 3, True)])
def test_laplacian_quadrature_bounds_bracket_the_oracle(ctx, hp, dims, mass, seed, mf):
    """Every prefix T_s lies between the Gauss and Gauss-Radau bounds, and the brackets closed to
    the requested relative width; the last case uses a mass field (node m + min mu)."""
    V = int(np.prod(dims))
    field = synth.mass_field(dims, 0.02, 40) if mf else None
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass, 0.0, None, dev(field) if mf else None)
    s = min(32, hp.basis_info(dims)["n_vectors"])
    T, lo, hi, st = ctx.trace_inv_bounds(op, dims, s, 1e-10, ctx.make_opts("fp64", z0_seed=seed, rhs_block=64))
    T_ref = E.trace_prefix(E.laplacian_quadratures(dims, mass, 0, s, seed, mass_field=field, method="dense")).real
    assert np.all(lo <= T_ref * (1 + 1e-12)) and np.all(hi >= T_ref * (1 - 1e-12))
    assert np.all((hi - lo) <= 1.1e-10 * np.abs(lo))
    assert np.all(rel(T.real, T_ref) <= 1e-9)
    assert st["rhs_solved"] == s * (2 if hp.basis_info(dims)["period"] > 2 else 1)


def test_quadrature_bounds_stop_earlier_than_the_residual(ctx, hp):
    """The quadrature error falls as the square of the residual: bracketing each quadrature to 1e-10
    takes fewer CG iterations than a 1e-10 residual, for the same estimate."""
    dims = (8, 8, 8, 8)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.05)
    opts = ctx.make_opts("fp64", z0_seed=2, rhs_block=64)
    T, lo, hi, sb = ctx.trace_inv_bounds(op, dims, 64, 1e-10, opts)
    T2, _, sr = ctx.trace_inv(op, dims, 64, 1e-10, opts)
    assert sb["iterations_total"] < 0.8 * sr["iterations_total"]
    assert np.all(rel(T, T2) <= 1e-9)


def test_quadrature_bounds_reject_wilson_and_bad_node(ctx, hp):
    U = synth.gauge_links((4, 4, 2, 4), 0.3, 1)
    opw = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links_dev(U), None)
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_bounds(opw, (4, 4, 2, 4), 2, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EINVAL
    opl = ctx.make_operator(hp.OP_LAPLACIAN, -0.5)
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_bounds(opl, (4, 4), 2, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EINVAL
