"""The even-odd iteration's own kernels and the headline solve against the oracle, on small
lattices and at the full 32^3x64 size of the headline workload.

* hp_schur_apply runs the solver's V-step launches (k_eo_even, then k_eo_odd) on given fields;
  the oracle's wilson_schur_apply is S = A_o - kappa^2 H_oe A_e^-1 H_eo written with its own
  Wilson operator.  Errors are per site: the largest component error of any site, relative to
  the largest component of the reference field (a single wrong site fails).
* hp_trace_inv_solutions returns the solutions of the headline solve (FP16 iteration on the
  Schur complement, 24 slots); the oracle's FP64 operator recomputes their true residuals and
  the quadrature q_0 = sum_a v_{0,a}^H x_{0,a}.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import operators as O
from paper_1302_4018_gb300 import synth

pytestmark = pytest.mark.gpu

# per-site error bounds of the Schur complement by storage precision: two hops, the intermediate
# A_e^-1 H_eo x stored in the iteration precision (FP16 / BF16 with a per-site norm)
SCHUR_TOL = {"fp64": 1e-13, "fp32": 5e-6, "fp16": 6e-3, "bf16": 5e-2}
# the full-lattice stencil (one hop)
WILSON_TOL = {"fp64": 1e-13, "fp32": 3e-6, "fp16": 4e-3, "bf16": 3e-2}


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


def site_max_err(got, ref, sites=None):
    """max over sites of the largest |got - ref| component, relative to max |ref| (fields [V, 4, 3])."""
    d = np.abs(got - ref).reshape(got.shape[0], -1).max(axis=1)
    if sites is not None:
        d = d[sites]
    return d.max() / np.abs(ref).max()


SCHUR_CASES = [((4, 4, 4, 4), 1, 0.0), ((4, 4, 4, 4), 5, 0.0), ((6, 2, 4, 6), 3, 0.0), ((2, 2, 2, 2), 2, 0.0),
               ((8, 4, 6, 2), 4, 0.0), ((4, 4, 4, 4), 3, 1.0), ((6, 4, 2, 4), 2, 0.8), ((2, 6, 2, 2), 2, 0.0)]


@pytest.mark.parametrize("dims,nrhs,csw", SCHUR_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_schur_apply_matches_oracle(ctx, hp, dims, nrhs, csw, prec):
    d4 = tuple(dims) + (1,) * (4 - len(dims))
    U = synth.gauge_links(dims, 0.4, 17)
    mf = synth.mass_field(dims, 0.02, 18)
    psi = synth.random_spinors(dims, nrhs, 19)
    op = ctx.make_operator(hp.OP_WILSON, 0.03, 0.12, dev(U.view(np.float64).reshape(-1)), dev(mf), csw=csw)
    out = torch.full((psi.size * 2,), float("nan"), dtype=torch.float64, device="cuda:0")
    ctx.schur_apply(op, dims, nrhs, prec, dev(psi.view(np.float64).reshape(-1)), out)
    got = out.cpu().numpy().view(np.complex128).reshape(psi.shape)
    C = O.clover_term(U, d4, 0.12, csw) if csw else None
    for r in range(nrhs):
        ref = O.wilson_schur_apply(psi[r], U, d4, 0.12, 0.03, mf, clover=C)
        assert site_max_err(got[r], ref) <= SCHUR_TOL[prec], (prec, r, site_max_err(got[r], ref))
        assert not np.any(got[r][O.site_parity(d4) == 0])


# every kernel variant of the V step (eo_kernel: 1 one right-hand side per thread, 3 / 4 / 13 / 14 the
# pair kernels, 5 pair even + single odd, 6 the tensor-core even-site kernel for binary16 -- with
# up to 32 right-hand sides in row groups of 8, so 3, 9, 20 and 30 fill one to four groups, the
# last ragged; other precisions and the clover term run the pair kernels in its place)
VARIANT_CASES = [("fp16", k) for k in (1, 3, 4, 5, 6, 13, 14)] + [("bf16", 1), ("bf16", 4), ("bf16", 6),
                                                                   ("fp32", 1), ("fp32", 4), ("fp32", 6)]


@pytest.mark.parametrize("dims,nrhs,csw", [((4, 4, 4, 4), 3, 0.0), ((6, 2, 4, 6), 9, 0.0), ((8, 4, 6, 2), 20, 0.0),
                                           ((4, 6, 2, 4), 30, 0.0), ((4, 4, 2, 4), 9, 1.0)])
@pytest.mark.parametrize("prec,kernel", VARIANT_CASES)
def test_schur_apply_kernel_variants_match_oracle(ctx, hp, dims, nrhs, csw, prec, kernel):
    U = synth.gauge_links(dims, 0.4, 27)
    mf = synth.mass_field(dims, 0.02, 28)
    psi = synth.random_spinors(dims, nrhs, 29)
    op = ctx.make_operator(hp.OP_WILSON, 0.03, 0.12, dev(U.view(np.float64).reshape(-1)), dev(mf), csw=csw)
    out = torch.full((psi.size * 2,), float("nan"), dtype=torch.float64, device="cuda:0")
    ctx.schur_apply(op, dims, nrhs, prec, dev(psi.view(np.float64).reshape(-1)), out, eo_kernel=kernel)
    got = out.cpu().numpy().view(np.complex128).reshape(psi.shape)
    C = O.clover_term(U, dims, 0.12, csw) if csw else None
    for r in range(nrhs):
        ref = O.wilson_schur_apply(psi[r], U, dims, 0.12, 0.03, mf, clover=C)
        assert site_max_err(got[r], ref) <= SCHUR_TOL[prec], (prec, kernel, r, site_max_err(got[r], ref))
        assert not np.any(got[r][O.site_parity(dims) == 0])


@pytest.mark.parametrize("dims", [(3, 4, 2, 2), (4, 3, 2, 2), (2, 2, 2, 5), (2, 6)])
def test_schur_apply_rejects_lattices_without_a_red_black_split(ctx, hp, dims):
    """An odd extent (or a padded one of size 1) makes some hop join sites of one parity."""
    V = int(np.prod(dims))
    U = synth.gauge_links(dims, 0.3, 1)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, dev(U.view(np.float64).reshape(-1)), None)
    x = torch.zeros(V * 24, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hp.HProbeError) as e:
        ctx.schur_apply(op, dims, 1, "fp64", x, torch.empty_like(x))
    assert e.value.status == hp.HP_EINVAL


@pytest.fixture(scope="module")
def headline(ctx, hp):
    """32^3x64, kappa 0.12, eps 0.4, link seed 1003 (the headline workload's links)."""
    dims = (32, 32, 32, 64)
    U = synth.gauge_links(dims, 0.4, 1003, device="cuda:0")
    links = dev(U.view(np.float64).reshape(-1))
    return dims, U, links


def test_schur_apply_full_size(ctx, hp, headline):
    """The even-odd stencils at the headline size in every iteration precision, per site over
    every odd site, against one oracle evaluation of S."""
    dims, U, links = headline
    V = int(np.prod(dims))
    psi = synth.random_spinors(dims, 1, 31)[0]
    ref = O.wilson_schur_apply(psi, U, dims, 0.12)
    odd = O.site_parity(dims) == 1
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links, None)
    out = torch.empty(V * 24, dtype=torch.float64, device="cuda:0")
    inp = dev(psi.view(np.float64).reshape(-1))
    for prec, kernel in (("fp64", 0), ("fp32", 0), ("fp16", 0), ("bf16", 0), ("fp16", 4), ("fp16", 6)):
        ctx.schur_apply(op, dims, 1, prec, inp, out, eo_kernel=kernel)
        got = out.cpu().numpy().view(np.complex128).reshape(V, 4, 3)
        err = site_max_err(got, ref, odd)
        assert err <= SCHUR_TOL[prec], (prec, kernel, err)


def test_wilson_apply_full_size_per_site(ctx, hp, headline):
    """The full-lattice stencil at the headline size in every precision, per site."""
    dims, U, links = headline
    V = int(np.prod(dims))
    psi = synth.random_spinors(dims, 1, 5)[0]
    ref = O.wilson_apply(psi, U, dims, 0.12)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links, None)
    out = torch.empty(V * 24, dtype=torch.float64, device="cuda:0")
    inp = dev(psi.view(np.float64).reshape(-1))
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        ctx.operator_apply(op, dims, 1, prec, inp, out)
        got = out.cpu().numpy().view(np.complex128).reshape(V, 4, 3)
        err = site_max_err(got, ref)
        assert err <= WILSON_TOL[prec], (prec, err)


def test_headline_solutions_against_the_oracle(ctx, hp, headline):
    """The headline solve (FP16 iteration on the Schur complement, 24 slots, tol 1e-10, z_0 seed
    2003): the twelve solutions of probe 0 come back through hp_trace_inv_solutions; the
    oracle's FP64 Wilson operator gives their true residuals (three of them: 15 s each) and the
    quadrature q_0 from all twelve."""
    dims, U, links = headline
    V = int(np.prod(dims))
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, links, None)
    opts = ctx.make_opts("fp16", z0_seed=2003, rhs_block=24, even_odd=1)
    x = torch.empty(12 * V * 24, dtype=torch.float64, device="cuda:0")
    q = np.zeros(2, dtype=np.complex128)
    T, q, st = ctx.trace_inv_solutions(op, dims, 2, 1e-10, opts, x, q_inout=q)
    assert st["max_true_residual"] <= 1e-10 and st["n_unconverged"] == 0
    xs = x.cpu().numpy().view(np.complex128).reshape(12, V, 4, 3)
    del x
    v = E.probe_vectors(dims, 0, 1, 2003)[0]
    q0 = 0.0
    for a in range(12):
        q0 += np.vdot(v, xs[a].reshape(V, 12)[:, a])
    assert abs(q0 - q[0]) <= 1e-9 * abs(q[0]), (q0, q[0])
    assert abs(T[0] - q[0]) == 0 and abs(T[1] - (q[0] + q[1]) / 2) <= 1e-15 * abs(T[1])
    for a in (0, 5, 11):
        b = np.zeros((V, 12), dtype=np.complex128)
        b[:, a] = v
        b = b.reshape(V, 4, 3)
        r = b - O.wilson_apply(xs[a], U, dims, 0.12)
        res = np.linalg.norm(r) / np.linalg.norm(b)
        assert res <= 1e-10, (a, res)


@pytest.mark.parametrize("dims", [(4, 3, 2, 2), (2, 2, 2, 5)])
def test_even_odd_request_on_an_odd_extent_iterates_the_full_lattice(ctx, hp, dims):
    """With an odd extent the wrap-around joins sites of one parity, so the even-odd split does not
    exist: the solver iterates the full lattice instead and the trace still matches dense LU."""
    U = synth.gauge_links(dims, 0.4, 3)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, dev(U.view(np.float64).reshape(-1)), None)
    T, _, st = ctx.trace_inv(op, dims, 3, 1e-10, ctx.make_opts("fp16", z0_seed=7, even_odd=1))
    T_ref = E.trace_prefix(E.wilson_quadratures(dims, U, 0.12, 0, 3, 7, method="dense"))
    assert np.all(np.abs(T - T_ref) <= 1e-9 * np.abs(T_ref)), (T, T_ref)
    assert st["max_true_residual"] <= 1e-10


def test_trace_prefix_of_gathered_blocks_equals_one_call(ctx, hp):
    """The multi-rank path on one GPU: two probe blocks solved by separate calls (the second
    without the first's quadratures, as another rank would), concatenated, and the prefix
    formed by hp_trace_prefix, against one call over the whole sequence."""
    dims = (4, 4, 4, 8)
    U = synth.gauge_links(dims, 0.3, 41)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, dev(U.view(np.float64).reshape(-1)), None)

    def opts(first):
        return ctx.make_opts("fp64", z0_seed=9, first=first, even_odd=1)

    T1, q1, _ = ctx.trace_inv(op, dims, 6, 1e-12, opts(0), q_inout=np.zeros(6, dtype=np.complex128))
    _, qa, _ = ctx.trace_inv(op, dims, 3, 1e-12, opts(0), q_inout=np.zeros(3, dtype=np.complex128))
    _, qb, _ = ctx.trace_inv(op, dims, 6, 1e-12, opts(3), q_inout=np.zeros(6, dtype=np.complex128))
    gathered = np.concatenate([qa, qb[3:]])
    assert np.allclose(gathered, q1, rtol=1e-13, atol=0)
    assert ctx.trace_prefix(q1).tobytes() == T1.tobytes()       # same kernel, same order
    Tg = ctx.trace_prefix(gathered)
    assert np.allclose(Tg, T1, rtol=1e-13, atol=0)
    assert np.allclose(Tg, E.trace_prefix(gathered), rtol=1e-15, atol=0)
