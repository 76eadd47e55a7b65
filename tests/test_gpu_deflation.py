"""Deflated hierarchical probing (Laplacian and Wilson) on the GPU vs the oracle.

The trace estimate T_s = sum_j 1/lambda_j + (1/s) sum_m (P v_m)^H A^-1 (P v_m) is compared with
the oracle's dense-solve restatement within 1e-9 relative (CG to a true residual of 1e-12,
||A^-1|| <= 1/0.3); at s = N the GPU estimate must equal the Fourier closed form of Tr A^-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import operators as O
from paper_1302_4018_gb300 import synth
from pins import laplacian_trace_inverse

pytestmark = pytest.mark.gpu


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


def _eig(dims, mass, k):
    lam, V = np.linalg.eigh(O.laplacian_dense(dims, mass))
    return lam[:k], np.ascontiguousarray(V[:, :k].T)   # [k][V]


@pytest.mark.parametrize("dims,k,s,z0,device", [((4, 4, 4, 4), 1, 16, 0, False), ((4, 4, 4, 4), 8, 16, 7, True),
                                               ((4, 4, 4, 4), 40, 32, 3, False), ((6, 4, 2, 2), 6, 48, 11, False)])
def test_deflated_trace_matches_oracle(ctx, hp, dims, k, s, z0, device):
    mass = 0.3
    lam, Vt = _eig(dims, mass, k)
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass)
    ev = torch.from_numpy(Vt).cuda() if device else Vt
    q = np.zeros(s, dtype=np.complex128)
    T, q, st = ctx.trace_inv_deflated(op, dims, ev, lam, s, 1e-12, ctx.make_opts("fp64", z0_seed=z0), q_inout=q)
    qo = E.laplacian_deflated_quadratures(dims, mass, Vt.T, 0, s, z0)
    To = E.deflated_trace_prefix(lam, qo)
    assert np.abs(q - qo).max() <= 1e-9 * np.abs(qo).max()
    assert np.abs(T - To).max() <= 1e-9 * np.abs(To).max()
    assert st["max_true_residual"] <= 1e-12


def test_deflated_full_sequence_is_exact_on_gpu(ctx, hp):
    dims, mass, k = (4, 4, 2, 2), 0.3, 5
    lam, Vt = _eig(dims, mass, k)
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass)
    T, _, _ = ctx.trace_inv_deflated(op, dims, Vt, lam, 64, 1e-13, ctx.make_opts("fp64", z0_seed=2))
    exact = laplacian_trace_inverse(dims, mass)
    assert abs(T[-1].real - exact) <= 1e-10 * exact


def test_deflated_errors(ctx, hp):
    dims, mass = (4, 4, 2, 2), 0.3
    lam, Vt = _eig(dims, mass, 3)
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass)
    bad = lam.copy()
    bad[1] = -1.0
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_deflated(op, dims, Vt, bad, 8, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EINVAL
    links = torch.zeros(64 * 72, dtype=torch.float64, device="cuda:0")
    opw = ctx.make_operator(hp.OP_WILSON, 0.0, 0.1, links)
    with pytest.raises(ValueError):   # Laplacian-shaped (real [k][V]) vectors for a Wilson operator
        ctx.trace_inv_deflated(opw, dims, Vt, lam, 8, 1e-10, ctx.make_opts("fp64"))


# ------------------------------------------------------------------ eigenpairs computed by the library
def _projector(Vt):
    return Vt.T @ Vt


@pytest.mark.parametrize("dims,mass,k", [((8, 8, 8), 0.1, 7), ((4, 4, 4, 4), 0.3, 9), ((6, 6, 4, 2), 0.2, 1)])
def test_laplacian_eigs_match_the_oracle(ctx, hp, dims, mass, k):
    """k at a gap of the spectrum (8^3: the constant mode and the six waves of the first shell;
    4^4: 1 + 8): eigenvalues within 1e-10, the spanned subspace equal to the oracle's (the
    eigenvectors of a repeated eigenvalue are a basis the method does not fix)."""
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass)
    lam, V, res = ctx.laplacian_eigs(op, dims, k, tol=1e-10)
    lam_o, V_o = E.laplacian_lowest_eigenpairs(dims, mass, k)
    assert np.allclose(lam, lam_o, rtol=1e-10, atol=0), (lam, lam_o)
    assert np.all(res <= 1e-10)
    assert np.allclose(V @ V.T, np.eye(k), atol=1e-12)
    assert np.abs(_projector(V) - _projector(V_o)).max() <= 1e-8
    A = O.laplacian_dense(dims, mass)
    assert np.abs(A @ V.T - V.T * lam[None, :]).max() <= 1e-9 * lam.max()


def test_laplacian_eigs_with_a_mass_field_and_device_output(ctx, hp):
    """A random mass field splits every degeneracy: each eigenvector agrees with the oracle's up
    to its sign; the vectors are written to device memory."""
    dims, mass, k = (4, 4, 4, 4), 0.3, 6
    from paper_1302_4018_gb300 import synth

    mf = 0.2 * synth.mass_field(dims, 1.0, 77)
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass, 0.0, None, torch.from_numpy(mf).cuda())
    out = torch.zeros(k * 256, dtype=torch.float64, device="cuda:0")
    lam, _, res = ctx.laplacian_eigs(op, dims, k, tol=1e-11, evecs=out)
    V = out.cpu().numpy().reshape(k, 256)
    lam_o, V_o = E.laplacian_lowest_eigenpairs(dims, mass, k, mf)
    assert np.allclose(lam, lam_o, rtol=1e-10, atol=0)
    assert np.all(res <= 1e-11)
    for j in range(k):
        assert abs(abs(V[j] @ V_o[j]) - 1.0) <= 1e-9, j


def test_deflation_with_library_eigenvectors(ctx, hp):
    """Deflated probing with the library's own eigenpairs equals the oracle's deflated estimate
    with the exact eigenpairs (the deflated subspace is the same)."""
    dims, mass, k, s = (8, 8, 8), 0.1, 7, 32
    op = ctx.make_operator(hp.OP_LAPLACIAN, mass)
    lam, V, _ = ctx.laplacian_eigs(op, dims, k, tol=1e-11)
    q = np.zeros(s, dtype=np.complex128)
    T, q, _ = ctx.trace_inv_deflated(op, dims, V, lam, s, 1e-12, ctx.make_opts("fp64", z0_seed=4), q_inout=q)
    lam_o, V_o = E.laplacian_lowest_eigenpairs(dims, mass, k)
    To = E.deflated_trace_prefix(lam_o, E.laplacian_deflated_quadratures(dims, mass, V_o.T, 0, s, 4))
    assert np.abs(T - To).max() <= 1e-9 * np.abs(To).max()


def test_laplacian_eigs_errors(ctx, hp):
    dims = (4, 4, 2, 2)
    op = ctx.make_operator(hp.OP_LAPLACIAN, 0.3)
    with pytest.raises(hp.HProbeError) as e:
        ctx.laplacian_eigs(op, dims, 40)                       # k > V / 2
    assert e.value.status == hp.HP_EINVAL
    links = torch.zeros(64 * 72, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hp.HProbeError) as e:
        ctx.laplacian_eigs(ctx.make_operator(hp.OP_WILSON, 0.0, 0.1, links), dims, 2)
    assert e.value.status == hp.HP_EINVAL
    with pytest.raises(hp.HProbeError) as e:
        ctx.laplacian_eigs(op, (8, 8, 8, 8), 1025)             # above the cap of 1024, below V / 2
    assert e.value.status == hp.HP_EINVAL


# ------------------------------------------------------------------ Wilson: eigenpairs of gamma_5 D, deflation
def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _wilson_op(ctx, hp, dims, seed, kappa=0.12, mass=0.0, mf=None, csw=0.0):
    U = synth.gauge_links(dims, 0.4, seed)
    op = ctx.make_operator(hp.OP_WILSON, mass, kappa, _dev(U.view(np.float64).reshape(-1)),
                           None if mf is None else _dev(mf), csw=csw)
    return U, op


@pytest.mark.parametrize("dims,k,mfs,csw", [((4, 4, 2, 4), 8, 0.0, 0.0), ((4, 2, 4, 2), 12, 0.02, 0.0),
                                            ((2, 4, 2, 4), 6, 0.0, 1.0)])
def test_wilson_eigs_match_the_oracle(ctx, hp, dims, k, mfs, csw):
    """Eigenvalues of gamma_5 D within 1e-9 of the dense oracle's (ordered by |lambda|), unit
    overlap of every eigenvector with the oracle's (non-degenerate for random links)."""
    mf = synth.mass_field(dims, mfs, 41) if mfs else None
    U, op = _wilson_op(ctx, hp, dims, 40, mass=0.01, mf=mf, csw=csw)
    lam, W, res = ctx.wilson_eigs(op, dims, k, 1e-11)
    lam_o, W_o = E.wilson_lowest_eigenpairs(dims, U, 0.12, k, mass=0.01, mass_field=mf, csw=csw)
    assert np.all(res <= 1e-11)
    assert np.allclose(lam, lam_o, rtol=1e-9, atol=0), (lam, lam_o)
    for j in range(k):
        assert abs(abs(np.vdot(W_o[j], W[j])) - 1.0) <= 1e-8, j
    G = np.einsum("ixsc,jxsc->ij", np.conj(W), W)
    assert np.allclose(G, np.eye(k), atol=1e-12)


@pytest.mark.parametrize("dims,k,s,prec,eo,device", [((4, 4, 2, 4), 8, 16, "fp64", 0, False),
                                                     ((4, 4, 2, 4), 20, 32, "fp16", 1, True),
                                                     ((6, 2, 2, 2), 6, 24, "fp64", 0, False),
                                                     ((6, 2, 2, 2), 6, 7, "fp32", 0, True)])
def test_wilson_deflated_trace_matches_oracle(ctx, hp, dims, k, s, prec, eo, device):
    """T_s = sum_j (w_j^H g5 w_j) / lambda_j + (1/s) sum_m q'_m against the oracle's dense solves
    with the projected sources, within 1e-9; (6, 2, 2, 2) has 16 binary vectors, so s = 24 uses the
    three-colour level (every position its own block) and s = 7 the binary blocks."""
    mf = synth.mass_field(dims, 0.01, 43)
    U, op = _wilson_op(ctx, hp, dims, 42, mf=mf)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, 0.12, k, mass_field=mf)
    q = np.zeros(s, dtype=np.complex128)
    ev = _dev(W) if device else W
    T, q, st = ctx.trace_inv_deflated(op, dims, ev, lam, s, 1e-12,
                                      ctx.make_opts(prec, z0_seed=5, even_odd=eo, rhs_block=24), q_inout=q)
    qo, exact = E.wilson_deflated_quadratures(dims, U, 0.12, lam, W, 0, s, 5, mass_field=mf)
    To = exact + E.trace_prefix(qo)
    assert np.abs(q - qo).max() <= 1e-9 * np.abs(qo).max()
    assert np.abs(T - To).max() <= 1e-9 * np.abs(To).max()
    assert st["rhs_solved"] == 12 * s


def test_wilson_full_deflation_is_exact_on_gpu(ctx, hp):
    """All 12 V eigenvectors: every corrected quadrature vanishes and T_s = Tr D^-1 for every s."""
    dims = (2, 2, 2, 2)
    U, op = _wilson_op(ctx, hp, dims, 44)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, 0.12, 192)
    T, q, _ = ctx.trace_inv_deflated(op, dims, W, lam, 8, 1e-12, ctx.make_opts("fp64", z0_seed=2),
                                     q_inout=np.zeros(8, dtype=np.complex128))
    ref = np.trace(np.linalg.inv(O.wilson_dense(U, dims, 0.12)))
    assert np.abs(q).max() <= 1e-9 * abs(ref)
    assert np.allclose(T, ref, rtol=1e-10, atol=0)


def test_wilson_deflation_with_library_eigenvectors(ctx, hp):
    """hp_wilson_eigs feeding hp_trace_inv_deflated gives the oracle's deflated estimate."""
    dims = (4, 4, 2, 4)
    U, op = _wilson_op(ctx, hp, dims, 45)
    ev = torch.zeros((10, 128, 4, 3), dtype=torch.complex128, device="cuda:0")
    lam, ev, _ = ctx.wilson_eigs(op, dims, 10, 1e-11, evecs=ev)
    T, q, _ = ctx.trace_inv_deflated(op, dims, ev, lam, 16, 1e-12, ctx.make_opts("fp64", z0_seed=6),
                                     q_inout=np.zeros(16, dtype=np.complex128))
    lam_o, W_o = E.wilson_lowest_eigenpairs(dims, U, 0.12, 10)
    qo, exact = E.wilson_deflated_quadratures(dims, U, 0.12, lam_o, W_o, 0, 16, 6)
    To = exact + E.trace_prefix(qo)
    assert np.abs(T - To).max() <= 1e-8 * np.abs(To).max()


def test_wilson_deflation_and_eigs_errors(ctx, hp):
    dims = (4, 4, 2, 4)
    U, op = _wilson_op(ctx, hp, dims, 46)
    lam, W = E.wilson_lowest_eigenpairs(dims, U, 0.12, 4)
    for bad_lam, opts, status in ((np.array([lam[0], 0.0, lam[2], lam[3]]), ctx.make_opts("fp64"), hp.HP_EINVAL),
                                  (lam, ctx.make_opts("fp64", first=2), hp.HP_EINVAL),
                                  (lam, ctx.make_opts("fp64", probe_kind="natural"), hp.HP_EUNSUPPORTED)):
        with pytest.raises(hp.HProbeError) as e:
            ctx.trace_inv_deflated(op, dims, W, bad_lam, 8, 1e-10, opts, q_inout=np.zeros(8, dtype=np.complex128))
        assert e.value.status == status
    lap = ctx.make_operator(hp.OP_LAPLACIAN, 0.3)
    for o, k in ((lap, 2), (op, 0), (op, 6 * 128 + 1)):
        with pytest.raises(hp.HProbeError) as e:
            ctx.wilson_eigs(o, dims, k)
        assert e.value.status == hp.HP_EINVAL


# ------------------------------------------------------------------ Wilson: singular triplets
@pytest.mark.parametrize("dims,k,mfs,csw", [((4, 4, 2, 4), 8, 0.0, 0.0), ((4, 2, 4, 2), 12, 0.02, 0.0),
                                            ((2, 4, 2, 4), 6, 0.0, 1.0)])
def test_wilson_svd_matches_the_oracle(ctx, hp, dims, k, mfs, csw):
    """Singular values within 1e-9 of the oracle's dense SVD; D v_j = sigma_j u_j by the oracle's
    stencil; both sets orthonormal.  (The residual is measured on Q^2 relative to sigma^2, about
    ||Q|| / sigma times the relative residual of the same pair of Q: 1e-9 here is ~3e-11 there.)"""
    mf = synth.mass_field(dims, mfs, 41) if mfs else None
    U, op = _wilson_op(ctx, hp, dims, 40, mass=0.01, mf=mf, csw=csw)
    sig, R, L, res = ctx.wilson_svd(op, dims, k, 1e-9)
    sig_o, _, _ = E.wilson_smallest_singular_triplets(dims, U, 0.12, k, mass=0.01, mass_field=mf, csw=csw)
    assert np.all(res <= 1e-9)
    assert np.allclose(sig, sig_o, rtol=1e-9, atol=0), (sig, sig_o)
    C = O.clover_term(U, dims, 0.12, csw) if csw else None
    for j in range(k):
        Dv = O.wilson_apply(R[j], U, dims, 0.12, 0.01, mf, clover=C)
        assert np.linalg.norm(Dv - sig[j] * L[j]) <= 1e-9 * sig[j], j
    for X in (R, L):
        G = np.einsum("ixsc,jxsc->ij", np.conj(X), X)
        assert np.allclose(G, np.eye(k), atol=1e-10)


@pytest.mark.parametrize("dims,k,s,prec,eo,device", [((4, 4, 2, 4), 8, 16, "fp64", 0, False),
                                                     ((4, 4, 2, 4), 20, 32, "fp16", 1, True),
                                                     ((6, 2, 2, 2), 6, 24, "fp64", 0, False)])
def test_wilson_svd_deflated_trace_matches_oracle(ctx, hp, dims, k, s, prec, eo, device):
    """T_s = sum_j u_j^H v_j / sigma_j + (1/s) sum_m q'_m against the oracle's dense solves with the
    left projector on the sources, within 1e-9 (complex exact part included)."""
    mf = synth.mass_field(dims, 0.01, 43)
    U, op = _wilson_op(ctx, hp, dims, 42, mf=mf)
    sig, R, L = E.wilson_smallest_singular_triplets(dims, U, 0.12, k, mass_field=mf)
    q = np.zeros(s, dtype=np.complex128)
    r, l = (_dev(R), _dev(L)) if device else (R, L)
    T, q, st = ctx.trace_inv_deflated_svd(op, dims, r, l, sig, s, 1e-12,
                                          ctx.make_opts(prec, z0_seed=5, even_odd=eo, rhs_block=24), q_inout=q)
    qo, exact = E.wilson_deflated_quadratures_svd(dims, U, 0.12, sig, R, L, 0, s, 5, mass_field=mf)
    To = exact + E.trace_prefix(qo)
    assert np.abs(q - qo).max() <= 1e-9 * np.abs(qo).max()
    assert np.abs(T - To).max() <= 1e-9 * np.abs(To).max()


def test_wilson_svd_deflation_with_library_triplets(ctx, hp):
    """hp_wilson_svd feeding hp_trace_inv_deflated_svd gives the oracle's deflated estimate, and
    the full set of triplets leaves nothing to probe."""
    dims = (4, 4, 2, 4)
    U, op = _wilson_op(ctx, hp, dims, 45)
    R = torch.zeros((10, 128, 4, 3), dtype=torch.complex128, device="cuda:0")
    L = torch.zeros_like(R)
    sig, R, L, _ = ctx.wilson_svd(op, dims, 10, 1e-10, right=R, left=L)
    T, _, _ = ctx.trace_inv_deflated_svd(op, dims, R, L, sig, 16, 1e-12, ctx.make_opts("fp64", z0_seed=6))
    s_o, R_o, L_o = E.wilson_smallest_singular_triplets(dims, U, 0.12, 10)
    qo, exact = E.wilson_deflated_quadratures_svd(dims, U, 0.12, s_o, R_o, L_o, 0, 16, 6)
    To = exact + E.trace_prefix(qo)
    assert np.abs(T - To).max() <= 1e-8 * np.abs(To).max()
    d2 = (2, 2, 2, 2)
    U2, op2 = _wilson_op(ctx, hp, d2, 46)
    s2, R2, L2 = E.wilson_smallest_singular_triplets(d2, U2, 0.12, 192)
    T2, q2, _ = ctx.trace_inv_deflated_svd(op2, d2, R2, L2, s2, 8, 1e-12, ctx.make_opts("fp64", z0_seed=2),
                                           q_inout=np.zeros(8, dtype=np.complex128))
    ref = np.trace(np.linalg.inv(O.wilson_dense(U2, d2, 0.12)))
    assert np.abs(q2).max() <= 1e-9 * abs(ref) and np.allclose(T2, ref, rtol=1e-10, atol=0)


def test_wilson_svd_at_8x8x8x8_by_the_oracle_stencil(ctx, hp):
    """The 48 triplets of the 8^4 deflation workload (kappa 0.124, eps 0.4, link seed 1004): the
    adjoint relation D^H u_j = sigma_j v_j, which the solver never forms (it returns u_j = D v_j /
    sigma_j), holds to the residual bound tol sigma_j with D^H applied by the oracle's stencil;
    D v_j = sigma_j u_j to rounding; both sets orthonormal; sigma ascending."""
    dims, k, tol = (8, 8, 8, 8), 48, 1e-9
    U = synth.gauge_links(dims, 0.4, 1004)
    op = ctx.make_operator(hp.OP_WILSON, 0.0, 0.124, _dev(U.view(np.float64).reshape(-1)), None)
    sig, R, L, res = ctx.wilson_svd(op, dims, k, tol)
    assert np.all(res <= tol) and np.all(np.diff(sig) >= 0) and sig[0] > 0
    for j in range(k):
        Dv = O.wilson_apply(R[j], U, dims, 0.124)
        assert np.linalg.norm(Dv - sig[j] * L[j]) <= 1e-12 * sig[j], j
        DHu = O.wilson_apply(L[j], U, dims, 0.124, dagger=True)
        assert np.linalg.norm(DHu - sig[j] * R[j]) <= 1.5 * tol * sig[j], j
    for X, atol in ((R, 1e-10), (L, 1e-8)):
        G = np.einsum("ixsc,jxsc->ij", np.conj(X), X)
        assert np.abs(G - np.eye(k)).max() <= atol


def test_wilson_svd_unconverged_triplets_deflate_exactly(ctx, hp):
    """After one sweep (far from tol) hp_wilson_svd's outputs are Rayleigh-Ritz triplets: D v_j =
    sigma_j u_j by the oracle's stencil and both sets orthonormal, while D^H u_j = sigma_j v_j fails;
    the deflated sequence with them matches the oracle's and reaches Tr D^-1 (dense inverse) at
    s = N."""
    dims, k, N = (4, 4, 2, 4), 8, 128
    U, op = _wilson_op(ctx, hp, dims, 48)
    with pytest.raises(hp.HProbeError) as e:
        ctx.wilson_svd(op, dims, k, 1e-12, max_sweeps=1)
    assert e.value.status == hp.HP_ENOCONV
    sig, R, L, res = ctx.wilson_svd(op, dims, k, 1e-12, max_sweeps=1, check=False)
    assert res.max() > 1e-6 and np.all(sig > 0)
    off = 0.0
    for j in range(k):
        assert np.linalg.norm(O.wilson_apply(R[j], U, dims, 0.12) - sig[j] * L[j]) <= 1e-12 * sig[j], j
        off = max(off, np.linalg.norm(O.wilson_apply(L[j], U, dims, 0.12, dagger=True) - sig[j] * R[j]))
    assert off > 1e-6
    for X in (R, L):
        G = np.einsum("ixsc,jxsc->ij", np.conj(X), X)
        assert np.abs(G - np.eye(k)).max() <= 1e-10
    T, q, _ = ctx.trace_inv_deflated_svd(op, dims, R, L, sig, N, 1e-12, ctx.make_opts("fp64", z0_seed=8),
                                         q_inout=np.zeros(N, dtype=np.complex128))
    qo, exact = E.wilson_deflated_quadratures_svd(dims, U, 0.12, sig, R, L, 0, 16, 8)
    To = exact + E.trace_prefix(qo)
    assert np.abs(T[:16] - To).max() <= 1e-9 * np.abs(To).max()
    ref = np.trace(np.linalg.inv(O.wilson_dense(U, dims, 0.12)))
    assert abs(T[-1] - ref) <= 1e-9 * abs(ref)


def test_wilson_svd_errors(ctx, hp):
    dims = (4, 4, 2, 4)
    U, op = _wilson_op(ctx, hp, dims, 47)
    sig, R, L = E.wilson_smallest_singular_triplets(dims, U, 0.12, 4)
    bad = sig.copy()
    bad[2] = 0.0
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_deflated_svd(op, dims, R, L, bad, 8, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EINVAL
    with pytest.raises(ValueError):
        ctx.trace_inv_deflated_svd(op, dims, R, L[:2], sig, 8, 1e-10, ctx.make_opts("fp64"))
    lap = ctx.make_operator(hp.OP_LAPLACIAN, 0.3)
    with pytest.raises(hp.HProbeError) as e:
        ctx.wilson_svd(lap, dims, 2)
    assert e.value.status == hp.HP_EINVAL
    d4 = (4, 4, 4, 4)   # k above the cap of 1024, below 6 V = 1536 (rejected before the links are read)
    op4 = ctx.make_operator(hp.OP_WILSON, 0.0, 0.12, torch.zeros(256 * 72, dtype=torch.float64, device="cuda:0"))
    for fn in (ctx.wilson_svd, ctx.wilson_eigs):
        with pytest.raises(hp.HProbeError) as e:
            fn(op4, d4, 1025)
        assert e.value.status == hp.HP_EINVAL
