"""Hierarchical probing of general sparse matrices (Algorithm 1, Section 2.2) on the GPU vs the oracle.

The colouring is integer work and compared bit for bit: the GPU's level-parallel
Jones-Plassmann rounds with the row index as priority reproduce the sequential
greedy colouring of every block, so every row's colour path must equal the
oracle's.  The probe phases are compared bit for bit (up to the common period);
the quadratures within 1e-9 relative (CG to a true residual of 1e-12 on
matrices with ||A^-1|| <= 10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")

from oracle import probing as Pr
from oracle import sparse_probing as S
from paper_1302_4018_gb300 import synth

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


def _pattern(name):
    if name == "ring64":
        return synth.grid_matrix((64,), 1, renumber=False)[:2]
    if name == "torus16":
        return synth.grid_matrix((16, 16), 2, renumber=False)[:2]
    if name == "grid6_renumbered":
        return synth.grid_matrix((6, 6, 6), 3)[:2]
    if name == "grid28_renumbered":   # 21952 rows: several scan tiles, thousands of blocks
        return synth.grid_matrix((28, 28, 28), 4)[:2]
    if name == "lattice4d_5":
        return synth.grid_matrix((5, 5, 5, 5), 5, renumber=False)[:2]
    if name == "random400":
        return synth.random_graph_matrix(400, 3, 6)[:2]
    if name == "nonsym300":
        return synth.random_pattern(300, 3, 7, symmetric=False, diagonal=True)
    if name == "nonsym_nodiag":
        return synth.random_pattern(200, 2, 8, symmetric=False, diagonal=False)
    if name == "diagonal50":
        return synth.csr_from_entries(50, np.arange(50), np.arange(50))
    if name in ("dense20", "dense100"):   # dense100: colours beyond the first window of 64
        n = int(name[5:])
        i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        return synth.csr_from_entries(n, i.ravel(), j.ravel())
    if name == "empty_rows":
        r = np.array([0, 3, 3, 7, 12, 12, 20, 29])
        c = np.array([3, 0, 7, 3, 20, 29, 12, 12])
        return synth.csr_from_entries(30, r, c)
    if name == "single":
        return synth.csr_from_entries(1, [0], [0])
    if name == "single_empty":
        return np.zeros(2, dtype=np.int32), np.zeros(0, dtype=np.int32)
    raise KeyError(name)


CASES = ["ring64", "torus16", "grid6_renumbered", "grid28_renumbered", "lattice4d_5", "random400", "nonsym300",
         "nonsym_nodiag", "diagonal50", "dense20", "dense100", "empty_rows", "single", "single_empty"]


def _oracle_levels(offsets, max_levels):
    return min(max(lv for (_, _, lv) in offsets), max_levels)


def _check_against_oracle(ctx, rp, ci, max_levels, device):
    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    operm, offsets, opaths = S.hierarchical_coloring(A, max_levels=max_levels)
    if device:
        rp_d, ci_d = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
        out = torch.full((max_levels, n), -7, dtype=torch.int32, device="cuda:0")
        paths, rad = ctx.sparse_coloring(rp_d, ci_d, max_levels, paths_out=out)
        paths = paths.cpu().numpy()
        full = out.cpu().numpy()
    else:
        paths, rad = ctx.sparse_coloring(rp, ci, max_levels)
        full = None
    nlev = paths.shape[0]
    assert nlev == _oracle_levels(offsets, max_levels)
    assert np.array_equal(paths, opaths[:, :nlev].T)
    assert not opaths[:, nlev:].any()
    assert rad == [int(opaths[:, l].max()) + 1 for l in range(nlev)]
    if full is not None:
        assert not full[nlev:].any()
    # Algorithm 1's perm and colorOffsets from the GPU's paths, on the GPU (device arrays when the
    # colouring ran on device arrays)
    if device:
        perm_d = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
        offs_d = torch.full((2 * n - 1, 3), -1, dtype=torch.int32, device="cuda:0")
        perm, offs = ctx.sparse_ordering(out[:nlev], perm_d, offs_d)
        perm, offs = perm.cpu().numpy(), offs.cpu().numpy()
    else:
        perm, offs = ctx.sparse_ordering(np.ascontiguousarray(paths))
    assert np.array_equal(perm, operm)
    assert [tuple(int(v) for v in o) for o in offs] == [tuple(o) for o in offsets]
    return paths, rad


@pytest.mark.parametrize("name", CASES)
def test_sparse_coloring_bit_exact(ctx, name):
    rp, ci = _pattern(name)
    _check_against_oracle(ctx, rp, ci, 32, device=(name in ("grid28_renumbered", "random400")))


@pytest.mark.parametrize("max_levels", [1, 2, 3])
def test_sparse_coloring_max_levels(ctx, max_levels):
    rp, ci = _pattern("grid6_renumbered")
    _check_against_oracle(ctx, rp, ci, max_levels, device=False)


def test_sparse_ordering_properties_and_errors(ctx, hp):
    """perm is a permutation that makes A(perm, perm) block diagonal per colour of level 1; every
    recorded block lies inside its parent; a colour beyond its block and a short offsets array fail."""
    rp, ci = _pattern("grid28_renumbered")
    n = len(rp) - 1
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    perm, offs = ctx.sparse_ordering(np.ascontiguousarray(paths))
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.all(np.diff(paths[0][perm]) >= 0)   # level-1 colours in ascending runs
    starts = {(int(s), int(lv)): int(e) for s, e, lv in offs}
    for s, e, lv in offs:
        if lv > 1:   # the enclosing block of the level above
            parent = [(ps, pe) for (ps, plv), pe in starts.items() if plv == lv - 1 and ps <= s and e <= pe]
            assert len(parent) == 1
    bad = np.ascontiguousarray(paths.copy())
    bad[0, 5] = n + 3
    with pytest.raises(hp.HProbeError) as e:
        ctx.sparse_ordering(bad)
    assert e.value.status == hp.HP_EINVAL
    short = np.zeros((3, 3), dtype=np.int32)
    with pytest.raises(hp.HProbeError) as e:
        ctx.sparse_ordering(np.ascontiguousarray(paths), offsets_out=short)
    assert e.value.status == hp.HP_EINVAL and "offsets_cap" in str(e.value)


def test_sparse_coloring_rerun_same_context(ctx):
    """Workspace reuse: a large run, then a small one, then the large again."""
    for name in ("grid28_renumbered", "ring64", "grid28_renumbered"):
        rp, ci = _pattern(name)
        _check_against_oracle(ctx, rp, ci, 32, device=False)


@pytest.mark.parametrize("name,first,count,z0", [("grid6_renumbered", 0, 216, 0), ("grid6_renumbered", 37, 100, 91),
                                                  ("random400", 0, 400, 17), ("diagonal50", 0, 1, 5)])
def test_sparse_probe_phases_bit_exact(ctx, name, first, count, z0):
    rp, ci = _pattern(name)
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    gam = int(np.prod(rad))
    count = min(count, gam - first)
    out = torch.empty(count * paths.shape[1], dtype=torch.int16, device="cuda:0")
    P = ctx.sparse_probe_vectors(np.ascontiguousarray(paths), rad, first, count, z0, out)
    got = out.cpu().numpy().view(np.uint16).astype(np.int64).reshape(count, -1)
    ph, Po = S.path_phases(np.ascontiguousarray(paths.T), first, count, z0)
    assert Po % P == 0
    assert np.array_equal(got * (Po // P), ph)


def _spd(name):
    if name == "random400":
        return synth.random_graph_matrix(400, 3, 21, shift=0.5)
    if name == "grid6_renumbered":
        return synth.grid_matrix((6, 6, 6), 22, shift=0.3)
    if name == "grid12x10":
        return synth.grid_matrix((12, 10), 23, shift=0.2)
    raise KeyError(name)


@pytest.mark.parametrize("name,s_max,z0", [("random400", 96, 31), ("grid6_renumbered", 216, 0),
                                           ("grid12x10", 120, 33)])
def test_sparse_trace_parity(ctx, hp, name, s_max, z0):
    rp, ci, val = _spd(name)
    n = len(rp) - 1
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    gam = int(np.prod(rad))
    s_max = min(s_max, gam, n)
    q = np.zeros(s_max, dtype=np.complex128)
    T, q, st = ctx.trace_inv_sparse(rp, ci, val, np.ascontiguousarray(paths), rad, s_max, 1e-12,
                                    ctx.make_opts("fp64", z0_seed=z0), q_inout=q)
    A = sp.csr_matrix((val, ci, rp), shape=(n, n))
    qo = S.sparse_quadratures(A, np.ascontiguousarray(paths.T), 0, s_max, z0)
    scale = np.abs(qo).max()
    assert np.abs(q - qo).max() <= 1e-9 * scale
    To = np.cumsum(qo) / np.arange(1, s_max + 1)
    assert np.abs(T - To).max() <= 1e-9 * np.abs(To).max()
    assert st["rhs_solved"] >= s_max


@pytest.mark.parametrize("prec,rhs_block", [("fp64", 64), ("fp64", 128), ("fp32", 0), ("fp32", 64), ("fp32", 128)])
def test_sparse_trace_blocks_and_mixed_precision(ctx, prec, rhs_block):
    """Every block size of the blocked CG, in FP64 and with FP32 iteration + FP64 reliable
    updates: the certified true residual gives the same quadratures."""
    rp, ci, val = _spd("random400")
    n = len(rp) - 1
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    s_max = 96
    q = np.zeros(s_max, dtype=np.complex128)
    T, q, st = ctx.trace_inv_sparse(rp, ci, val, np.ascontiguousarray(paths), rad, s_max, 1e-12,
                                    ctx.make_opts(prec, z0_seed=5, rhs_block=rhs_block), q_inout=q)
    A = sp.csr_matrix((val, ci, rp), shape=(n, n))
    qo = S.sparse_quadratures(A, np.ascontiguousarray(paths.T), 0, s_max, 5)
    assert np.abs(q - qo).max() <= 1e-9 * np.abs(qo).max()
    assert st["max_true_residual"] <= 1e-12
    if prec == "fp32":
        assert st["reliable_updates"] >= st["rhs_solved"]   # at least the final FP64 check per solve


def test_sparse_trace_device_inputs_and_restart(ctx):
    """Device CSR and paths; first > 0 continues from earlier quadratures."""
    rp, ci, val = _spd("random400")
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    P = np.ascontiguousarray(paths)
    q_full = np.zeros(64, dtype=np.complex128)
    T_full, _, _ = ctx.trace_inv_sparse(rp, ci, val, P, rad, 64, 1e-12, ctx.make_opts("fp64", z0_seed=3),
                                        q_inout=q_full)
    q = np.zeros(64, dtype=np.complex128)
    q[:20] = q_full[:20]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    T, q, _ = ctx.trace_inv_sparse(d(rp), d(ci), d(val), d(P), rad, 64, 1e-12,
                                   ctx.make_opts("fp64", z0_seed=3, first=20), q_inout=q)
    assert np.abs(q - q_full).max() <= 1e-9 * np.abs(q_full).max()
    assert np.abs(T - T_full).max() <= 1e-9 * np.abs(T_full).max()


@pytest.mark.parametrize("kind", ["natural", "z2"])
def test_sparse_trace_comparison_sequences(ctx, kind):
    rp, ci, val = synth.grid_matrix((16, 16), 24, shift=0.4)   # n = 256: natural order needs 2^k
    n = len(rp) - 1
    s = 40
    q = np.zeros(s, dtype=np.complex128)
    T, q, _ = ctx.trace_inv_sparse(rp, ci, val, None, [], s, 1e-12,
                                   ctx.make_opts("fp64", z0_seed=77, probe_kind=kind), q_inout=q)
    if kind == "natural":
        ph = Pr.probe_phases_natural(n, 0, s, 77)
    else:
        ph = Pr.probe_phases_z2(n, 0, s, 77)
    A = sp.csr_matrix((val, ci, rp), shape=(n, n))
    qo = S.quadratures_of_phases(A, np.asarray(ph), 2)
    assert np.abs(q - qo).max() <= 1e-9 * np.abs(qo).max()


def test_sparse_errors(ctx, hp):
    rp, ci, val = _spd("grid6_renumbered")
    paths, rad = ctx.sparse_coloring(rp, ci, 32)
    P = np.ascontiguousarray(paths)
    bad_ci = ci.copy()
    bad_ci[5] = len(rp) + 3
    with pytest.raises(hp.HProbeError) as e:
        ctx.sparse_coloring(rp, bad_ci, 32)
    assert e.value.status == hp.HP_EINVAL
    bad_rp = rp.copy()
    bad_rp[10] = bad_rp[12] + 1
    with pytest.raises(hp.HProbeError) as e:
        ctx.sparse_coloring(bad_rp, ci, 32)
    assert e.value.status == hp.HP_EINVAL
    with pytest.raises(hp.HProbeError) as e:   # more vectors than the first level resolves
        ctx.trace_inv_sparse(rp, ci, val, P[:1], rad[:1], rad[0] + 1, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EUNSUPPORTED
    bad_p = P.copy()
    bad_p[0, 3] = rad[0]
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_sparse(rp, ci, val, bad_p, rad, 8, 1e-10, ctx.make_opts("fp64"))
    assert e.value.status == hp.HP_EINVAL
    with pytest.raises(hp.HProbeError) as e:
        ctx.trace_inv_sparse(rp, ci, val, P, rad, 8, 1e-10, ctx.make_opts("fp16"))
    assert e.value.status == hp.HP_EUNSUPPORTED
