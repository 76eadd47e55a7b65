"""The variance-study statistics of the package (Sections 5.2, 5.3) against the oracle's plain
definitions, on synthetic estimate tables.  No GPU."""
import numpy as np

from oracle import estimator as E
from paper_1302_4018_gb300 import study


def _table(seed, n=23, S=9, complex_=False):
    rng = np.random.default_rng(seed)
    T = rng.normal(5.0, 1.0, (n, S)) / np.sqrt(np.arange(1, S + 1))[None, :] ** 1.3
    if complex_:
        T = T + 1j * rng.normal(0, 0.01, (n, S))
    return T


def test_speedup_ratio_matches_the_oracle():
    for cplx in (False, True):
        T = _table(1, complex_=cplx)
        assert np.allclose(study.speedup_ratio(T), E.speedup_ratio(T), rtol=1e-12)
        assert np.allclose(study.variance_over_runs(T),
                           [E.sample_variance(T[:, s]) for s in range(T.shape[1])], rtol=1e-12)


def test_jackknife_errors_match_the_oracle():
    T = _table(2, complex_=True)
    full, err = study.jackknife_speedup(T)
    for s in range(T.shape[1]):
        f, e = E.jackknife(T, lambda a, s=s: E.speedup_ratio(a[:, :s + 1])[s])
        assert abs(full[s] - f) <= 1e-12 * abs(f)
        assert abs(err[s] - e) <= 1e-9 * abs(e) + 1e-15
    v, ev = study.jackknife_variance(T)
    for s in (0, 4, 8):
        f, e = E.jackknife(T[:, s], lambda a: E.sample_variance(a))
        assert abs(v[s] - f) <= 1e-12 * f and abs(ev[s] - e) <= 1e-9 * e


def test_z2_interval_is_twice_the_standard_error():
    q = np.random.default_rng(5).normal(3.0, 2.0, 50)
    w = study.z2_interval(q)
    assert np.isnan(w[0])
    for s in (2, 10, 50):
        assert abs(w[s - 1] - 2 * np.sqrt(E.sample_variance(q[:s]) / s)) <= 1e-12 * w[s - 1]
