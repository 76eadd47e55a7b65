"""Statistics of the variance studies of Sections 5.2 and 5.3 (host logic on the estimates T_s the
library returns; no solver work here).

* variance over runs: the spread of T_s over n runs that differ only in the bias-removal vector
  z_0 (Section 5.2: 100 vectors z_0, confidence intervals +-2 sigma around the mean);
* speed-up ratio (Section 5.3): R_s = V_stoc / (V_hp(s) s), V_hp(s) the variance of T_s over the
  runs and V_stoc that of the standard Z_2 estimator with one vector, by default V_hp(1) (the
  first probing vector is z_0 (.) h_0 = z_0, a Z_2 noise vector), with delete-one jackknife errors
  over the runs;
* the Z_2 estimator's own interval (Section 5.2): +-2 (Var / s)^{1/2} with Var the sample variance
  of its first s quadratures.

Complex estimates use |x - mean|^2.  The leave-one-out moments are updated from running sums, so
the jackknife over n runs costs O(n S), not O(n^2 S).
"""
from __future__ import annotations

import numpy as np


def _moments(T: np.ndarray):
    T = np.asarray(T)
    return T.shape[0], T.sum(axis=0), (np.abs(T) ** 2).sum(axis=0)


def variance_over_runs(T: np.ndarray) -> np.ndarray:
    """Unbiased variance over the rows of T[run, s - 1] for every s."""
    n, S1, S2 = _moments(T)
    return (S2 - np.abs(S1) ** 2 / n) / (n - 1)


def _loo_variances(T: np.ndarray) -> np.ndarray:
    """[n, S]: the variance of each column with run i left out."""
    T = np.asarray(T)
    n, S1, S2 = _moments(T)
    S1i = S1[None, :] - T
    S2i = S2[None, :] - np.abs(T) ** 2
    return (S2i - np.abs(S1i) ** 2 / (n - 1)) / (n - 2)


def speedup_ratio(T: np.ndarray, v_stoc: float | None = None) -> np.ndarray:
    """R_s = V_stoc / (V_hp(s) s), s = 1..S (columns of T)."""
    v = variance_over_runs(T)
    s = np.arange(1, v.shape[0] + 1)
    return (v[0] if v_stoc is None else v_stoc) / (v * s)


def jackknife_speedup(T: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(R_s over all runs, its delete-one jackknife error) with V_stoc = V_hp(1) of the same runs."""
    T = np.asarray(T)
    n = T.shape[0]
    if n < 3:
        raise ValueError("the jackknife of a variance needs at least 3 runs")
    full = speedup_ratio(T)
    loo = _loo_variances(T)
    s = np.arange(1, T.shape[1] + 1)
    r = loo[:, :1] / (loo * s[None, :])
    m = r.mean(axis=0)
    err = np.sqrt((n - 1) / n * ((r - m[None, :]) ** 2).sum(axis=0))
    return full, err


def jackknife_variance(T: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(V_hp(s), its delete-one jackknife error)."""
    T = np.asarray(T)
    n = T.shape[0]
    loo = _loo_variances(T)
    m = loo.mean(axis=0)
    return variance_over_runs(T), np.sqrt((n - 1) / n * ((loo - m[None, :]) ** 2).sum(axis=0))


def z2_interval(q: np.ndarray) -> np.ndarray:
    """Half width of the Z_2 estimator's interval after s vectors: 2 (Var_s / s)^{1/2}, Var_s the
    sample variance of its first s quadratures (undefined, NaN, for s = 1)."""
    q = np.asarray(q)
    out = np.full(q.shape[0], np.nan)
    c1 = np.cumsum(q)
    c2 = np.cumsum(np.abs(q) ** 2)
    s = np.arange(1, q.shape[0] + 1)
    ok = s > 1
    var = (c2[ok] - np.abs(c1[ok]) ** 2 / s[ok]) / (s[ok] - 1)
    out[ok] = 2.0 * np.sqrt(var / s[ok])
    return out
