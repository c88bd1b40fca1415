"""Statistical equivalence of two simulations, as the paper validates its
simulator against a reference (Sec. 3.1).

For every population, three distributions are taken from the recorded spike
trains (after a discarded transient):

* the firing rate of each neuron;
* the coefficient of variation of each neuron's inter-spike intervals
  (standard deviation / mean; neurons with at least two intervals);
* the Pearson correlation coefficients between the spike trains of a subset
  of neurons (200 by default), binned at 2 ms (the refractory time): the
  off-diagonal elements of their correlation matrix.

Each distribution is smoothed by a Gaussian kernel density estimate whose
bandwidth follows Silverman's rule, b = 0.9 min(sigma, IQR / 1.349) N^(-1/5),
and two simulations are compared by the Kullback-Leibler divergence of their
densities on a common grid, sum p1 log(p1 / p2) (the paper prints a leading
minus sign; the divergence it evaluates, with scipy's entropy function, is
this non-negative sum).  Comparing a simulation with the reference and the
reference with itself under other seeds tells whether the two agree as well
as two runs of the reference do.

Host-side analysis with numpy only; spike trains come from ngb_get_spikes
(or any source giving (neuron, step) pairs).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def silverman_bandwidth(x: np.ndarray) -> float:
    """Silverman's rule of thumb: 0.9 min(sigma, IQR / 1.349) N^(-1/5)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        return 1.0
    sigma = x.std(ddof=1)
    q75, q25 = np.percentile(x, [75.0, 25.0])
    spread = min(sigma, (q75 - q25) / 1.349)
    if not spread > 0:
        spread = sigma if sigma > 0 else 1.0
    return 0.9 * spread * n ** (-0.2)


def kde(x: np.ndarray, grid: np.ndarray, bandwidth: Optional[float] = None) -> np.ndarray:
    """Gaussian kernel density estimate of samples x on `grid`: the mean of
    unit-area Gaussians of width `bandwidth` (Silverman's rule by default)
    centred on the samples."""
    x = np.asarray(x, dtype=np.float64)
    grid = np.asarray(grid, dtype=np.float64)
    b = silverman_bandwidth(x) if bandwidth is None else bandwidth
    out = np.zeros_like(grid)
    for lo in range(0, x.size, 4096):  # blocks of samples, to bound the temporary
        z = (grid[:, None] - x[None, lo:lo + 4096]) / b
        out += np.exp(-0.5 * z * z).sum(axis=1)
    return out / (x.size * b * np.sqrt(2.0 * np.pi))


def kl_divergence(p1: np.ndarray, p2: np.ndarray, eps: float = 1e-300) -> float:
    """sum_i p1_i log(p1_i / p2_i) of two densities sampled on the same grid,
    each normalised to unit sum first."""
    p1 = np.asarray(p1, dtype=np.float64)
    p2 = np.asarray(p2, dtype=np.float64)
    p1 = p1 / p1.sum()
    p2 = p2 / p2.sum()
    m = p1 > 0
    q = p2[m]
    return float(np.sum(p1[m] * np.log(p1[m] / np.where(q > 0, q, eps))))


def firing_rates(ids: np.ndarray, steps: np.ndarray, lo: int, hi: int, t0: int, t1: int, dt_ms: float) -> np.ndarray:
    """Rate (Hz) of each neuron in [lo, hi) over steps [t0, t1)."""
    m = (ids >= lo) & (ids < hi) & (steps >= t0) & (steps < t1)
    cnt = np.bincount(ids[m] - lo, minlength=hi - lo)
    return cnt / ((t1 - t0) * dt_ms * 1e-3)


def cv_isi(ids: np.ndarray, steps: np.ndarray, lo: int, hi: int, t0: int, t1: int) -> np.ndarray:
    """CV of the inter-spike intervals of each neuron in [lo, hi) with at
    least two intervals in steps [t0, t1)."""
    m = (ids >= lo) & (ids < hi) & (steps >= t0) & (steps < t1)
    i, s = ids[m], steps[m]
    order = np.lexsort((s, i))
    i, s = i[order], s[order]
    out = []
    starts = np.flatnonzero(np.r_[True, i[1:] != i[:-1]])
    ends = np.r_[starts[1:], i.size]
    for a, b in zip(starts, ends):
        if b - a >= 3:
            isi = np.diff(s[a:b]).astype(np.float64)
            out.append(isi.std() / isi.mean())
    return np.array(out)


def pearson_correlations(ids: np.ndarray, steps: np.ndarray, neurons: Sequence[int], t0: int, t1: int,
                         bin_steps: int) -> np.ndarray:
    """Off-diagonal Pearson correlation coefficients of the spike trains of
    `neurons`, binned at `bin_steps` steps over [t0, t1).  Trains without a
    spike (zero variance) are left out."""
    neurons = np.asarray(neurons)
    nb = (t1 - t0) // bin_steps
    pos = {int(n): k for k, n in enumerate(neurons)}
    B = np.zeros((len(neurons), nb))
    m = (steps >= t0) & (steps < t0 + nb * bin_steps) & np.isin(ids, neurons)
    for n, s in zip(ids[m], steps[m]):
        B[pos[int(n)], (s - t0) // bin_steps] += 1.0
    B -= B.mean(axis=1, keepdims=True)
    norm = np.sqrt((B * B).sum(axis=1))
    keep = norm > 0
    B = B[keep] / norm[keep][:, None]
    C = B @ B.T
    return C[~np.eye(C.shape[0], dtype=bool)]


def population_statistics(ids: np.ndarray, steps: np.ndarray, bounds: Sequence[int], t0: int, t1: int,
                          dt_ms: float, n_corr: int = 200, bin_ms: float = 2.0,
                          seed: int = 0) -> List[Dict[str, np.ndarray]]:
    """The three distributions of every population [bounds[k], bounds[k+1])."""
    rng = np.random.default_rng(seed)
    out = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        sub = np.sort(rng.choice(np.arange(lo, hi), size=min(n_corr, hi - lo), replace=False))
        out.append({"rate": firing_rates(ids, steps, lo, hi, t0, t1, dt_ms),
                    "cv_isi": cv_isi(ids, steps, lo, hi, t0, t1),
                    "corr": pearson_correlations(ids, steps, sub, t0, t1, max(1, int(round(bin_ms / dt_ms))))})
    return out


def _grid(a: np.ndarray, b: np.ndarray, n: int = 512) -> np.ndarray:
    lo = min(a.min(initial=0.0), b.min(initial=0.0))
    hi = max(a.max(initial=1.0), b.max(initial=1.0))
    pad = 0.1 * (hi - lo) + 1e-9
    return np.linspace(lo - pad, hi + pad, n)


def compare(stats_a: List[Dict[str, np.ndarray]],
            stats_b: List[Dict[str, np.ndarray]]) -> List[Dict[str, float]]:
    """KL divergence of the smoothed distributions of run a from those of run
    b, per population and statistic (nan where a distribution has fewer than
    two samples)."""
    res = []
    for sa, sb in zip(stats_a, stats_b):
        row = {}
        for key in ("rate", "cv_isi", "corr"):
            a, b = sa[key], sb[key]
            if a.size < 2 or b.size < 2:
                row[key] = float("nan")
                continue
            g = _grid(a, b)
            row[key] = kl_divergence(kde(a, g), kde(b, g))
        res.append(row)
    return res


def mean_std(values: Sequence[List[Dict[str, float]]]) -> List[Dict[str, Tuple[float, float]]]:
    """Mean and standard deviation over pairs of runs, per population and statistic."""
    out = []
    for k in range(len(values[0])):
        row = {}
        for key in ("rate", "cv_isi", "corr"):
            v = np.array([pair[k][key] for pair in values])
            v = v[np.isfinite(v)]
            row[key] = (float(v.mean()) if v.size else float("nan"), float(v.std()) if v.size else float("nan"))
        out.append(row)
    return out
