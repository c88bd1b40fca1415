"""Pins of the statistical-equivalence tools (the paper's validation method,
Sec. 3.1) -- CPU only.

* Gaussian KDE equals scipy.stats.gaussian_kde at the same bandwidth, and
  integrates to one.
* Silverman's bandwidth: 0.9 sigma N^-1/5 for normal samples (IQR / 1.349 ~
  sigma there); the IQR term takes over for heavy tails.
* KL divergence of two sampled normal densities equals the closed form
  ln(s2/s1) + (s1^2 + (m1 - m2)^2) / (2 s2^2) - 1/2.
* CV of inter-spike intervals: 0 for a regular train, 1 for a Poisson train.
* Pearson correlations equal numpy's corrcoef of the binned trains.
* Two oracle runs of the same network with different seeds give small but
  non-zero divergences; a run compared with itself gives zero.
"""
import numpy as np
import pytest

import oracle
from paper_2007_14236_gb300 import validate as V
from paper_2007_14236_gb300 import workloads as W

stats = pytest.importorskip("scipy.stats")


def test_kde_matches_scipy_and_integrates_to_one():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 700), rng.normal(4, 0.5, 300)])
    b = V.silverman_bandwidth(x)
    grid = np.linspace(-6, 9, 3001)
    ours = V.kde(x, grid)
    ref = stats.gaussian_kde(x, bw_method=b / x.std(ddof=1))(grid)
    assert np.allclose(ours, ref, rtol=1e-10, atol=1e-14)
    assert abs(np.trapezoid(ours, grid) - 1.0) < 1e-6


def test_silverman_bandwidth_normal_and_heavy_tails():
    rng = np.random.default_rng(2)
    x = rng.normal(3.0, 2.0, 200_000)
    b = V.silverman_bandwidth(x)
    assert abs(b / (0.9 * 2.0 * x.size ** -0.2) - 1.0) < 0.01
    t = rng.standard_t(1.5, 200_000)  # heavy tails: sigma >> IQR / 1.349
    q75, q25 = np.percentile(t, [75, 25])
    assert V.silverman_bandwidth(t) < 0.9 * t.std(ddof=1) * t.size ** -0.2
    assert abs(V.silverman_bandwidth(t) / (0.9 * (q75 - q25) / 1.349 * t.size ** -0.2) - 1) < 1e-12


def test_kl_divergence_of_normals_closed_form():
    m1, s1, m2, s2 = 0.0, 1.0, 0.5, 1.5
    grid = np.linspace(-15, 15, 200_001)
    p1 = stats.norm.pdf(grid, m1, s1)
    p2 = stats.norm.pdf(grid, m2, s2)
    exact = np.log(s2 / s1) + (s1 ** 2 + (m1 - m2) ** 2) / (2 * s2 ** 2) - 0.5
    assert abs(V.kl_divergence(p1, p2) - exact) < 1e-6
    assert V.kl_divergence(p1, p1) == 0.0


def test_cv_isi_regular_and_poisson():
    steps = np.arange(0, 100_000, 10)
    ids = np.zeros_like(steps)
    assert V.cv_isi(ids, steps, 0, 1, 0, 100_000)[0] == 0.0
    rng = np.random.default_rng(3)
    st = np.cumsum(rng.geometric(0.01, 200_000))  # Bernoulli process: ISI CV sqrt(1 - p) ~ 1
    cv = V.cv_isi(np.zeros_like(st), st, 0, 1, 0, int(st[-1]) + 1)[0]
    assert abs(cv - np.sqrt(1 - 0.01)) < 0.01
    # rates: spikes per second
    r = V.firing_rates(np.array([0, 0, 1, 2, 2, 2]), np.array([1, 5, 3, 2, 4, 9]), 0, 4, 0, 10, 0.1)
    assert np.allclose(r, [2000.0, 1000.0, 3000.0, 0.0])


def test_pearson_matches_corrcoef():
    rng = np.random.default_rng(4)
    n, T, bins = 12, 20_000, 20
    common = rng.random(T) < 0.01
    ids, steps = [], []
    for k in range(n):
        s = np.flatnonzero(common & (rng.random(T) < 0.5) | (rng.random(T) < 0.005))
        ids.append(np.full(s.size, 100 + k))
        steps.append(s)
    ids, steps = np.concatenate(ids), np.concatenate(steps)
    c = V.pearson_correlations(ids, steps, np.arange(100, 100 + n), 0, T, bins)
    B = np.zeros((n, T // bins))
    np.add.at(B, (ids - 100, steps // bins), 1.0)
    ref = np.corrcoef(B)[~np.eye(n, dtype=bool)]
    assert np.allclose(c, ref, atol=1e-12)
    assert c.mean() > 0.1  # the shared component correlates the trains


def test_oracle_runs_compare_small_and_self_zero():
    stats_runs = []
    for seed in (1, 2):
        spec = W.microcircuit(scale=0.03, seed=seed, keep_indegree=False)
        net = oracle.OracleNet(spec)
        net.finalize()
        net.simulate(3000)
        ids, st = net.spikes()
        bounds = np.cumsum([0] + [p.n for p in spec.pops])
        stats_runs.append(V.population_statistics(ids, st, bounds, 1000, 3000, spec.dt, n_corr=50))
    same = V.compare(stats_runs[0], stats_runs[0])
    assert all(v == 0.0 for row in same for v in row.values() if np.isfinite(v))
    cross = V.compare(stats_runs[0], stats_runs[1])
    vals = np.array([v for row in cross for v in row.values() if np.isfinite(v)])
    assert vals.size >= 16 and np.all(vals >= 0) and np.median(vals) < 1.0
