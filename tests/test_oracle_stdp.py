"""Pins of the oracle's nearest-neighbour STDP (Sec. 2.1; Morrison et al.
2008 pairing, Guetig et al. 2003 weight dependence) -- CPU only.

* One pre-post pair and one post-pre pair on a single synapse, spikes forced
  by injected current: the weight change equals the closed form
  lambda W_max (1 - w/W_max)^mu+ e^(-lag/tau+) (potentiation) or
  -alpha lambda W_max (w/W_max)^mu- e^(-lag/tau-) (depression), with the lag
  measured from the spike's arrival (firing step + delay); multiplicative,
  additive and fractional exponents.
* The weight a spike delivers is the weight after the depression of its
  arrival.
* Nearest-neighbour pairing on Poisson-driven spike trains (additive rule,
  no clipping): every synapse's final weight equals its initial weight plus
  the pair sums computed from the recorded spike lists by brute force (each
  post spike with the latest arrival at or before it, each arrival with the
  latest post spike strictly before it).  All-pairs summation would differ.
* Clipping: weights stay in [0, W_max] and reach both bounds under a large
  learning rate.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_14236_gb300 import workloads as W

DT = 0.1
KICK = 1.0e5  # pA: an input that makes a resting LIF neuron fire at the next step


def _pair_spec(w0, stdp, delay_ms=1.5):
    lif = W.LifParams(tau_m=10.0, C_m=250.0, E_L=-65.0, V_reset=-65.0, V_th=-50.0, t_ref=2.0, tau_syn=0.5,
                      V_init_mean=-65.0, V_init_sd=0.0)
    spec = W.NetSpec(name="stdp_pair", seeds=[1])
    spec.pops = [W.Population("pre", W.LIF, 1, lif), W.Population("post", W.LIF, 1, lif)]
    spec.conns = [W.Connection(0, 1, W.ONE_TO_ONE, 0, W.Dist("const", w0), W.Dist("const", delay_ms), stdp=stdp)]
    return spec


def _run_forced(spec, spikes_at, steps):
    """Simulate, making neuron i fire at each step of spikes_at[i]."""
    o = oracle.OracleNet(spec)
    o.finalize()
    weights = []
    for t in range(steps):
        for i, sts in spikes_at.items():
            if t + 1 in sts:
                o.inject(i, 0, 0, KICK)  # enters I at step t, V crosses at step t + 1
        o.simulate(1)
        weights.append(float(o.csr()["weight"][0]))
    ids, st = o.spikes()
    for i, sts in spikes_at.items():
        assert list(st[ids == i]) == sorted(sts), (i, st[ids == i])
    return o, np.array(weights)


@pytest.mark.parametrize("mu", [1.0, 0.0, 0.4])
def test_single_pre_post_pair_potentiates_by_closed_form(mu):
    q = W.Stdp(tau_plus=17.0, tau_minus=34.0, lam=0.05, alpha=1.2, mu_plus=mu, mu_minus=mu, W_max=100.0)
    w0 = 40.0
    # pre fires at step 10, arrives at step 25 (delay 15 steps); post fires at step 40
    o, w = _run_forced(_pair_spec(w0, q), {0: [10], 1: [40]}, 60)
    lag_ms = (40 - 25) * DT
    expect = w0 + q.lam * q.W_max * (1.0 - w0 / q.W_max) ** mu * math.exp(-lag_ms / q.tau_plus)
    assert np.all(w[:40] == np.float32(w0))  # no change before the post spike (no earlier post spike)
    assert abs(w[-1] - expect) <= 2e-6 * expect, (w[-1], expect)
    assert w[-1] > w0


@pytest.mark.parametrize("mu", [1.0, 0.0, 0.4])
def test_single_post_pre_pair_depresses_by_closed_form(mu):
    q = W.Stdp(tau_plus=17.0, tau_minus=34.0, lam=0.05, alpha=1.2, mu_plus=mu, mu_minus=mu, W_max=100.0)
    w0 = 40.0
    # post fires at step 20; pre fires at step 30 and arrives at step 45
    o, w = _run_forced(_pair_spec(w0, q), {1: [20], 0: [30]}, 60)
    lag_ms = (45 - 20) * DT
    expect = w0 - q.alpha * q.lam * q.W_max * (w0 / q.W_max) ** mu * math.exp(-lag_ms / q.tau_minus)
    assert np.all(w[:44] == np.float32(w0))  # the arrival is delivered at the end of step 44
    assert abs(w[-1] - expect) <= 2e-6 * expect, (w[-1], expect)
    assert w[-1] < w0


def test_delivered_weight_is_the_depressed_weight():
    q = W.Stdp(tau_plus=20.0, tau_minus=20.0, lam=0.1, alpha=1.0, mu_plus=1.0, mu_minus=1.0, W_max=100.0)
    w0 = 60.0
    o = oracle.OracleNet(_pair_spec(w0, q))
    o.finalize()
    for t in range(45):
        if t + 1 == 20:
            o.inject(1, 0, 0, KICK)
        if t + 1 == 30:
            o.inject(0, 0, 0, KICK)
        o.simulate(1)
    # the pre spike of step 30 arrives at step 45: delivered after step 44 into the input of step 45
    got = float(o.input(0, 0)[0][1])
    w1 = float(o.csr()["weight"][0])
    assert w1 < w0 and got == np.float32(w1)


def _pairs_expected(a_steps, p_steps, q, w0):
    """w0 plus the nearest-neighbour pair sums of the additive rule, from the
    spike lists alone (brute force, FP64)."""
    A_p = q.lam * q.W_max
    A_m = q.alpha * q.lam * q.W_max
    w = w0
    a_steps = np.sort(np.asarray(a_steps))
    p_steps = np.sort(np.asarray(p_steps))
    for p in p_steps:
        prev = a_steps[a_steps <= p]
        if prev.size and (p - prev[-1]) * DT <= 20.0 * q.tau_plus:
            w += A_p * math.exp(-(p - prev[-1]) * DT / q.tau_plus)
    for a in a_steps:
        prev = p_steps[p_steps < a]
        if prev.size and (a - prev[-1]) * DT <= 20.0 * q.tau_minus:
            w -= A_m * math.exp(-(a - prev[-1]) * DT / q.tau_minus)
    return w


def _all_pairs(a_steps, p_steps, q, w0):
    A_p = q.lam * q.W_max
    A_m = q.alpha * q.lam * q.W_max
    w = w0
    for p in p_steps:
        for a in a_steps:
            if a <= p:
                w += A_p * math.exp(-(p - a) * DT / q.tau_plus)
            else:
                w -= A_m * math.exp(-(a - p) * DT / q.tau_minus)
    return w


def test_nearest_neighbour_pairing_on_poisson_trains():
    lif = W.LifParams(V_init_mean=-65.0, V_init_sd=4.0,
                      poisson=W.Poisson(n_inputs=1000.0, rate_hz=11.0, weight=87.8))
    q = W.Stdp(tau_plus=16.8, tau_minus=33.7, lam=1e-4, alpha=1.05, mu_plus=0.0, mu_minus=0.0, W_max=1000.0)
    w0 = 500.0
    spec = W.NetSpec(name="stdp_nn", seeds=[7])
    spec.pops = [W.Population("pre", W.LIF, 12, lif), W.Population("post", W.LIF, 10, lif)]
    spec.conns = [W.Connection(0, 1, W.ALL_TO_ALL, 0, W.Dist("const", w0), W.Dist("uniform", 0.5, 3.0), stdp=q)]
    o = oracle.OracleNet(spec)
    o.finalize()
    T = 8000
    o.simulate(T)
    ids, st = o.spikes()
    c = o.csr()
    src = np.repeat(np.arange(o.N), np.diff(c["src_ptr"].astype(np.int64)))
    n_checked = n_changed = 0
    for j in range(len(c["tgt"])):
        s, t_, d = int(src[j]), int(c["tgt"][j]), int(c["delay"][j])
        arr = st[ids == s] + d
        arr = arr[arr <= T]  # arrivals processed so far (the last one at the end of step T - 1)
        post = st[ids == t_]
        expect = _pairs_expected(arr, post, q, w0)
        assert abs(float(c["weight"][j]) - expect) <= 2e-3, (j, float(c["weight"][j]), expect)
        n_checked += 1
        if abs(expect - w0) > 0.05:
            n_changed += 1
            # the all-pairs rule would give a clearly different weight
            assert abs(_all_pairs(arr, post, q, w0) - expect) > 5e-3
    assert n_checked == 120 and n_changed >= 100
    assert len(ids) > 300


def test_weights_stay_within_bounds():
    lif = W.LifParams(V_init_mean=-65.0, V_init_sd=4.0,
                      poisson=W.Poisson(n_inputs=1000.0, rate_hz=11.0, weight=87.8))
    q = W.Stdp(tau_plus=20.0, tau_minus=20.0, lam=0.5, alpha=1.0, mu_plus=0.0, mu_minus=0.0, W_max=50.0)
    spec = W.NetSpec(name="stdp_clip", seeds=[3])
    spec.pops = [W.Population("a", W.LIF, 30, lif)]
    spec.conns = [W.Connection(0, 0, W.INDEGREE, 10, W.Dist("uniform", 0.0, 50.0), W.Dist("const", 1.0),
                               allow_autapses=False, stdp=q)]
    o = oracle.OracleNet(spec)
    o.simulate(5000)
    w = o.csr()["weight"]
    assert np.all(w >= 0.0) and np.all(w <= 50.0)
    assert np.count_nonzero(w == 0.0) > 0 and np.count_nonzero(w == np.float32(50.0)) > 0
