"""Pins of the oracle's connection builder and spike delivery -- CPU only.

Builder (Sec. 2.1 connection rules, Sec. 2.2 delay-ordered connection groups):
exact in-degrees / pathway totals, canonical (source, delay) order, source
uniformity (chi-square), weight moments and sign, delay histograms against the
clipped-normal and uniform distributions rounded to the grid.

Delivery (Sec. 2.2): the per-step input of every neuron equals a brute-force
dense evaluation  in_t = sum_d W_d s_{t-d}  from the synapse list and the spike
trains, in FP64 (FP32 sums within their rounding bound); the deterministic
fixed-point mode equals the exact sum rounded once.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import paper_values
from paper_2007_14236_gb300 import workloads as W

stats = pytest.importorskip("scipy.stats")


def _net(spec, **kw):
    n = oracle.OracleNet(spec, **kw)
    n.finalize()
    return n


def _src_of(csr):
    sp = csr["src_ptr"].astype(np.int64)
    return np.repeat(np.arange(len(sp) - 1), np.diff(sp))


def test_fixed_indegree_exact_counts_and_order():
    spec = W.balanced_lif(n=1000, indegree=100, seed=5)
    net = _net(spec)
    csr = net.csr()
    src = _src_of(csr)
    assert net.num_synapses == spec.num_synapses() == 1000 * 100
    tgt = csr["tgt"].astype(np.int64)
    from_e = np.bincount(tgt[src < 800], minlength=1000)
    from_i = np.bincount(tgt[src >= 800], minlength=1000)
    assert np.all(from_e == 80) and np.all(from_i == 20)
    # canonical order: source ascending, then delay ascending inside a source
    key = src * 4096 + csr["delay"].astype(np.int64)
    assert np.all(np.diff(key) >= 0)
    # constant weights / delays as specified
    assert set(np.unique(csr["weight"][src < 800])) == {np.float32(87.8)}
    assert set(np.unique(csr["weight"][src >= 800])) == {np.float32(-351.2)}
    assert set(np.unique(csr["delay"][src < 800])) == {15}
    assert set(np.unique(csr["delay"][src >= 800])) == {8}
    # sources uniform: chi-square over the 800 E sources
    cnt = np.bincount(src[src < 800], minlength=800)
    chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
    assert stats.chi2.sf(chi2, 799) > 1e-4


def test_fixed_indegree_without_autapses():
    spec = W.balanced_lif(n=200, indegree=50, seed=9)
    for c in spec.conns:
        c.allow_autapses = False
    net = _net(spec)
    csr = net.csr()
    src = _src_of(csr)
    assert not np.any(src == csr["tgt"].astype(np.int64))
    # with autapses allowed some appear (200 targets x 50 draws of 1/160 or 1/40)
    spec2 = W.balanced_lif(n=200, indegree=50, seed=9)
    csr2 = _net(spec2).csr()
    assert np.any(_src_of(csr2) == csr2["tgt"].astype(np.int64))


def test_fixed_total_number_pathway_counts_and_distributions():
    spec = W.microcircuit(scale=0.02, seed=3, keep_indegree=False)
    net = _net(spec)
    csr = net.csr()
    src = _src_of(csr)
    tgt = csr["tgt"].astype(np.int64)
    offs = np.cumsum([0] + [p.n for p in spec.pops])
    pop_of = np.searchsorted(offs, np.arange(offs[-1]), side="right") - 1
    for c in spec.conns:
        cnt = np.count_nonzero((pop_of[src] == c.src) & (pop_of[tgt] == c.tgt))
        assert cnt == c.K, (c.src, c.tgt, cnt, c.K)
    assert net.num_synapses == spec.num_synapses()
    # weights: inhibitory negative, excitatory positive, 10 % spread
    w = csr["weight"].astype(np.float64)
    exc = pop_of[src] % 2 == 0
    assert np.all(w[exc] > 0) and np.all(w[~exc] < 0)
    l4e_l23e = (pop_of[src] == 2) & (pop_of[tgt] == 0)
    plain_e = exc & ~l4e_l23e
    assert abs(w[plain_e].mean() - 87.8) < 0.5
    assert abs(w[plain_e].std() / 8.78 - 1) < 0.05
    assert abs(w[l4e_l23e].mean() - 175.6) < 2.0
    assert abs(w[~exc].mean() + 351.2) < 2.0
    # delays: Normal(1.5, 0.75) ms re-drawn below dt, rounded to 0.1 ms steps
    d = csr["delay"][plain_e].astype(np.int64)
    ks = np.arange(1, d.max() + 1)
    lo = np.maximum((ks - 0.5) * 0.1, 0.1)
    hi = (ks + 0.5) * 0.1
    p = stats.norm.cdf(hi, 1.5, 0.75) - stats.norm.cdf(lo, 1.5, 0.75)
    p /= 1.0 - stats.norm.cdf(0.1, 1.5, 0.75)
    obs = np.bincount(d, minlength=d.max() + 1)[1:]
    exp = p * len(d)
    ok = exp > 5
    chi2 = (((obs - exp) ** 2 / exp)[ok]).sum()
    assert stats.chi2.sf(chi2, ok.sum() - 1) > 1e-4, chi2
    assert d.min() >= 1


def test_rules_one_to_one_outdegree_all_to_all():
    """Sec. 2.1 rules, each checked against its definition."""
    spec = W.rules_net(seed=4)
    net = _net(spec)
    csr = net.csr()
    src = _src_of(csr)
    tgt = csr["tgt"].astype(np.int64)
    offs = np.cumsum([0] + [p.n for p in spec.pops])
    pop_of = np.searchsorted(offs, np.arange(offs[-1]), side="right") - 1
    ps, pt = pop_of[src], pop_of[tgt]
    assert net.num_synapses == spec.num_synapses() == 300 + 300 * 40 + 200 * 300 + 300 * 299 + 300
    # one-to-one A -> B and B -> B: neuron i to neuron i, exactly once
    for a, b in ((0, 1), (1, 1)):
        m = (ps == a) & (pt == b)
        assert np.count_nonzero(m) == 300
        assert np.array_equal(np.sort(src[m] - offs[a]), np.arange(300))
        assert np.all(src[m] - offs[a] == tgt[m] - offs[b])
    # fixed out-degree B -> C: exactly 40 per source, targets uniform
    m = (ps == 1) & (pt == 2)
    assert np.all(np.bincount(src[m] - offs[1], minlength=300) == 40)
    cnt = np.bincount(tgt[m] - offs[2], minlength=200)
    chi2 = ((cnt - cnt.mean()) ** 2 / cnt.mean()).sum()
    assert stats.chi2.sf(chi2, 199) > 1e-4
    # all-to-all C -> A: every pair once; A -> A without autapses: every pair but (i, i)
    m = (ps == 2) & (pt == 0)
    pairs = (src[m] - offs[2]) * 300 + (tgt[m] - offs[0])
    assert np.array_equal(np.sort(pairs), np.arange(200 * 300))
    m = (ps == 0) & (pt == 0)
    a_s, a_t = src[m], tgt[m]
    assert len(a_s) == 300 * 299 and not np.any(a_s == a_t)
    assert len(np.unique(a_s * 300 + a_t)) == 300 * 299
    # delays: constant / uniform (0.5, 2] ms / clipped normal, as specified
    assert set(np.unique(csr["delay"][(ps == 0) & (pt == 1)])) == {10}
    d_ca = csr["delay"][(ps == 2) & (pt == 0)].astype(np.int64)
    assert d_ca.min() == 5 and d_ca.max() == 20
    assert np.all(csr["delay"] >= 1)


def test_rules_rows_for_sources():
    spec = W.rules_net(seed=4)
    net = _net(spec)
    csr = net.csr()
    sp = csr["src_ptr"].astype(np.int64)
    lazy = oracle.OracleNet(spec)
    srcs = np.array([3, 299, 301, 450, 600, 799])
    rows = lazy.rows_for_sources(srcs)
    want = np.concatenate([np.arange(sp[s], sp[s + 1]) for s in srcs])
    for k in ("tgt", "receptor", "weight", "delay"):
        assert np.array_equal(rows[k], csr[k][want]), k


def test_uniform_delay_histogram():
    spec = W.balanced_adex(n=500, indegree=100, seed=2, weight_dtype="fp32")
    net = _net(spec)
    csr = net.csr()
    d = csr["delay"].astype(np.int64)
    assert d.min() == 10 and d.max() == 20
    obs = np.bincount(d, minlength=21)[10:21]
    # U(1, 2] ms rounded half-to-even: steps 10 and 20 get half a bin each
    p = np.full(11, 0.1)
    p[0] = p[-1] = 0.05
    chi2 = ((obs - p * len(d)) ** 2 / (p * len(d))).sum()
    assert stats.chi2.sf(chi2, 10) > 1e-4
    # receptor 1 exactly for inhibitory sources, positive conductance weights
    src = _src_of(csr)
    assert np.all(csr["receptor"][src >= 400] == 1) and np.all(csr["receptor"][src < 400] == 0)
    assert np.all(csr["weight"] > 0)


def test_microcircuit_synapse_total_matches_formula_and_paper():
    K = sum(c.K for c in W.microcircuit(scale=1.0).conns)
    assert K == 298_880_968
    # the paper's approximate neuron and connection counts (golden fixture)
    mc = paper_values()["microcircuit"]
    assert abs(sum(W.MC_SIZES) - mc["neurons_about"]) < 500
    assert abs(K - mc["connections_about"]) / mc["connections_about"] < 0.01


def test_paper_balanced_workload_follows_the_paper_table():
    """The workload recipe of the balanced network against the paper's
    parameter table (golden fixture): population and in-degree ratios,
    weights, delay distribution and Poisson drive."""
    tab = paper_values()["balanced_network_table"]
    adex = paper_values()["adex_table"]
    spec = W.paper_balanced(n_ex=8000, ce=800, seed=1)
    ex, inh = spec.pops
    assert inh.n / ex.n == tab["N_in_over_N_ex"]
    ee, ie = spec.conns[0], spec.conns[1]
    assert ie.K / ee.K == tab["CI_over_CE"]
    assert ee.weight.p0 == tab["W_ex_nS"] and ie.weight.p0 == tab["W_in_nS"] and ie.receptor == 1
    assert ee.delay.kind == "normal" and (ee.delay.p0, ee.delay.p1) == (tab["delay_mean_ms"], tab["delay_sd_ms"])
    for p in spec.pops:
        q = p.params
        assert (q.poisson.weight, q.poisson.n_inputs * q.poisson.rate_hz) == (tab["W_poisson_nS"], tab["rate_poisson_hz"])
        assert (q.C_m, q.g_L, q.E_L, q.V_T, q.Delta_T, q.tau_w, q.a, q.b, q.V_reset, q.E_ex, q.E_in) == (
            adex["C_m_pF"], adex["g_L_nS"], adex["E_L_mV"], adex["V_T_mV"], adex["Delta_T_mV"], adex["tau_w_ms"],
            adex["a_nS"], adex["b_pA"], adex["V_reset_mV"], adex["E_ex_mV"], adex["E_in_mV"])
        assert q.tau_ex == q.tau_in == adex["tau_syn_ms"]


def _run_with_inputs(spec, steps, **kw):
    net = _net(spec, track_abs=True, **kw)
    R = 2 if any(p.model == W.AEIF for p in spec.pops) else 1
    ins, abss, exact = [], [], []
    for _ in range(steps):
        per_r = [net.input(r, 0) for r in range(R)]
        ins.append(np.stack([x[0] for x in per_r]))
        abss.append(np.stack([x[1] for x in per_r]))
        exact.append(np.stack([x[2] for x in per_r]))
        net.simulate(1)
    return net, np.array(ins), np.array(abss), np.array(exact)


def _brute_force_inputs(net, steps, R):
    csr = net.csr()
    src = _src_of(csr)
    N = net.N
    dmax = int(csr["delay"].max())
    Wd = np.zeros((dmax + 1, R, N, N))
    np.add.at(Wd, (csr["delay"].astype(np.int64), csr["receptor"].astype(np.int64), csr["tgt"].astype(np.int64),
                   src), csr["weight"].astype(np.float64))
    ids, st = net.spikes()
    S = np.zeros((steps, N))
    np.add.at(S, (st, ids), 1.0)
    expect = np.zeros((steps, R, N))
    for t in range(steps):
        for d in range(1, dmax + 1):
            if t - d >= 0:
                expect[t] += Wd[d] @ S[t - d]
    return expect


@pytest.mark.parametrize("deterministic", [False, True])
def test_delivery_equals_brute_force_dense(deterministic):
    spec = W.balanced_lif(n=120, indegree=20, seed=4, n_ext=1600.0)
    spec.conns[0].delay = W.Dist("normal", 1.5, 0.75)
    spec.conns[2].delay = W.Dist("uniform", 0.3, 1.2)
    steps = 400
    net, ins, abss, exact = _run_with_inputs(spec, steps, deterministic=deterministic)
    assert len(net.spikes()[0]) > 100
    expect = _brute_force_inputs(net, steps, 1)
    assert np.allclose(exact, expect, rtol=0, atol=1e-9)
    bound = 1e-6 * abss + 1e-6
    assert np.all(np.abs(ins - expect) <= bound)
    if deterministic:
        # fixed point: exactly the exact sum rounded once to FP32
        assert np.array_equal(ins, expect.astype(np.float32))
    # invariant: the total delivered at step t is the weight sum of the spikes of step t - d
    assert np.allclose(exact.sum(axis=(1, 2)), expect.sum(axis=(1, 2)), atol=1e-6)


def test_delivery_two_receptors_adex():
    spec = W.balanced_adex(n=100, indegree=20, seed=6, weight_dtype="fp32", poisson_weight=4.0,
                           w_ex=2.0, w_in=4.0)
    steps = 300
    net, ins, abss, exact = _run_with_inputs(spec, steps)
    assert len(net.spikes()[0]) > 10
    expect = _brute_force_inputs(net, steps, 2)
    assert np.allclose(exact, expect, rtol=0, atol=1e-9)
    assert np.all(np.abs(ins - expect) <= 1e-6 * abss + 1e-6)


def test_events_count_and_spike_order():
    spec = W.balanced_lif(n=300, indegree=30, seed=8, n_ext=1400.0)
    net = _net(spec)
    net.simulate(500)
    ids, st = net.spikes()
    assert len(ids) > 50
    order = np.lexsort((ids, st))
    assert np.array_equal(order, np.arange(len(ids)))  # (step, id) order
    outdeg = np.diff(net.csr()["src_ptr"].astype(np.int64))
    assert net.events == int(outdeg[ids].sum())


def test_rows_for_sources_equal_the_built_csr():
    spec = W.microcircuit(scale=0.02, seed=11, keep_indegree=False)
    for c in spec.conns[:6]:
        c.allow_autapses = False
    built = _net(spec)
    csr = built.csr()
    lazy = oracle.OracleNet(spec)  # never finalised: rows are drawn one by one
    srcs = [0, 5, 17, 400, int(built.N) - 1]
    rows = lazy.rows_for_sources(srcs)
    sp = csr["src_ptr"].astype(np.int64)
    sel = np.concatenate([np.arange(sp[s], sp[s + 1]) for s in sorted(srcs)])
    for k in ("tgt", "receptor", "weight", "delay"):
        assert np.array_equal(rows[k], csr[k][sel]), k


def test_paper_balanced_network_rate_matches_paper():
    """The paper's balanced network (Sec. 2.4: AdEx with alpha-function
    conductances, its parameter tables) fires at 30.7 Hz on average; the
    oracle's steady-state rate at 10,000 neurons and in-degree 1,000 is within
    10 % of it."""
    spec = W.paper_balanced(n_ex=8000, ce=800, seed=2)
    net = _net(spec)
    net.simulate(2500)
    ids, st = net.spikes()
    rate = np.count_nonzero(st >= 1000) / 10000 / 0.15
    paper = paper_values()["balanced_network_table"]["mean_firing_rate_hz"]
    assert abs(rate - paper) <= 0.1 * paper, rate
