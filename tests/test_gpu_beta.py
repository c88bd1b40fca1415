"""Multisynapse AdEx with beta-function conductances (the paper's interface
example, Sec. 2.1), GPU path against the oracle through the C ABI (needs a
GB300).

* One four-port neuron driven by a current and by Poisson input on port 3
  (the port stored outside the two-receptor arrays): V, g_3 and x_3 of the
  FP32-state GPU integration against the FP64 oracle; spike steps within one.
* A three-population network with 1, 3 and 4 ports: the synapses' receptor
  fields bit-exact, per-step inputs on all four receptor planes within the
  FP32 summation bound, identical spikes over the first steps, per-population
  spike counts within 5 % of the FP32 oracle.
* Deterministic mode: the ring and spike-buffer schemes, the pipelined loop
  and attempt budgets 0, 1 and 8 give bit-identical runs; requests for the
  persistent or fused loop fall back to per-step kernels.
* Invalid port counts, time constants and receptors are rejected.
"""
import os
from contextlib import contextmanager

import numpy as np
import pytest

import oracle
from paper_2007_14236_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ngb():
    from paper_2007_14236_gb300 import ngb as m
    m.load()
    return m


@contextmanager
def _env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    os.environ.update({k: str(v) for k, v in kv.items()})
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


BOUNDS = [0, 400, 750, 1000]  # B3, B4, B1 of the beta network


def test_beta_four_port_neuron_vs_fp64_oracle(ngb):
    ports = [(0.0, 0.2, 2.0), (-85.0, 0.5, 5.0), (-75.0, 1.0, 1.0), (0.0, 0.3, 3.0)]
    par = W.AeifParams(V_reset=-60.0, I_e=450.0, rk_h_min=1e-9, rk_max_substeps=100000, ports=ports,
                       poisson=W.Poisson(n_inputs=1.0, rate_hz=20000.0, weight=0.37, receptor=3))
    spec = W.NetSpec(name="beta1", seeds=[1], pops=[W.Population("n", W.AEIF_BETA, 1, par)])
    g = ngb.from_spec(spec)
    g.finalize()
    o = oracle.OracleNet(spec, adex_fp64=True)
    o.finalize()
    steps = 1500
    Vg, Vo, Gg, Go, Xg, Xo = (np.zeros(steps) for _ in range(6))
    for k in range(steps):
        g.simulate(1)
        o.simulate(1)
        Vg[k], Vo[k] = g.state("V_m")[0], o.state("V_m")[0]
        Gg[k], Go[k] = g.state("g_3")[0], o.state("g_3")[0]
        Xg[k], Xo[k] = g.state("x_3")[0], o.state("x_3")[0]
    assert Go.max() > 1.0  # port 3 carries the drive
    assert g.state("g_0")[0] == 0.0 and g.state("g_2")[0] == 0.0  # the other ports receive nothing
    assert np.abs(Gg - Go).max() <= 1e-4 * Go.max()
    assert np.abs(Xg - Xo).max() <= 1e-4 * np.abs(Xo).max()
    sg, so = g.spikes()[1], o.spikes()[1]
    assert len(so) >= 3 and len(sg) == len(so)
    assert np.all(np.abs(sg - so) <= 1)
    mask = np.ones(steps, dtype=bool)
    for s_ in so:
        mask[max(0, s_ - 20):s_ + 2] = False
    assert np.abs(Vg - Vo)[mask].max() <= 5e-3


def test_beta_network_matches_fp32_oracle(ngb):
    spec = W.beta_net(seed=2)
    g = ngb.from_spec(spec)
    g.finalize()
    o = oracle.OracleNet(spec, track_abs=True)
    o.finalize()
    gs, oc = g.synapses(), o.csr()
    assert np.array_equal(gs["tgt"], oc["tgt"]) and np.array_equal(gs["delay"], oc["delay"])
    assert np.array_equal(gs["receptor"], oc["receptor"])
    assert set(np.unique(gs["receptor"]).tolist()) == {0, 1, 2, 3}
    for step in range(30):
        for r in range(4):
            gin = g.input(r, 0).astype(np.float64)
            _, oabs, oex = o.input(r, 0)
            assert np.all(np.abs(gin - oex) <= 1e-5 * oabs + 1e-7), (step, r)
        g.simulate(1)
        o.simulate(1)
    g.simulate(970)
    o.simulate(970)
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    early = 20
    assert np.array_equal(np.sort(gi[gt < early]), np.sort(oi[ot < early]))
    for p in range(3):
        ng = np.count_nonzero((gi >= BOUNDS[p]) & (gi < BOUNDS[p + 1]))
        no = np.count_nonzero((oi >= BOUNDS[p]) & (oi < BOUNDS[p + 1]))
        assert no > 200 and abs(ng - no) <= 0.05 * no + 10, (p, ng, no)


BETA_VARS = ("V_m", "w", "h", "g_0", "g_1", "g_2", "g_3", "x_0", "x_1", "x_2", "x_3")


def _det_run(ngb, spec, delivery="ring", env=None, chunks=(300, 300)):
    with _env(**(env or {})):
        sim = ngb.from_spec(spec, deterministic=True, delivery=delivery, drain_steps=250)
        sim.finalize()
    for c in chunks:
        sim.simulate(c)
    return sim


def _assert_same_run(a, b):
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 100
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    for var in BETA_VARS:
        assert np.array_equal(a.state(var), b.state(var)), var
    assert a.stats()["rk_substeps"] == b.stats()["rk_substeps"]
    assert a.stats()["events"] == b.stats()["events"]


def test_beta_schemes_loops_and_budgets_bit_identical(ngb):
    spec = W.beta_net(seed=3)
    a = _det_run(ngb, spec)
    assert a.stats()["delivery"] == 1
    b = _det_run(ngb, spec, delivery="spike_buffer")
    assert b.stats()["delivery"] == 2
    _assert_same_run(a, b)
    for r in range(4):
        assert np.array_equal(a.input(r, 0), b.input(r, 0)), r
    c = _det_run(ngb, spec, env={"NGB_MODE": "pipelined"})
    assert c.stats()["mode"] == 3
    _assert_same_run(a, c)
    for budget in (0, 1):
        _assert_same_run(a, _det_run(ngb, spec, env={"NGB_AEIF_BUDGET": budget}))
    for mode in ("persistent", "fused"):  # not available with beta populations: per-step kernels
        d = _det_run(ngb, spec, env={"NGB_MODE": mode})
        assert d.stats()["mode"] == 0
        _assert_same_run(a, d)


def test_beta_invalid_arguments(ngb):
    base = dict(V_reset=-60.0)
    for ports in ([], [(0.0, 0.2, 2.0)] * 5, [(0.0, 0.0, 2.0)], [(0.0, 0.2, -1.0)]):
        sim = ngb.Simulator()
        with pytest.raises(RuntimeError, match="INVALID_ARG"):
            sim.add_population(W.AEIF_BETA, 10, W.AeifParams(ports=ports, **base))
    sim = ngb.Simulator()
    with pytest.raises(RuntimeError, match="INVALID_ARG"):  # Poisson drive on a port the model lacks
        sim.add_population(W.AEIF_BETA, 10, W.AeifParams(ports=[(0.0, 0.2, 2.0)] * 2,
                                                         poisson=W.Poisson(receptor=2), **base))
    p3 = sim.add_population(W.AEIF_BETA, 10, W.AeifParams(ports=[(0.0, 0.2, 2.0)] * 3, **base))
    lif = sim.add_population(W.LIF, 10, W.LifParams())
    ok = dict(weight=W.Dist("const", 1.0), delay=W.Dist("const", 1.0))
    sim.connect(lif, p3, W.INDEGREE, 2, receptor=2, **ok)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        sim.connect(lif, p3, W.INDEGREE, 2, receptor=3, **ok)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        sim.connect(p3, lif, W.INDEGREE, 2, receptor=1, **ok)
    sim.simulate(10)
    assert sim.stats()["steps"] == 10
