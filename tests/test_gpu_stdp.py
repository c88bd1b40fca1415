"""Nearest-neighbour STDP synapses (Sec. 2.1) on the GPU against the oracle,
through the C ABI (needs a GB300).

* Deterministic mode, multiplicative and additive rules: spike trains and
  every synapse's final weight bit-exact against the oracle over 1,500
  steps (graph replay, eager steps and the profiled path all taken).
* A fractional exponent (powf on both sides, not bit-identical): weights
  within 1e-5 relative after 300 steps, rates within 5 % over 2,000 steps.
* FP32 mode: rates within 5 % and the mean plastic weight within 0.5 % of
  the oracle's.
* The autotuner's trial steps leave the weights untouched.
* Restrictions: the ring scheme and BF16 weights are rejected; requests for
  other step loops fall back to per-step kernels; serving handles refuse
  plastic synapses.
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


def _plastic_mask(c_tgt, src_ptr, n_e=800):
    src = np.repeat(np.arange(len(src_ptr) - 1), np.diff(src_ptr.astype(np.int64)))
    return (src < n_e) & (c_tgt < n_e)


@pytest.mark.parametrize("mu", [1.0, 0.0])
def test_stdp_deterministic_bit_exact(ngb, mu):
    spec = W.stdp_net(seed=2, mu=mu)
    g = ngb.from_spec(spec, deterministic=True, steps_per_graph=100, drain_steps=250)
    o = oracle.OracleNet(spec, deterministic=True)
    g.finalize()
    o.finalize()
    assert g.stats()["delivery"] == 2 and g.stats()["mode"] == 0
    w0 = g.synapses()["weight"].copy()
    for chunk in (1, 99, 400):  # eager steps, then graph replays
        g.simulate(chunk)
        o.simulate(chunk)
    g.simulate_profiled(50)
    o.simulate(50)
    g.simulate(950)
    o.simulate(950)
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    assert len(oi) > 2000
    assert np.array_equal(gt, ot) and np.array_equal(gi, oi)
    gs, oc = g.synapses(), o.csr()
    assert np.array_equal(gs["tgt"], oc["tgt"])
    assert np.array_equal(gs["weight"], oc["weight"])
    pl = _plastic_mask(gs["tgt"], oc["src_ptr"])
    assert np.mean(gs["weight"][pl] != w0[pl]) > 0.95  # the plastic weights moved
    assert np.array_equal(gs["weight"][~pl], w0[~pl])  # the static ones did not
    assert np.array_equal(g.input(0, 0), o.input(0, 0)[0])


def test_stdp_fractional_exponent(ngb):
    spec = W.stdp_net(seed=3, mu=0.4)
    g = ngb.from_spec(spec, deterministic=True)
    o = oracle.OracleNet(spec, deterministic=True)
    g.simulate(300)
    o.simulate(300)
    gw, ow = g.synapses()["weight"].astype(np.float64), o.csr()["weight"].astype(np.float64)
    assert np.all(np.abs(gw - ow) <= 1e-5 * np.abs(ow) + 1e-6)
    g.simulate(1700)
    o.simulate(1700)
    ng, no = len(g.spikes()[0]), len(o.spikes()[0])
    assert no > 2500 and abs(ng - no) <= 0.05 * no, (ng, no)


def test_stdp_fp32_statistics(ngb):
    spec = W.stdp_net(seed=4, mu=1.0)
    g = ngb.from_spec(spec)
    o = oracle.OracleNet(spec)
    g.simulate(3000)
    o.simulate(3000)
    ng, no = len(g.spikes()[0]), len(o.spikes()[0])
    assert no > 4000 and abs(ng - no) <= 0.05 * no, (ng, no)
    gs, oc = g.synapses(), o.csr()
    pl = _plastic_mask(gs["tgt"], oc["src_ptr"])
    mg, mo = gs["weight"][pl].mean(), oc["weight"][pl].mean()
    assert abs(mg - mo) <= 0.005 * mo, (mg, mo)
    assert abs(gs["weight"][pl].std() - oc["weight"][pl].std()) <= 0.05 * oc["weight"][pl].std()


def test_stdp_autotune_leaves_weights(ngb):
    spec = W.stdp_net(seed=5, mu=1.0)
    a = ngb.from_spec(spec, deterministic=True)
    b = ngb.from_spec(spec, deterministic=True)
    a.simulate(200)
    b.simulate(200)
    b.autotune(300)
    assert b.stats()["steps"] == 200 and b.stats()["mode"] == 0 and b.stats()["delivery"] == 2
    assert np.array_equal(a.synapses()["weight"], b.synapses()["weight"])
    a.simulate(300)
    b.simulate(300)
    assert np.array_equal(a.spikes()[0], b.spikes()[0]) and np.array_equal(a.spikes()[1], b.spikes()[1])
    assert np.array_equal(a.synapses()["weight"], b.synapses()["weight"])


def test_stdp_restrictions(ngb):
    spec = W.stdp_net(seed=1, n=200, indegree=20)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        ngb.from_spec(spec, delivery="ring")
    spec_bf = W.stdp_net(seed=1, n=200, indegree=20)
    spec_bf.weight_dtype = "bf16"
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        ngb.from_spec(spec_bf)
    for mode in ("persistent", "fused", "pipelined", "target_owned"):
        with _env(NGB_MODE=mode):
            sim = ngb.from_spec(spec, deterministic=True)
            sim.finalize()
        assert sim.stats()["mode"] == 0 and sim.stats()["delivery"] == 2
        sim.simulate(20)
    sim = ngb.from_spec(spec)
    with pytest.raises(RuntimeError, match="STATE"):
        sim.reserve(10000, 10 ** 6, 10 ** 5, 64, 1)
