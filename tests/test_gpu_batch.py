"""Batched execution (several independent networks advanced by the same
kernels): each instance's result in the mix equals the instance run alone,
bit for bit in deterministic mode (instance keys and instance-local ids make
the random streams placement-independent), and equals the oracle."""
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


def _instance_spikes(sim, spec, inst):
    pops = spec.instance_pops(inst)
    lo = sim.population_range(pops[0])[0]
    last = sim.population_range(pops[-1])
    hi = last[0] + last[1]
    ids, st = sim.spikes()
    m = (ids >= lo) & (ids < hi)
    return ids[m] - lo, st[m]


def test_batched_instances_equal_alone_and_oracle(ngb):
    spec = W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7)
    assert len(spec.pops) > 12  # beyond the inline segment table
    batch = ngb.from_spec(spec, deterministic=True)
    batch.simulate(500)
    for i in range(3):
        alone_spec = W.instance_spec(spec, i)
        alone = ngb.from_spec(alone_spec, deterministic=True)
        alone.simulate(500)
        ai, at = alone.spikes()
        bi, bt = _instance_spikes(batch, spec, i)
        assert len(ai) > 50
        assert np.array_equal(at, bt) and np.array_equal(ai, bi), i
        if i == 0:
            o = oracle.OracleNet(alone_spec, deterministic=True)
            o.simulate(500)
            oi, ot = o.spikes()
            assert np.array_equal(ot, at) and np.array_equal(oi, ai)
        alone.close()


def test_batched_fp32_rates_match_alone(ngb):
    spec = W.batched_microcircuits(n_instances=4, scale_lo=0.05, scale_hi=0.1, seed=8)
    batch = ngb.from_spec(spec)
    batch.simulate(3000)
    for i in range(4):
        alone = ngb.from_spec(W.instance_spec(spec, i))
        alone.simulate(3000)
        na = len(alone.spikes()[0])
        nb = len(_instance_spikes(batch, spec, i)[0])
        assert abs(na - nb) <= 0.05 * na + 20, (i, na, nb)
        alone.close()
