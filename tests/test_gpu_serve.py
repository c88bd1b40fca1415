"""Continuous batching (serving handles): networks are committed into and
retired from the pools while others run in the same kernels.

* Each served network's spikes equal the same network run alone through the
  plain path, bit for bit in deterministic mode, although networks join and
  leave at different steps and reuse each other's pool ranges; the first and
  the last admitted networks also equal the CPU oracle's run of the same
  network, spike for spike.
* FP32 mode: spike counts within tolerance of the plain path.
* A commit that does not fit the pools fails with NGB_ERR_OOM and leaves the
  running networks untouched; it succeeds once space is freed.
"""
import numpy as np
import pytest

import oracle
from paper_2007_14236_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2007_14236_gb300 import ngb, serve
    ngb.load()
    return ngb, serve


def _requests(n, seed, n_lo=2000, n_hi=6000, k_lo=50, k_hi=120, t_lo=20.0, t_hi=80.0, burst=True):
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(n):
        if not burst:
            t += rng.exponential(0.01)
        out.append(W.Request(arrival_s=t, n=int(rng.integers(n_lo, n_hi)), indegree=int(rng.integers(k_lo, k_hi)),
                             bio_time_ms=float(round(rng.uniform(t_lo, t_hi), 1)), seed=500 + i))
    return out


def test_served_equals_alone_deterministic(mods):
    ngb, serve = mods
    reqs = _requests(10, seed=1)
    # pools for about three networks at a time: later ones wait and reuse freed ranges
    srv = serve.Server(max_neurons=16000, max_synapses=1_500_000, max_groups=16000, ring_slots=16,
                       chunk_steps=100, deterministic=True, keep_spikes=True)
    done, summary = srv.run(reqs)
    srv.close()
    assert summary["requests"] == 10 and summary["max_active"] >= 2
    for d in done:
        _, _, ids, st = serve.run_alone(d.req, deterministic=True, keep_spikes=True)
        o = np.lexsort((ids, st))
        assert len(ids) > 0
        assert np.array_equal(d.steps, st[o]) and np.array_equal(d.ids, ids[o]), d.req.seed
    # anchor to the oracle: served networks that joined late, after others had left (pool ranges
    # reused), and the first one, spike for spike against the CPU oracle of the same network
    late = sorted(done, key=lambda d: d.admit_s)
    for d in (late[0], late[-2], late[-1]):
        ora = oracle.OracleNet(W.request_net(d.req), deterministic=True)
        ora.finalize()
        ora.simulate(int(round(d.req.bio_time_ms / 0.1)))
        oi, ot = ora.spikes()
        o = np.lexsort((oi, ot))
        assert len(oi) > 0
        assert np.array_equal(d.steps, ot[o]) and np.array_equal(d.ids, oi[o]), d.req.seed


def test_served_fp32_counts_close_to_alone(mods):
    ngb, serve = mods
    reqs = _requests(6, seed=2, t_lo=100.0, t_hi=150.0)
    srv = serve.Server(max_neurons=40000, max_synapses=4_000_000, max_groups=40000, ring_slots=16,
                       chunk_steps=250, keep_spikes=True)
    done, _ = srv.run(reqs)
    srv.close()
    for d in done:
        _, ev, ids, _ = serve.run_alone(d.req, keep_spikes=True)
        assert abs(d.spikes - len(ids)) <= 0.05 * len(ids) + 20


def test_commit_out_of_room_then_retry(mods):
    ngb, serve = mods
    sim = ngb.Simulator(deterministic=True)
    sim.reserve(5000, 400_000, 5000, 16, 1)
    a, _ = sim.add_spec_instance(W.balanced_lif(n=3000, indegree=100, seed=1))
    sim.commit(a)
    sim.simulate(50)
    b, _ = sim.add_spec_instance(W.balanced_lif(n=3000, indegree=100, seed=2))
    with pytest.raises(ngb.NgbError) as e:
        sim.commit(b)
    assert e.value.code == -3
    sim.simulate(50)  # the running network is unaffected
    assert sim.instance_info(a) == (0, 1) and sim.instance_info(b)[1] == 0
    sim.retire(a)
    sim.commit(b)
    t0, state = sim.instance_info(b)
    assert t0 == 100 and state == 1
    sim.simulate(100)
    assert sim.stats()["steps"] == 200
