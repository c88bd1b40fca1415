"""Step loops against each other: the persistent step kernel (many steps per
cooperative launch, grid barriers between the update and delivery phases),
the fused loop (each update block delivers its own spikes, one launch per
step), the pipelined loop (delay-1 groups delivered by the update kernels,
the other groups by a delivery kernel beside the next step's update) and the
update kernel at four neurons per thread, against the per-step kernels; and
the bounded barrier wait.

* Deterministic mode: the persistent kernel gives bit-identical spike trains
  and state to the per-step path (LIF, AdEx, batched instances), and to the
  oracle.
* Autotuning (which times both step loops on a snapshot) leaves the
  simulation where it was.
* A block that never arrives at a barrier (test hook) makes every wait give
  up after its poll limit: ngb_simulate returns NGB_ERR_TIMEOUT instead of
  hanging, and the GPU stays usable.
"""
import os

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


class _env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update({k: str(v) for k, v in self.kv.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _persistent(ngb, spec, **kw):
    with _env(NGB_MODE="persistent"):
        sim = ngb.from_spec(spec, **kw)
        sim.finalize()
    assert sim.stats()["mode"] == 1
    return sim


@pytest.mark.parametrize("name", ["balanced_lif", "microcircuit", "adex", "batched", "paper_alpha", "mixed"])
def test_persistent_equals_per_step_kernels(ngb, name):
    spec = {"balanced_lif": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
            "mixed": lambda: W.mixed_net(seed=2),
            "paper_alpha": lambda: W.paper_balanced(n_ex=1600, ce=160, seed=3),
            "microcircuit": lambda: W.microcircuit(scale=0.03, seed=7, keep_indegree=False),
            "adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                            w_ex=2.0, w_in=4.0),
            "batched": lambda: W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7)}[name]()
    a = ngb.from_spec(spec, deterministic=True)
    b = _persistent(ngb, spec, deterministic=True, drain_steps=250)
    a.simulate(700)
    b.simulate(300)
    b.simulate(400)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert a.stats()["events"] == b.stats()["events"]
    if name in ("adex", "paper_alpha"):
        assert a.stats()["rk_substeps"] == b.stats()["rk_substeps"]
    if name == "balanced_lif":
        o = oracle.OracleNet(spec, deterministic=True)
        o.simulate(700)
        oi, ot = o.spikes()
        assert np.array_equal(ot, bt) and np.array_equal(oi, bi)


@pytest.mark.parametrize("name", ["balanced_lif", "microcircuit", "adex", "batched", "paper_alpha", "mixed",
                                  "mc_bf16"])
def test_pipelined_persistent_equals_per_step_kernels(ngb, name):
    """The pipelined persistent kernel (one grid barrier per step; delay-1
    groups delivered by the update phase, the others one phase later), in
    launches of uneven length: bit-identical spike trains, state, inputs of the
    coming steps and event counts."""
    spec = {"balanced_lif": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
            "mixed": lambda: W.mixed_net(seed=2),
            "paper_alpha": lambda: W.paper_balanced(n_ex=1600, ce=160, seed=3),
            "microcircuit": lambda: W.microcircuit(scale=0.03, seed=7, keep_indegree=False),
            "mc_bf16": lambda: W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="bf16"),
            "adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                            w_ex=2.0, w_in=4.0),
            "batched": lambda: W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7)}[name]()
    a = ngb.from_spec(spec, deterministic=True, delivery="ring")
    with _env(NGB_MODE="persistent_pipelined"):
        b = ngb.from_spec(spec, deterministic=True, delivery="ring", drain_steps=250)
        b.finalize()
    assert b.stats()["mode"] == 4
    a.simulate(700)
    for chunk in (1, 2, 97, 300, 300):  # 1- and 2-step launches, then chunks of 250
        b.simulate(chunk)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert a.stats()["events"] == b.stats()["events"]
    for off in range(0, 4):
        assert np.array_equal(a.input(0, off), b.input(0, off))
    b.simulate_profiled(20)  # per-step kernels after a pipelined persistent launch, then back
    b.simulate(30)
    a.simulate(50)
    assert np.array_equal(a.spikes()[0], b.spikes()[0]) and np.array_equal(a.state("V_m"), b.state("V_m"))


def test_pipelined_persistent_barrier_wait_is_bounded(ngb):
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    with _env(NGB_TEST_WITHHOLD_BLOCK=0, NGB_BARRIER_SPIN_LIMIT=20000, NGB_MODE="persistent_pipelined"):
        sim = ngb.from_spec(spec, delivery="ring")
        sim.finalize()
    assert sim.stats()["mode"] == 4
    with pytest.raises(ngb.NgbError) as e:
        sim.simulate(50)
    assert e.value.code == -5  # NGB_ERR_TIMEOUT
    sim.close()
    with _env(NGB_MODE="persistent_pipelined"):
        ok = ngb.from_spec(spec, deterministic=True, delivery="ring")
        ok.simulate(100)
    assert ok.stats()["steps"] == 100


def test_persistent_fp32_rates(ngb):
    spec = W.microcircuit(scale=0.05, seed=5, keep_indegree=False)
    a = ngb.from_spec(spec)
    b = _persistent(ngb, spec)
    a.simulate(3000)
    b.simulate(3000)
    na, nb = len(a.spikes()[0]), len(b.spikes()[0])
    assert abs(na - nb) <= 0.05 * na + 20


def test_autotune_does_not_advance_the_simulation(ngb):
    spec = W.microcircuit(scale=0.03, seed=3, keep_indegree=False)
    a = ngb.from_spec(spec, deterministic=True)
    b = ngb.from_spec(spec, deterministic=True)
    a.simulate(200)
    b.simulate(200)
    grid = b.autotune(300)
    st = b.stats()
    assert grid > 0 and st["steps"] == 200 and st["mode"] in (0, 1, 2, 3, 4, 5, 6)
    a.simulate(500)
    b.simulate(500)
    assert np.array_equal(a.spikes()[0], b.spikes()[0]) and np.array_equal(a.spikes()[1], b.spikes()[1])
    assert a.stats()["events"] == b.stats()["events"]


def test_barrier_wait_is_bounded(ngb):
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    with _env(NGB_TEST_WITHHOLD_BLOCK=0, NGB_BARRIER_SPIN_LIMIT=20000):
        sim = _persistent(ngb, spec)
    with pytest.raises(ngb.NgbError) as e:
        sim.simulate(50)
    assert e.value.code == -5  # NGB_ERR_TIMEOUT
    sim.close()
    # the GPU is still usable
    ok = _persistent(ngb, spec, deterministic=True)
    ok.simulate(100)
    assert ok.stats()["steps"] == 100


@pytest.mark.parametrize("name", ["balanced_lif", "microcircuit", "adex", "batched", "mc_bf16", "paper_alpha",
                                  "mixed"])
def test_fused_equals_per_step_kernels(ngb, name):
    spec = {"balanced_lif": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
            "mixed": lambda: W.mixed_net(seed=2),
            "paper_alpha": lambda: W.paper_balanced(n_ex=1600, ce=160, seed=3),
            "microcircuit": lambda: W.microcircuit(scale=0.03, seed=7, keep_indegree=False),
            "adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                            w_ex=2.0, w_in=4.0),
            "batched": lambda: W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7),
            "mc_bf16": lambda: W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="bf16")}[name]()
    a = ngb.from_spec(spec, deterministic=True, delivery="ring")
    with _env(NGB_MODE="fused"):
        b = ngb.from_spec(spec, deterministic=True, delivery="ring", drain_steps=250)
        b.finalize()
    assert b.stats()["mode"] == 2
    a.simulate(700)
    b.simulate(250)  # graphs of 100 steps and eager steps, in chunks of 250
    b.simulate_profiled(50)
    b.simulate(400)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert a.stats()["events"] == b.stats()["events"]
    for off in range(0, 4):
        assert np.array_equal(a.input(0, off), b.input(0, off))


@pytest.mark.parametrize("delivery", ["ring", "spike_buffer"])
def test_four_neurons_per_thread_equal_one(ngb, delivery):
    spec = W.microcircuit(scale=0.05, seed=5, keep_indegree=False)  # population sizes not multiples of 1024
    sims = []
    for npt in (1, 4):
        with _env(NGB_LIF_NPT=npt):
            s = ngb.from_spec(spec, deterministic=True, delivery=delivery)
            s.finalize()
        s.simulate(600)
        sims.append(s)
    a, b = sims
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert np.array_equal(a.state("I_syn"), b.state("I_syn"))
    assert a.stats()["events"] == b.stats()["events"]


@pytest.mark.parametrize("delivery", ["ring", "spike_buffer"])
def test_tiled_update_with_several_tiles_per_block(ngb, delivery):
    """Two or four neurons per thread on a network of more tiles than
    resident blocks (each block walks several tiles, crossing population
    boundaries, with the next tile's state prefetched and the spikes compacted
    once per block): bit-identical to one neuron per thread."""
    spec = W.NetSpec(name="tiles", seeds=[])
    for i in range(4):
        W.request_net(W.Request(arrival_s=0.0, n=110_000 + 333 * i, indegree=40, bio_time_ms=30.0, seed=100 + i),
                      spec, instance=i)
    sims = []
    for npt in (1, 2, 4):
        with _env(NGB_LIF_NPT=npt):
            s = ngb.from_spec(spec, deterministic=True, delivery=delivery)
            s.finalize()
        s.simulate(300)
        sims.append(s)
    a = sims[0]
    assert a.stats()["num_neurons"] > 400_000
    ai, at = a.spikes()
    assert len(ai) > 1000
    for b in sims[1:]:
        bi, bt = b.spikes()
        assert np.array_equal(at, bt) and np.array_equal(ai, bi)
        assert np.array_equal(a.state("V_m"), b.state("V_m"))
        assert np.array_equal(a.state("I_syn"), b.state("I_syn"))
        assert a.stats()["events"] == b.stats()["events"]


@pytest.mark.parametrize("name", ["adex", "paper_alpha", "mixed"])
def test_aeif_attempt_budget_does_not_change_results(ngb, name):
    """AdEx neurons not finished within the update kernel's attempt budget
    continue in a second kernel from their saved position: budgets 0 (no
    deferral), 1 (nearly every neuron deferred) and 8 give bit-identical runs,
    and so do the persistent and fused loops, which never defer."""
    spec = {"adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                            w_ex=2.0, w_in=4.0),
            "paper_alpha": lambda: W.paper_balanced(n_ex=1600, ce=160, seed=3),
            "mixed": lambda: W.mixed_net(seed=2)}[name]()
    runs = []
    for env in ({"NGB_AEIF_BUDGET": 0}, {"NGB_AEIF_BUDGET": 1}, {"NGB_AEIF_BUDGET": 8},
                {"NGB_MODE": "persistent"}, {"NGB_MODE": "fused"}):
        with _env(**env):
            sim = ngb.from_spec(spec, deterministic=True, delivery="ring", drain_steps=250)
            sim.finalize()
        sim.simulate(300)
        sim.simulate(300)
        runs.append(sim)
    a = runs[0]
    ai, at = a.spikes()
    assert len(ai) > 100
    for b in runs[1:]:
        bi, bt = b.spikes()
        assert np.array_equal(at, bt) and np.array_equal(ai, bi)
        for var in ("V_m", "w", "g_ex", "g_in", "h"):
            assert np.array_equal(a.state(var), b.state(var)), var
        assert a.stats()["rk_substeps"] == b.stats()["rk_substeps"]
        assert a.stats()["events"] == b.stats()["events"]


_LOOP_SPECS = {
    "balanced_lif": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
    "microcircuit": lambda: W.microcircuit(scale=0.03, seed=7, keep_indegree=False),
    "adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                    w_ex=2.0, w_in=4.0),
    "batched": lambda: W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7),
    "mc_bf16": lambda: W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="bf16"),
    "paper_alpha": lambda: W.paper_balanced(n_ex=1600, ce=160, seed=3),
    "mixed": lambda: W.mixed_net(seed=2),
}


@pytest.mark.parametrize("name", sorted(_LOOP_SPECS))
def test_pipelined_equals_per_step_kernels(ngb, name):
    spec = _LOOP_SPECS[name]()
    a = ngb.from_spec(spec, deterministic=True, delivery="ring")
    with _env(NGB_MODE="pipelined"):
        b = ngb.from_spec(spec, deterministic=True, delivery="ring", drain_steps=250)
        b.finalize()
    assert b.stats()["mode"] == 3
    a.simulate(700)
    b.simulate(250)  # 100-step graphs and eager steps, in chunks of 250
    b.simulate_profiled(50)
    b.simulate(400)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert a.stats()["events"] == b.stats()["events"]
    for off in range(0, 4):
        assert np.array_equal(a.input(0, off), b.input(0, off))


@pytest.mark.parametrize("name", ["balanced_lif", "microcircuit", "batched", "mc_bf16", "adex"])
def test_pipelined_one_kernel_equals_per_step_kernels(ngb, name):
    """The one-kernel pipelined loop (update of step t and delivery of step
    t - 1's queue in one launch, chained by programmatic dependent launch):
    bit-identical to the per-step kernels through graphs, eager and profiled
    steps; networks with AdEx populations use the per-step kernels."""
    spec = _LOOP_SPECS[name]()
    a = ngb.from_spec(spec, deterministic=True, delivery="ring")
    with _env(NGB_MODE="pipelined_one_kernel"):
        b = ngb.from_spec(spec, deterministic=True, delivery="ring", drain_steps=250)
        b.finalize()
    assert b.stats()["mode"] == (0 if name == "adex" else 5)
    a.simulate(700)
    b.simulate(250)
    b.simulate_profiled(50)
    b.simulate(7)
    b.simulate(393)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert a.stats()["events"] == b.stats()["events"]
    for off in range(0, 4):
        assert np.array_equal(a.input(0, off), b.input(0, off))


def test_pipelined_with_four_neurons_per_thread(ngb):
    spec = W.microcircuit(scale=0.05, seed=5, keep_indegree=False)
    a = ngb.from_spec(spec, deterministic=True, delivery="ring")
    with _env(NGB_MODE="pipelined", NGB_LIF_NPT=4):
        b = ngb.from_spec(spec, deterministic=True, delivery="ring")
        b.finalize()
    assert b.stats()["mode"] == 3
    a.simulate(600)
    b.simulate(600)
    assert np.array_equal(a.spikes()[0], b.spikes()[0]) and np.array_equal(a.spikes()[1], b.spikes()[1])
    assert np.array_equal(a.state("I_syn"), b.state("I_syn"))
