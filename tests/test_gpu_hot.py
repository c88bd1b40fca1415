"""Hot lists of the AdEx per-step kernels (Sec. 2.1: adaptive Runge-Kutta
integration of every AdEx neuron over each step).

A neuron whose step ends above V_T + c * Delta_T (c = 4 by default) is listed
for the next step, whose whole integration then runs in a warp of listed
neurons on a stream of its own, beside the update kernel, which skips it.
The arithmetic of every neuron's step is unchanged, so:

* deterministic runs (64-bit fixed-point inputs) are bit-identical with the
  lists on and off (NGB_AEIF_HOT=0): spikes, membrane potentials and every
  receptor's input, for the exponential, alpha and beta conductance models,
  under both delivery schemes, in the graph, pipelined and profiled (eager)
  launch paths, and across autotuning (snapshot restores, other loops tried);
* with a threshold just above V_T (c = 0.01) a large share of the neuron
  steps runs from the lists, still bit-identical;
* the lists are used: the hot-list kernel's neuron steps are counted.
"""
import os

import numpy as np
import pytest

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
        for k, v in self.kv.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = str(v)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


SPECS = {
    "paper_alpha": lambda: W.paper_balanced(n_ex=2000, ce=200, seed=4),
    "adex_exp": lambda: W.balanced_adex(n=3000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                        w_ex=2.0, w_in=4.0),
    "beta": lambda: W.beta_net(seed=3),
    "mixed": lambda: W.mixed_net(seed=3),
}


def _build(ngb, spec, hot, mode=None, **kw):
    with _env(NGB_AEIF_HOT=hot, NGB_MODE=mode):
        sim = ngb.from_spec(spec, deterministic=True, **kw)
        sim.finalize()
    return sim


def _receptors(spec):
    return max(2, max((len(p.params.ports) for p in spec.pops if getattr(p.params, "ports", None)), default=2))


def _same(a, b, R):
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    for r in range(R):
        assert np.array_equal(a.input(r, 0), b.input(r, 0)), r


@pytest.mark.parametrize("delivery", ["spike_buffer", "ring"])
@pytest.mark.parametrize("name", sorted(SPECS))
def test_hot_lists_bit_identical(ngb, name, delivery):
    spec = SPECS[name]()
    R = _receptors(spec)
    off = _build(ngb, spec, 0, delivery=delivery)
    on = _build(ngb, spec, None, delivery=delivery)
    for chunk in (1, 150, 600):
        off.simulate(chunk)
        on.simulate(chunk)
        _same(off, on, R)
    assert len(on.spikes()[0]) > 50
    assert off.stats()["hot_steps"] == 0
    assert on.stats()["hot_steps"] > 0
    assert on.stats()["rk_substeps"] == off.stats()["rk_substeps"]


@pytest.mark.parametrize("name", ["paper_alpha", "mixed"])
def test_hot_lists_low_threshold_stress(ngb, name):
    """c = 0.01: every neuron a hair above V_T is listed (a large share of all steps)."""
    spec = SPECS[name]()
    R = _receptors(spec)
    off = _build(ngb, spec, 0)
    on = _build(ngb, spec, 0.01)
    off.simulate(700)
    on.simulate(700)
    _same(off, on, R)
    assert on.stats()["hot_steps"] > 0.05 * 700 * spec.num_neurons()


def test_hot_lists_pipelined_and_profiled(ngb):
    spec = SPECS["paper_alpha"]()
    off = _build(ngb, spec, 0, delivery="ring")
    pipe = _build(ngb, spec, None, mode="pipelined", delivery="ring")
    assert pipe.stats()["mode"] == 3
    prof = _build(ngb, spec, None, delivery="ring")
    off.simulate(500)
    pipe.simulate(500)
    for _ in range(5):
        prof.simulate_profiled(100)
    _same(off, pipe, 2)
    _same(off, prof, 2)
    assert pipe.stats()["hot_steps"] > 0 and prof.stats()["hot_steps"] > 0


def test_hot_lists_across_autotune_and_persistent_loop(ngb):
    """Autotuning tries other loops and restores the state after each trial;
    a handle in the persistent loop keeps no lists.  Both leave the lists
    empty, so the next per-step steps start from a consistent state."""
    spec = SPECS["paper_alpha"]()
    ref = _build(ngb, spec, 0)
    tuned = _build(ngb, spec, None)
    pers = _build(ngb, spec, None, mode="persistent")
    assert pers.stats()["mode"] == 1
    ref.simulate(300)
    tuned.simulate(300)
    pers.simulate(300)
    tuned.autotune(100)
    ref.simulate(400)
    tuned.simulate(400)
    pers.simulate_profiled(200)  # per-step kernels after the persistent loop
    pers.simulate(200)
    _same(ref, tuned, 2)
    _same(ref, pers, 2)
    assert pers.stats()["hot_steps"] > 0
