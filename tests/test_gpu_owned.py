"""The target-owned persistent step loop (each block owns a tile of neurons
with its ring buffer in shared memory; spikes exchanged through stamped
mailboxes) against the per-step kernels, through the C ABI (needs a GB300).

* Deterministic mode (int64 fixed-point ring): bit-identical spike trains,
  membrane state, synaptic current, inputs of the coming steps and event
  counts, over launches of 1, 2, 97 and 250 steps and a switch to the
  profiled per-step kernels and back; LIF networks with one and several
  populations, batched instances, BF16 and FP16 weights, fewer neurons than blocks,
  no synapses at all, a network whose first step fires thousands of
  neurons (mailbox overflow areas, more spikes than the shared-memory list
  holds), and busy networks of 160,000 neurons with 1,000 inputs each that
  fire thousands of spikes in every step, in bursts of well over 2,048
  (tiles of 1,053 neurons, more than 1,024 per block: 8-byte items for BF16
  weights too; every step through the overflow areas, and the bursts past
  the shared-memory entry list).
* FP32 mode: after one step the ring slots hold the same sums as the
  per-step kernels within the FP32 summation bound (1e-5 of the summed
  magnitudes), and spike counts agree within 5 % over 3,000 steps.
* Networks the loop does not take (AdEx populations, the spike-buffer
  scheme, serving handles, more than 2,048 neurons per block) run the
  per-step kernels.
* A block that never publishes (test hook) makes every mailbox wait give up
  after its poll limit: ngb_simulate returns NGB_ERR_TIMEOUT, and the GPU
  stays usable.
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
        os.environ.update({k: str(v) for k, v in self.kv.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


_SPECS = {
    "balanced_lif": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
    "microcircuit": lambda: W.microcircuit(scale=0.03, seed=7, keep_indegree=False),
    "mc_burst": lambda: W.microcircuit(scale=0.3, seed=9, keep_indegree=False),
    "batched": lambda: W.batched_microcircuits(n_instances=3, scale_lo=0.02, scale_hi=0.04, seed=7),
    "mc_bf16": lambda: W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="bf16"),
    "mc_fp16": lambda: W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="fp16"),
    "adex": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0,
                                    w_ex=2.0, w_in=4.0),
    "tiny": lambda: W.balanced_lif(n=100, indegree=10, seed=3),  # fewer neurons than blocks
    "unconnected": lambda: _unconnected(),                       # no synapses at all
    # thousands of spikes in every step; more than 1,024 neurons per tile
    "busy": lambda: W.balanced_lif(n=160_000, indegree=1000, seed=5),
    "busy_bf16": lambda: W.balanced_lif(n=160_000, indegree=1000, seed=6, weight_dtype="bf16"),
}


def _unconnected():
    lif = W.LifParams(V_init_mean=-65.0, V_init_sd=4.0, poisson=W.Poisson(n_inputs=1000.0, rate_hz=11.0, weight=87.8))
    spec = W.NetSpec(name="unconnected", seeds=[5])
    spec.pops = [W.Population("a", W.LIF, 300, lif)]
    return spec


def _owned(ngb, spec, **kw):
    with _env(NGB_MODE="target_owned"):
        sim = ngb.from_spec(spec, **kw)
        sim.finalize()
    return sim


@pytest.mark.parametrize("name", sorted(_SPECS))
def test_target_owned_equals_per_step_kernels(ngb, name):
    spec = _SPECS[name]()
    kw = {"record_capacity": 8_000_000} if name.startswith("busy") else {}  # ~3,000 spikes per step
    a = ngb.from_spec(spec, deterministic=True, delivery="ring", **kw)
    b = _owned(ngb, spec, deterministic=True, delivery="ring", drain_steps=250, **kw)
    assert b.stats()["mode"] == (0 if name == "adex" else 6)
    if name != "adex":
        assert b.stats()["launch_grid"] > 0
    a.simulate(700)
    for chunk in (1, 2, 97, 300, 300):  # launches of 1, 2 and 97 steps, then chunks of 250
        b.simulate(chunk)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert len(ai) > 50
    if name == "mc_burst":
        assert np.count_nonzero(at == 0) > 3000  # the first step fires thousands of neurons
    if name.startswith("busy"):
        assert len(ai) > 1000 * 1000  # over a thousand spikes per step on average
    assert np.array_equal(at, bt) and np.array_equal(ai, bi)
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    assert np.array_equal(a.state("I_syn"), b.state("I_syn"))
    assert a.stats()["events"] == b.stats()["events"]
    if name == "unconnected":
        assert a.stats()["events"] == 0
    for off in range(0, min(6, a.stats()["ring_slots"])):
        assert np.array_equal(a.input(0, off), b.input(0, off)), off
    b.simulate_profiled(20)  # per-step kernels after a target-owned launch, then back
    b.simulate(30)
    a.simulate(50)
    assert np.array_equal(a.spikes()[0], b.spikes()[0]) and np.array_equal(a.spikes()[1], b.spikes()[1])
    assert np.array_equal(a.state("V_m"), b.state("V_m"))
    for off in range(0, min(6, a.stats()["ring_slots"])):
        assert np.array_equal(a.input(0, off), b.input(0, off)), off


def _slot_magnitudes(sim, ids, steps, n, L):
    """Sum of |w| of the synapses of the given spikes, per ring slot offset
    and target (FP64), for the spikes of one step."""
    syn = sim.synapses()
    ptr = sim.src_ptr().astype(np.int64)
    mag = np.zeros((L, n))
    for s in ids:
        sl = slice(ptr[s], ptr[s + 1])
        np.add.at(mag, (syn["delay"][sl].astype(np.int64), syn["tgt"][sl].astype(np.int64)),
                  np.abs(syn["weight"][sl].astype(np.float64)))
    return mag


def test_target_owned_fp32_sums_and_rates(ngb):
    spec = W.microcircuit(scale=0.1, seed=11, keep_indegree=False)
    a = ngb.from_spec(spec, delivery="ring")
    b = _owned(ngb, spec, delivery="ring")
    assert b.stats()["mode"] == 6
    a.simulate(1)
    b.simulate(1)
    ai, at = a.spikes()
    bi, bt = b.spikes()
    assert np.array_equal(ai, bi) and len(ai) > 100  # step 0 has no synaptic input: same spikes
    n = a.stats()["num_neurons"]
    L = a.stats()["ring_slots"]
    mag = _slot_magnitudes(a, ai, at, n, L)
    for off in range(0, L - 1):
        ga = a.input(0, off).astype(np.float64)
        gb = b.input(0, off).astype(np.float64)
        # slot of step 1 + off holds the spikes of step 0 with delay 1 + off
        assert np.all(np.abs(ga - gb) <= 1e-5 * mag[1 + off] + 1e-7), off
    a.simulate(2999)
    b.simulate(2999)
    na, nb = len(a.spikes()[0]), len(b.spikes()[0])
    assert na > 5000 and abs(na - nb) <= 0.05 * na, (na, nb)


def test_target_owned_not_taken(ngb):
    spec = W.microcircuit(scale=0.03, seed=7, keep_indegree=False)
    sb = _owned(ngb, spec, delivery="spike_buffer")
    assert sb.stats()["mode"] == 0 and sb.stats()["delivery"] == 2
    sb.simulate(20)
    assert sb.stats()["steps"] == 20
    with _env(NGB_MODE="target_owned"):  # serving handles: instances come and go, no static layout
        sv = ngb.Simulator(deterministic=True)
        sv.reserve(5000, 400_000, 5000, 16, 1)
        a, _ = sv.add_spec_instance(W.balanced_lif(n=3000, indegree=100, seed=1))
        sv.commit(a)
        sv.simulate(50)
    assert sv.stats()["mode"] == 0 and sv.stats()["steps"] == 50
    big = W.balanced_lif(n=400_000, indegree=10, seed=1)  # more than 2,048 neurons per block
    bg = _owned(ngb, big, delivery="ring")
    assert bg.stats()["mode"] == 0
    bg.simulate(5)
    assert bg.stats()["steps"] == 5


def test_target_owned_mailbox_wait_is_bounded(ngb):
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    with _env(NGB_TEST_WITHHOLD_BLOCK=0, NGB_BARRIER_SPIN_LIMIT=20000):
        sim = _owned(ngb, spec, delivery="ring")
    assert sim.stats()["mode"] == 6
    with pytest.raises(ngb.NgbError) as e:
        sim.simulate(50)
    assert e.value.code == -5  # NGB_ERR_TIMEOUT
    sim.close()
    ok = _owned(ngb, spec, deterministic=True, delivery="ring")
    ok.simulate(100)
    assert ok.stats()["steps"] == 100 and ok.stats()["mode"] == 6


def test_autotune_cache_round_trip(ngb, tmp_path):
    """NGB_AUTOTUNE_CACHE: the first tuning appends one line per network shape
    and a second handle of the same shape takes its loop from the file without
    timing; a line naming the target-owned loop selects it, and the run is
    bit-identical to the per-step kernels."""
    spec = W.microcircuit(scale=0.03, seed=3, keep_indegree=False)
    cache = tmp_path / "tune.txt"
    with _env(NGB_AUTOTUNE_CACHE=str(cache)):
        a = ngb.from_spec(spec, deterministic=True, delivery="ring")
        ga = a.autotune(200)
        b = ngb.from_spec(spec, deterministic=True, delivery="ring")
        gb = b.autotune(200)
    lines = [ln for ln in cache.read_text().splitlines() if ln.strip()]
    assert len(lines) == 1 and len(lines[0].split()) == 5
    assert a.stats()["mode"] == b.stats()["mode"] and ga == gb
    key, _, g, pg, _ = lines[0].split()
    forced = tmp_path / "forced.txt"
    forced.write_text("%s 6 %s %s 1\n" % (key, g, pg))
    with _env(NGB_AUTOTUNE_CACHE=str(forced)):
        c = ngb.from_spec(spec, deterministic=True, delivery="ring")
        c.autotune(200)
    assert c.stats()["mode"] == 6 and c.stats()["steps"] == 0
    ref = ngb.from_spec(spec, deterministic=True, delivery="ring")
    c.simulate(400)
    ref.simulate(400)
    assert np.array_equal(c.spikes()[0], ref.spikes()[0]) and np.array_equal(c.spikes()[1], ref.spikes()[1])


def test_target_owned_16bit_items_bit_exact_against_oracle(ngb):
    """BF16 and FP16 weights travel as 4-byte items (weight bits, delay and
    local target in one word): spike trains bit-exact against the oracle in
    deterministic mode, and the item layout half the bytes of the FP32 one."""
    import oracle
    held = {}
    for wd in ("bf16", "fp16", "fp32"):
        spec = W.microcircuit(scale=0.05, seed=8, keep_indegree=False, weight_dtype=wd)
        b = _owned(ngb, spec, deterministic=True, delivery="ring")
        assert b.stats()["mode"] == 6
        o = oracle.OracleNet(spec, deterministic=True)
        o.finalize()
        b.simulate(400)
        o.simulate(400)
        bi, bt = b.spikes()
        oi, ot = o.spikes()
        assert len(oi) > 100
        assert np.array_equal(bt, ot) and np.array_equal(bi, oi), wd
        held[wd] = b.stats()["device_bytes"]
        b.close()
    # same network: the 16-bit handles hold 2-byte weights and 4-byte items against 4 + 8
    K = W.microcircuit(scale=0.05, seed=8, keep_indegree=False).num_synapses()
    assert held["fp32"] - held["bf16"] > 2 * K
