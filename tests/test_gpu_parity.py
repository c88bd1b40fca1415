"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

* Connectivity (tgt, receptor, delay, row pointers) bit-exact; weights equal
  up to one FP32 ulp where the FP64 Box-Muller draw's last bit differs between
  CUDA's and the C library's log/cos (counted, must be rare).
* Deterministic mode (64-bit fixed-point ring): spike trains and state
  bit-exact for whole runs.
* FP32 mode: per-step input currents within 1e-5 x sum|w|; spike trains
  identical up to the first step decided by FP32 summation order, where every
  differing neuron must sit at threshold; long-run rates within 2 % and CV ISI
  within 0.05.
* AdEx: FP32-state GPU integration against the FP64 oracle.
"""
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


def _pair(ngb, spec, deterministic=False, **kw):
    g = ngb.from_spec(spec, deterministic=deterministic, **kw)
    g.finalize()
    o = oracle.OracleNet(spec, deterministic=deterministic, track_abs=True)
    o.finalize()
    return g, o


def _ulp_diff(a, b):
    ai = a.astype(np.float32).view(np.int32).astype(np.int64)
    bi = b.astype(np.float32).view(np.int32).astype(np.int64)
    return np.abs(ai - bi)


def _assert_same_csr(g, o):
    oc = o.csr()
    assert np.array_equal(g.src_ptr(), oc["src_ptr"])
    gs = g.synapses()
    assert np.array_equal(gs["tgt"], oc["tgt"])
    assert np.array_equal(gs["receptor"], oc["receptor"])
    assert np.array_equal(gs["delay"], oc["delay"])
    du = _ulp_diff(gs["weight"], oc["weight"])
    assert du.max(initial=0) <= 1
    assert np.count_nonzero(du) <= max(2, 1e-5 * len(du))
    st = g.stats()
    assert st["num_synapses"] == o.num_synapses
    assert st["max_delay_steps"] == int(oc["delay"].max(initial=0))
    return gs, oc


SPECS = {
    "balanced_lif_1000": lambda: W.balanced_lif(n=1000, indegree=100, seed=1),
    "microcircuit_0.02_total": lambda: W.microcircuit(scale=0.02, seed=3, keep_indegree=False),
    "balanced_adex_2000": lambda: W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32"),
    "microcircuit_bf16": lambda: W.microcircuit(scale=0.02, seed=4, keep_indegree=False, weight_dtype="bf16"),
    "microcircuit_fp16": lambda: W.microcircuit(scale=0.02, seed=5, keep_indegree=False, weight_dtype="fp16"),
    "rules_net": lambda: W.rules_net(seed=4),
}


@pytest.mark.parametrize("name", sorted(SPECS))
def test_connectivity_matches_oracle(ngb, name):
    spec = SPECS[name]()
    g, o = _pair(ngb, spec)
    _assert_same_csr(g, o)


def test_connectivity_without_autapses_and_ragged_sizes(ngb):
    spec = W.balanced_lif(n=333, indegree=37, seed=17)
    for c in spec.conns:
        c.allow_autapses = False
    spec.pops[0].n = 267  # ragged, not a multiple of any block size
    g, o = _pair(ngb, spec)
    gs, oc = _assert_same_csr(g, o)
    src = np.repeat(np.arange(g.stats()["num_neurons"]), np.diff(g.src_ptr().astype(np.int64)))
    assert not np.any(src == gs["tgt"])


def test_deterministic_balanced_lif_bit_exact(ngb):
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)  # the 1,000-neuron network, 100 ms
    g, o = _pair(ngb, spec, deterministic=True)
    for chunk in (1, 9, 90, 400, 500):
        g.simulate(chunk)
        o.simulate(chunk)
        assert np.array_equal(g.state("V_m"), o.state("V_m").astype(np.float32))
        assert np.array_equal(g.state("I_syn"), o.state("I_syn").astype(np.float32))
        assert np.array_equal(g.state("refractory"), o.state("refractory").astype(np.float32))
        assert np.array_equal(g.input(0, 0), o.input(0, 0)[0])
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    assert len(oi) > 1000
    assert np.array_equal(gt, ot) and np.array_equal(gi, oi)
    assert g.stats()["events"] == o.events


def test_deterministic_microcircuit_small_bit_exact(ngb):
    spec = W.microcircuit(scale=0.03, seed=7, keep_indegree=False)
    g, o = _pair(ngb, spec, deterministic=True, delivery="ring")  # reads future ring slots
    g.simulate(600)
    o.simulate(600)
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    assert len(oi) > 200
    assert np.array_equal(gt, ot) and np.array_equal(gi, oi)
    assert np.array_equal(g.state("V_m"), o.state("V_m").astype(np.float32))
    for off in range(0, 8):
        assert np.array_equal(g.input(0, off), o.input(0, off)[0])


def test_deterministic_rules_net_bit_exact(ngb):
    """One-to-one, fixed out-degree and all-to-all wiring, simulated."""
    spec = W.rules_net(seed=4)
    g, o = _pair(ngb, spec, deterministic=True)
    g.simulate(500)
    o.simulate(500)
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    assert len(oi) > 100
    assert np.array_equal(gt, ot) and np.array_equal(gi, oi)
    assert np.array_equal(g.state("V_m"), o.state("V_m").astype(np.float32))
    assert g.stats()["events"] == o.events


def test_deterministic_bf16_weights_bit_exact(ngb):
    spec = W.microcircuit(scale=0.03, seed=8, keep_indegree=False, weight_dtype="bf16")
    g, o = _pair(ngb, spec, deterministic=True)
    g.simulate(400)
    o.simulate(400)
    gi, gt = g.spikes()
    oi, ot = o.spikes()
    assert np.array_equal(gt, ot) and np.array_equal(gi, oi)


def _arrival_counts(csr, ids, steps, step, N):
    """Synapses whose spike arrives at `step`, per target neuron (each adds one
    term to the target's input sum of that step)."""
    sp = csr["src_ptr"].astype(np.int64)
    cnt = np.zeros(N, dtype=np.int64)
    D = int(csr["delay"].max(initial=0))
    sel = (steps >= step - D) & (steps < step)
    for s_, t_ in zip(ids[sel], steps[sel]):
        row = slice(sp[s_], sp[s_ + 1])
        hit = csr["delay"][row].astype(np.int64) == step - t_
        np.add.at(cnt, csr["tgt"][row][hit].astype(np.int64), 1)
    return cnt


def test_fp32_inputs_and_spikes_until_summation_order_decides(ngb):
    """FP32 mode: per-step inputs within 1e-5 of the summed magnitudes; the GPU
    state stays within a rounding bound of the oracle's, and the first step
    whose spikes differ is one where summation order decides: every differing
    neuron's pre-threshold potential, from the ORACLE's state, lies within
    that bound of the threshold.  The bound follows the sums' rounding: an
    input of n terms summed in any order in FP32 differs from another order by
    at most (n - 1) 2^-23 sum|w|; it enters I, and V through the propagators
    (I -> P11 I, V -> P22 V + P21 I), with one ulp per FP32 operation of the
    update once the two states differ, and 4 ulp of the threshold for the test
    itself."""
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    g, o = _pair(ngb, spec)
    N = 1000
    lif = spec.pops[0].params
    P = oracle.lif_propagators(lif.tau_m, lif.C_m, lif.tau_syn, spec.dt)
    theta = lif.V_th - lif.E_L
    csr = o.csr()
    ulp = lambda x: np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)
    eY = np.zeros(N)  # bounds of |y_gpu - y_oracle| and |I_gpu - I_oracle| before the step
    eI = np.zeros(N)
    steps_same = 0
    for step in range(1000):
        gin = g.input(0, 0)
        oin, oabs, oex = o.input(0, 0)
        # per-step input: within 1e-5 of the summed magnitudes of the contributing weights
        assert np.all(np.abs(gin.astype(np.float64) - oex) <= 1e-5 * oabs + 1e-6), step
        Vo, Io, ro = o.state("V_m"), o.state("I_syn"), o.state("refractory")
        yo = Vo - lif.E_L
        Vg, Ig = g.state("V_m").astype(np.float64), g.state("I_syn").astype(np.float64)
        # the state differences stay within the bound (the GPU reports V = y + E_L rounded to FP32: one
        # more half ulp of V)
        assert np.all(np.abs(Vg - Vo) <= eY + ulp(Vo)) and np.all(np.abs(Ig - Io) <= eI), step
        oi_all, ot_all = o.spikes()
        n_terms = _arrival_counts(csr, oi_all, ot_all, step, N)
        delta = np.maximum(n_terms - 1, 0) * 2.0 ** -23 * oabs
        y_pre = P["P22"] * yo + P["P21"] * Io + P["P20"] * lif.I_e
        busy = (eY > 0) | (eI > 0)
        e_pre = P["P22"] * eY + P["P21"] * eI + np.where(busy, 4 * ulp(np.maximum(np.abs(yo), np.abs(y_pre))), 0.0)
        g.simulate(1)
        o.simulate(1)
        gi, gt = g.spikes(t0=step, t1=step + 1)
        oi_new, ot_new = o.spikes()
        oi = oi_new[ot_new == step]
        if not np.array_equal(np.sort(gi), np.sort(oi)):
            # first divergence: every differing neuron sat within the rounding bound of threshold
            diff = np.setxor1d(gi, oi)
            near = np.abs(y_pre[diff] - theta)
            assert np.all(ro[diff] == 0) and np.all(near <= e_pre[diff] + 4 * ulp(np.float32(theta))), \
                (step, diff, near, e_pre[diff])
            break
        steps_same += 1
        spiked = np.zeros(N, dtype=bool)
        spiked[oi] = True
        held = (ro > 0) | spiked  # V held or reset identically on both sides
        I_new = P["P11"] * Io + oex
        eY = np.where(held, 0.0, e_pre)
        mag = np.maximum(np.maximum(np.abs(Io), np.abs(I_new)), np.abs(oex))
        eI = P["P11"] * eI + delta + np.where((eI > 0) | (delta > 0), 3 * ulp(mag), 0.0)
    assert steps_same >= 50


def _rates_cv(ids, steps, n, t_lo, t_hi, dt):
    m = (steps >= t_lo) & (steps < t_hi)
    ids, steps = ids[m], steps[m]
    rate = len(ids) / n / ((t_hi - t_lo) * dt * 1e-3)
    cvs = []
    order = np.lexsort((steps, ids))
    ids, steps = ids[order], steps[order]
    bounds = np.flatnonzero(np.diff(ids)) + 1
    for a, b in zip(np.r_[0, bounds], np.r_[bounds, len(ids)]):
        if b - a >= 4:
            isi = np.diff(steps[a:b]).astype(np.float64)
            cvs.append(isi.std() / isi.mean())
    return rate, float(np.mean(cvs)) if cvs else float("nan")


def test_fp32_long_run_rates_and_cv(ngb):
    steps = 10_000  # 1 s
    rg, ro, cg, co = [], [], [], []
    for seed in (1, 2, 3):
        spec = W.balanced_lif(n=1000, indegree=100, seed=seed)
        g, o = _pair(ngb, spec)
        g.simulate(steps)
        o.simulate(steps)
        a = _rates_cv(*g.spikes(), 1000, 1000, steps, spec.dt)
        b = _rates_cv(*o.spikes(), 1000, 1000, steps, spec.dt)
        rg.append(a[0]); cg.append(a[1]); ro.append(b[0]); co.append(b[1])
    assert abs(np.mean(rg) - np.mean(ro)) <= 0.02 * np.mean(ro), (rg, ro)
    assert abs(np.mean(cg) - np.mean(co)) <= 0.05, (cg, co)


@pytest.mark.parametrize("k", [4, 5])
def test_adex_step_factor_bit_exact_against_oracle(ngb, k):
    """The Runge-Kutta step-size factor of the FP32-state AdEx integration is
    one exactly specified FP32 operation sequence: the kernel's and the
    oracle's agree bit for bit over 60 binades and at the range edges."""
    rng = np.random.default_rng(10 + k)
    r = np.concatenate([np.float32(2.0) ** rng.uniform(-30, 30, 20000),
                        rng.uniform(0.5, 2.0, 5000), [1e-31, 2.0 ** -100, 2.0 ** 100, np.inf, np.nan, 1.0]])
    r = r.astype(np.float32)
    got = ngb.eval_step_factor(r, k)
    want = np.array([oracle.step_factor_root(float(x), k) for x in r], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _adex_single(I_e, ctl32=False):
    par = W.AeifParams(V_reset=-60.0, tau_ex=1.0, tau_in=1.0, I_e=I_e, rk_h_min=1e-9, rk_max_substeps=100000,
                       rk_control_fp32=ctl32)
    return W.NetSpec(name="adex1", seeds=[1], pops=[W.Population("n", W.AEIF, 1, par)])


@pytest.mark.parametrize("ctl32", [False, True])
def test_adex_single_neuron_700pA_vs_fp64_oracle(ngb, ctl32):
    spec = _adex_single(700.0, ctl32)
    g = ngb.from_spec(spec)
    g.finalize()
    o = oracle.OracleNet(spec, adex_fp64=True)
    o.finalize()
    steps = 1500
    Vg = np.zeros(steps)
    Vo = np.zeros(steps)
    for k in range(steps):
        g.simulate(1)
        o.simulate(1)
        Vg[k] = g.state("V_m")[0]
        Vo[k] = o.state("V_m")[0]
    sg = g.spikes()[1]
    so = o.spikes()[1]
    assert len(so) >= 3 and len(sg) == len(so)
    assert np.all(np.abs(sg - so) <= 1)
    mask = np.ones(steps, dtype=bool)
    for s in so:
        mask[max(0, s - 20):s + 2] = False
    assert np.abs(Vg - Vo)[mask].max() <= 5e-3


@pytest.mark.parametrize("ctl32", [False, True])
def test_adex_network_matches_fp32_oracle_statistics(ngb, ctl32):
    spec = W.balanced_adex(n=2000, indegree=100, seed=2, weight_dtype="fp32", poisson_weight=4.0, w_ex=2.0,
                           w_in=4.0)
    for p in spec.pops:
        p.params.rk_control_fp32 = ctl32
    g, o = _pair(ngb, spec)
    g.simulate(2000)
    o.simulate(2000)
    ng, no = len(g.spikes()[0]), len(o.spikes()[0])
    assert no > 200
    assert abs(ng - no) <= 0.05 * no + 10, (ng, no)
    # identical for the first steps, before any order-dependent rounding
    gi, gt = g.spikes(t0=0, t1=50)
    oi, ot = o.spikes()
    assert np.array_equal(np.sort(gi), np.sort(oi[ot < 50]))
    st = g.stats()
    assert st["rk_substeps"] > 2000 * 2000


def test_adex_alpha_single_neuron_vs_fp64_oracle(ngb):
    """Alpha-function conductances (Sec. 2.4): a neuron driven by a current
    and by Poisson input through the alpha conductance (identical counts on
    both sides), GPU (FP32 state) against the FP64 oracle."""
    par = W.AeifParams(V_reset=-60.0, tau_ex=1.0, tau_in=1.0, I_e=450.0, rk_h_min=1e-9, rk_max_substeps=100000,
                       poisson=W.Poisson(n_inputs=1.0, rate_hz=20000.0, weight=0.37, receptor=0))
    spec = W.NetSpec(name="alpha1", seeds=[1], pops=[W.Population("n", W.AEIF_ALPHA, 1, par)])
    g = ngb.from_spec(spec)
    g.finalize()
    o = oracle.OracleNet(spec, adex_fp64=True)
    o.finalize()
    steps = 1500
    Vg, Vo, Gg, Go = (np.zeros(steps) for _ in range(4))
    for k in range(steps):
        g.simulate(1)
        o.simulate(1)
        Vg[k], Vo[k] = g.state("V_m")[0], o.state("V_m")[0]
        Gg[k], Go[k] = g.state("g_ex")[0], o.state("g_ex")[0]
    assert Go.max() > 5.0  # the alpha conductance carries the drive
    assert np.abs(Gg - Go).max() <= 1e-4 * Go.max()
    sg, so = g.spikes()[1], o.spikes()[1]
    assert len(so) >= 3 and len(sg) == len(so)
    assert np.all(np.abs(sg - so) <= 1)
    mask = np.ones(steps, dtype=bool)
    for s_ in so:
        mask[max(0, s_ - 20):s_ + 2] = False
    assert np.abs(Vg - Vo)[mask].max() <= 5e-3


def test_adex_alpha_network_matches_fp32_oracle_statistics(ngb):
    """The paper's balanced network at 2,500 neurons, in-degree 250."""
    spec = W.paper_balanced(n_ex=2000, ce=200, seed=2)
    g, o = _pair(ngb, spec)
    for step in range(40):
        gin = g.input(0, 0).astype(np.float64)
        _, oabs, oex = o.input(0, 0)
        assert np.all(np.abs(gin - oex) <= 1e-5 * oabs + 1e-7), step
        g.simulate(1)
        o.simulate(1)
    g.simulate(1960)
    o.simulate(1960)
    ng, no = len(g.spikes()[0]), len(o.spikes()[0])
    assert no > 5000
    assert abs(ng - no) <= 0.05 * no, (ng, no)
    gi, gt = g.spikes(t0=0, t1=30)
    oi, ot = o.spikes()
    assert np.array_equal(np.sort(gi), np.sort(oi[ot < 30]))


def test_mixed_models_match_oracle_statistics(ngb):
    """LIF, exponential and alpha AdEx populations in one network: per-step
    inputs on both receptors within the FP32 bound, per-population spike
    counts within 5 % of the oracle's over 100 ms."""
    spec = W.mixed_net(seed=2)
    g, o = _pair(ngb, spec)
    for step in range(30):
        for r in (0, 1):
            gin = g.input(r, 0).astype(np.float64)
            _, oabs, oex = o.input(r, 0)
            assert np.all(np.abs(gin - oex) <= 1e-5 * oabs + 1e-7), (step, r)
        g.simulate(1)
        o.simulate(1)
    g.simulate(970)
    o.simulate(970)
    gi, oi = g.spikes()[0], o.spikes()[0]
    bounds = [0, 400, 700, 1000]
    for p in range(3):
        ng = np.count_nonzero((gi >= bounds[p]) & (gi < bounds[p + 1]))
        no = np.count_nonzero((oi >= bounds[p]) & (oi < bounds[p + 1]))
        assert no > 100 and abs(ng - no) <= 0.05 * no + 10, (p, ng, no)


def test_graph_and_eager_paths_identical(ngb):
    spec = W.microcircuit(scale=0.02, seed=9, keep_indegree=False)
    a = ngb.from_spec(spec, deterministic=True)  # default: 100-step graphs
    b = ngb.from_spec(spec, deterministic=True, steps_per_graph=-1)
    c = ngb.from_spec(spec, deterministic=True, steps_per_graph=7, drain_steps=50)
    a.simulate(350)
    b.simulate(350)
    ms, n = c.simulate_profiled(350)
    for x in (b, c):
        assert np.array_equal(a.spikes()[0], x.spikes()[0])
        assert np.array_equal(a.spikes()[1], x.spikes()[1])
    assert n[0] == 350 and n[2] == 350 and ms[0] > 0 and ms[2] > 0


def test_record_overflow_is_reported(ngb):
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    g = ngb.from_spec(spec, record_capacity=16, drain_steps=500)
    with pytest.raises(ngb.NgbError) as e:
        g.simulate(1000)
    assert e.value.code == -6
    # the simulation itself carried on; the counters still count every spike
    assert g.stats()["steps"] == 1000 and g.stats()["spikes"] > 16


def test_edge_cases_empty_and_single(ngb):
    # a population with no connections and no drive, and a one-neuron population
    spec = W.NetSpec(name="edge", seeds=[5])
    spec.pops = [W.Population("a", W.LIF, 1, W.LifParams(I_e=500.0)),
                 W.Population("b", W.LIF, 70, W.LifParams())]
    spec.conns = [W.Connection(0, 1, W.TOTAL, 0, W.Dist("const", 10.0), W.Dist("const", 1.0))]
    g, o = _pair(ngb, spec, deterministic=True)
    g.simulate(1000)
    o.simulate(1000)
    assert np.array_equal(g.spikes()[1], o.spikes()[1])
    # constant 500 pA: one spike every 20 + 139 steps
    assert g.stats()["num_synapses"] == 0 and len(g.spikes()[0]) == 6
    assert np.all(g.state("V_m")[1:] == -65.0)
    with pytest.raises(ngb.NgbError):
        g.connect(0, 1, W.TOTAL, 1, W.Dist("const", 1.0), W.Dist("const", 1.0))  # after finalise
