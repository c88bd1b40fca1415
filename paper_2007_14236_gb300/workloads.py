"""Seeded synthetic workloads: network specifications only.

This module holds the recipes of the benchmark networks (population sizes,
neuron parameters, connection rules, weight/delay distributions, seeds) as
plain data.  It contains none of the method's arithmetic, so both the GPU
library binding and the CPU oracle build their networks from the same
description without sharing any simulation code.

Networks (all dt = 0.1 ms):
  * balanced_lif      -- 1,000 LIF neurons (800 E / 200 I), fixed in-degree 100.
  * microcircuit      -- the 8-population Potjans-Diesmann cortical
                         microcircuit (Sec. 2.3 of the paper), ~77k LIF
                         neurons, per-pathway synapse counts from the
                         connection probabilities (~3e8 synapses at scale 1).
  * balanced_adex     -- Brunel-type E/I network of AdEx neurons with
                         conductance synapses (Sec. 2.4), fixed in-degree.
  * batched_microcircuits / served_requests -- many independent instances.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

LIF = "lif_psc_exp"
AEIF = "aeif_cond_exp"
AEIF_ALPHA = "aeif_cond_alpha"  # AdEx with alpha-function conductances
AEIF_BETA = "aeif_cond_beta"    # multisynapse AdEx with beta-function conductances
INDEGREE = "fixed_indegree"
TOTAL = "fixed_total_number"
OUTDEGREE = "fixed_outdegree"
ONE_TO_ONE = "one_to_one"
ALL_TO_ALL = "all_to_all"


@dataclass
class Poisson:
    n_inputs: float = 0.0
    rate_hz: float = 0.0
    weight: float = 0.0
    receptor: int = 0


@dataclass
class LifParams:
    tau_m: float = 10.0
    C_m: float = 250.0
    E_L: float = -65.0
    V_reset: float = -65.0
    V_th: float = -50.0
    t_ref: float = 2.0
    tau_syn: float = 0.5
    I_e: float = 0.0
    V_init_mean: float = -65.0
    V_init_sd: float = 0.0
    poisson: Poisson = field(default_factory=Poisson)


@dataclass
class AeifParams:
    C_m: float = 281.0
    g_L: float = 30.0
    E_L: float = -70.6
    V_T: float = -50.4
    Delta_T: float = 2.0
    a: float = 4.0
    b: float = 80.5
    tau_w: float = 144.0
    V_peak: float = 0.0
    V_reset: float = -70.6
    E_ex: float = 0.0
    E_in: float = -85.0
    tau_ex: float = 0.2
    tau_in: float = 2.0
    I_e: float = 0.0
    V_init_mean: float = -70.6
    V_init_sd: float = 0.0
    w_init: float = 0.0
    rk_tol: float = 1e-10
    rk_h_min: float = 1e-6
    rk_h_init: float = 0.1
    rk_max_substeps: int = 10000
    rk_control_fp32: bool = False
    poisson: Poisson = field(default_factory=Poisson)
    # AEIF_BETA only: up to four synaptic ports (E_rev mV, tau_rise ms, tau_decay ms); the
    # E_ex / E_in / tau_ex / tau_in fields are then unused
    ports: Optional[List[Tuple[float, float, float]]] = None


@dataclass
class Dist:
    kind: str = "const"  # const | normal | uniform
    p0: float = 0.0
    p1: float = 0.0


@dataclass
class Population:
    name: str
    model: str
    n: int
    params: object
    instance: int = 0


@dataclass
class Stdp:
    """Nearest-neighbour STDP of a connection's synapses (Sec. 2.1): pair
    time constants (ms), learning rate lambda, depression ratio alpha, weight
    exponents mu (0 additive, 1 multiplicative) and the weight bound W_max."""
    tau_plus: float = 20.0
    tau_minus: float = 20.0
    lam: float = 0.01
    alpha: float = 1.0
    mu_plus: float = 1.0
    mu_minus: float = 1.0
    W_max: float = 100.0


@dataclass
class Connection:
    src: int
    tgt: int
    rule: str
    K: int
    weight: Dist
    delay: Dist
    receptor: int = 0
    allow_autapses: bool = True
    stdp: Optional[Stdp] = None


@dataclass
class NetSpec:
    name: str
    dt: float = 0.1
    seeds: List[int] = field(default_factory=lambda: [1])  # one seed per instance
    pops: List[Population] = field(default_factory=list)
    conns: List[Connection] = field(default_factory=list)
    weight_dtype: str = "fp32"  # fp32 | bf16 | fp16

    def num_neurons(self) -> int:
        return sum(p.n for p in self.pops)

    def num_synapses(self) -> int:
        total = 0
        for c in self.conns:
            ns, nt = self.pops[c.src].n, self.pops[c.tgt].n
            total += {INDEGREE: c.K * nt, TOTAL: c.K, OUTDEGREE: c.K * ns, ONE_TO_ONE: ns,
                      ALL_TO_ALL: ns * (ns - 1) if (c.src == c.tgt and not c.allow_autapses) else ns * nt}[c.rule]
        return total

    def instance_pops(self, instance: int) -> List[int]:
        return [i for i, p in enumerate(self.pops) if p.instance == instance]


# ----------------------------------------------------------------- config 0
def balanced_lif(n: int = 1000, indegree: int = 100, seed: int = 1, rate_hz: float = 8.0,
                 n_ext: float = 1000.0, j_ex: float = 87.8, g: float = 4.0,
                 d_ex: float = 1.5, d_in: float = 0.8, V_init_sd: float = 0.0,
                 weight_dtype: str = "fp32") -> NetSpec:
    """Plain small LIF balanced net: 80 % excitatory, fixed in-degree (80 % from E,
    20 % from I), constant weights and delays, independent Poisson drive."""
    n_e = (n * 4) // 5
    n_i = n - n_e
    k_e = (indegree * 4) // 5
    k_i = indegree - k_e
    par = LifParams(V_init_mean=-65.0, V_init_sd=V_init_sd,
                    poisson=Poisson(n_inputs=n_ext, rate_hz=rate_hz, weight=j_ex))
    spec = NetSpec(name="balanced_lif_%d" % n, seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("E", LIF, n_e, par), Population("I", LIF, n_i, replace(par))]
    for tgt in (0, 1):
        spec.conns.append(Connection(0, tgt, INDEGREE, k_e, Dist("const", j_ex), Dist("const", d_ex)))
        spec.conns.append(Connection(1, tgt, INDEGREE, k_i, Dist("const", -g * j_ex), Dist("const", d_in)))
    return spec


def stdp_net(n: int = 1000, indegree: int = 100, seed: int = 1, mu: float = 1.0, lam: float = 0.01,
             alpha: float = 1.05, j_ex: float = 87.8, rate_hz: float = 8.0, V_init_sd: float = 4.0) -> NetSpec:
    """The small balanced LIF net with plastic excitatory-to-excitatory
    synapses (nearest-neighbour STDP, Sec. 2.1): initial weights
    Normal(j_ex, 0.1 j_ex), W_max = 2 j_ex, delays Uniform(1, 2) ms, pair time
    constants 16.8 / 33.7 ms, weight exponents mu (0 additive, 1
    multiplicative)."""
    spec = balanced_lif(n=n, indegree=indegree, seed=seed, rate_hz=rate_hz, j_ex=j_ex, V_init_sd=V_init_sd)
    spec.name = "stdp_net_%d" % n
    ee = spec.conns[0]
    assert ee.src == 0 and ee.tgt == 0
    ee.weight = Dist("normal", j_ex, 0.1 * j_ex)
    ee.delay = Dist("uniform", 1.0, 2.0)
    ee.stdp = Stdp(tau_plus=16.8, tau_minus=33.7, lam=lam, alpha=alpha, mu_plus=mu, mu_minus=mu, W_max=2.0 * j_ex)
    return spec


def paper_balanced(n_ex: int = 8000, ce: int = 800, seed: int = 1, weight_dtype: str = "fp32",
                   rk_tol: float = 1e-10, rk_control_fp32: bool = False) -> NetSpec:
    """The paper's balanced network (Sec. 2.4 with its two parameter tables):
    N_in = N_ex / 4 and CI = CE / 4 (fixed in-degree), AdEx with alpha-function
    conductances (tau_syn 1 ms on both receptors), V_r = -60 mV, weights
    0.05 nS (excitatory) and 0.35 nS (inhibitory, receptor 1), delays
    Normal(0.5, 0.25) ms re-drawn below dt, Poisson drive 20 kHz x 0.37 nS on
    both populations.  Initial V = E_L, w = 0 (the paper gives none)."""
    n_in = n_ex // 4
    ci = ce // 4
    par = AeifParams(V_reset=-60.0, tau_ex=1.0, tau_in=1.0, rk_tol=rk_tol, rk_control_fp32=rk_control_fp32,
                     poisson=Poisson(n_inputs=1.0, rate_hz=20000.0, weight=0.37, receptor=0))
    spec = NetSpec(name="paper_balanced_%d_%d" % (n_ex + n_in, ce + ci), seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("E", AEIF_ALPHA, n_ex, par), Population("I", AEIF_ALPHA, n_in, replace(par))]
    for tgt in (0, 1):
        spec.conns.append(Connection(0, tgt, INDEGREE, ce, Dist("const", 0.05), Dist("normal", 0.5, 0.25), 0))
        spec.conns.append(Connection(1, tgt, INDEGREE, ci, Dist("const", 0.35), Dist("normal", 0.5, 0.25), 1))
    return spec


def mixed_net(seed: int = 1, weight_dtype: str = "fp32") -> NetSpec:
    """LIF, AdEx (exponential conductances) and AdEx (alpha conductances)
    populations in one network, connected in a loop with an inhibitory
    pathway: L -> E -> A -> L and L -| A."""
    lif = LifParams(V_init_mean=-65.0, V_init_sd=5.0, poisson=Poisson(n_inputs=1000.0, rate_hz=8.5, weight=87.8))
    ex = AeifParams(V_init_sd=3.0, poisson=Poisson(n_inputs=1.0, rate_hz=20000.0, weight=2.5, receptor=0))
    al = AeifParams(V_reset=-60.0, tau_ex=1.0, tau_in=1.0, V_init_sd=3.0,
                    poisson=Poisson(n_inputs=1.0, rate_hz=20000.0, weight=0.3, receptor=0))
    spec = NetSpec(name="mixed_net", seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("L", LIF, 400, lif), Population("E", AEIF, 300, ex), Population("A", AEIF_ALPHA, 300, al)]
    spec.conns = [
        Connection(0, 1, INDEGREE, 50, Dist("const", 6.0), Dist("const", 1.0), 0),
        Connection(1, 2, INDEGREE, 50, Dist("const", 0.5), Dist("uniform", 0.5, 1.5), 0),
        Connection(2, 0, INDEGREE, 40, Dist("const", 60.0), Dist("const", 2.0)),
        Connection(0, 2, INDEGREE, 30, Dist("const", 1.0), Dist("const", 0.8), 1),
    ]
    return spec


def beta_net(seed: int = 1, weight_dtype: str = "fp32", w_ex: float = 1.0, w_slow: float = 0.1,
             w_in: float = 2.0, drive: float = 0.4) -> NetSpec:
    """Multisynapse AdEx neurons with beta-function conductances (Sec. 2.1):
    a 3-port population (fast excitatory, slow excitatory, inhibitory), a
    4-port population (the same three plus a second inhibitory port whose
    rise and decay times are equal) and a 1-port population, each driven by
    Poisson input on port 0 and connected across all ports."""
    fast, slow, inh, inh2 = (0.0, 0.2, 2.0), (0.0, 1.0, 8.0), (-85.0, 0.5, 5.0), (-75.0, 1.0, 1.0)
    def par(ports):
        return AeifParams(V_reset=-60.0, V_init_sd=3.0, ports=ports,
                          poisson=Poisson(n_inputs=1.0, rate_hz=20000.0, weight=drive, receptor=0))
    spec = NetSpec(name="beta_net", seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("B3", AEIF_BETA, 400, par([fast, slow, inh])),
                 Population("B4", AEIF_BETA, 350, par([fast, slow, inh, inh2])),
                 Population("B1", AEIF_BETA, 250, par([fast]))]
    spec.conns = [
        Connection(0, 1, INDEGREE, 40, Dist("const", w_ex), Dist("uniform", 0.5, 1.5), 0),
        Connection(0, 0, INDEGREE, 40, Dist("const", w_slow), Dist("const", 1.0), 1),
        Connection(1, 1, INDEGREE, 30, Dist("const", w_slow), Dist("const", 1.2), 1),
        Connection(1, 0, INDEGREE, 30, Dist("const", w_in), Dist("const", 0.8), 2),
        Connection(1, 1, INDEGREE, 20, Dist("const", w_in), Dist("const", 0.6), 2),
        Connection(2, 1, INDEGREE, 25, Dist("const", w_in), Dist("uniform", 0.5, 2.0), 3),
        Connection(0, 2, INDEGREE, 30, Dist("const", w_ex), Dist("const", 1.5), 0),
    ]
    return spec


def rules_net(seed: int = 1, weight_dtype: str = "fp32") -> NetSpec:
    """A small LIF network wired with the rules beyond fixed in-degree / total
    number (Sec. 2.1): one-to-one A -> B, fixed out-degree B -> C, all-to-all
    C -> A, all-to-all without autapses A -> A and one-to-one B -> B
    (autapses).  A is driven by Poisson input."""
    drive = LifParams(V_init_mean=-65.0, V_init_sd=4.0, poisson=Poisson(n_inputs=1000.0, rate_hz=9.0, weight=87.8))
    quiet = LifParams(V_init_mean=-65.0, V_init_sd=4.0, poisson=Poisson(n_inputs=1000.0, rate_hz=7.0, weight=87.8))
    spec = NetSpec(name="rules_net", seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("A", LIF, 300, drive), Population("B", LIF, 300, quiet), Population("C", LIF, 200, quiet)]
    spec.conns = [
        Connection(0, 1, ONE_TO_ONE, 0, Dist("const", 2500.0), Dist("const", 1.0)),
        Connection(1, 2, OUTDEGREE, 40, Dist("normal", 60.0, 6.0), Dist("normal", 1.5, 0.5)),
        Connection(2, 0, ALL_TO_ALL, 0, Dist("const", -8.0), Dist("uniform", 0.5, 2.0)),
        Connection(0, 0, ALL_TO_ALL, 0, Dist("normal", 1.0, 0.1), Dist("const", 0.8), allow_autapses=False),
        Connection(1, 1, ONE_TO_ONE, 0, Dist("const", 20.0), Dist("const", 2.0)),
    ]
    return spec


# ----------------------------------------------------------------- config 1
MC_NAMES = ["L23E", "L23I", "L4E", "L4I", "L5E", "L5I", "L6E", "L6I"]
MC_SIZES = [20683, 5834, 21915, 5479, 4850, 1065, 14395, 2948]
# connection probabilities, rows = target, columns = source
MC_PROB = [
    [.1009, .1689, .0437, .0818, .0323, 0, .0076, 0],
    [.1346, .1371, .0316, .0515, .0755, 0, .0042, 0],
    [.0077, .0059, .0497, .135, .0067, .0003, .0453, 0],
    [.0691, .0029, .0794, .1597, .0033, 0, .1057, 0],
    [.1004, .0622, .0505, .0057, .0831, .3726, .0204, 0],
    [.0548, .0269, .0257, .0022, .06, .3158, .0086, 0],
    [.0156, .0066, .0211, .0166, .0572, .0197, .0396, .2252],
    [.0364, .001, .0034, .0005, .0277, .008, .0658, .1443],
]
MC_KEXT = [1600, 1500, 2100, 1900, 2000, 1900, 2900, 2100]


def microcircuit_synapse_count(p: float, n_pre: int, n_post: int) -> int:
    """Synapses of one pathway, K = round(ln(1-p) / ln(1 - 1/(Npre*Npost))),
    evaluated literally as written in the workload definition."""
    if p <= 0.0:
        return 0
    return int(round(math.log(1.0 - p) / math.log(1.0 - 1.0 / (n_pre * n_post))))


def microcircuit(scale: float = 1.0, seed: int = 1, g: float = 4.0, bg_rate_hz: float = 8.0,
                 weight_dtype: str = "fp32", instance: int = 0, spec: Optional[NetSpec] = None,
                 keep_indegree: bool = True, V_init_mean: float = -58.0,
                 V_init_sd: float = 10.0) -> NetSpec:
    """Potjans-Diesmann microcircuit.  With scale < 1 the population sizes are
    scaled and, if keep_indegree, the per-pathway synapse count is the
    full-scale count times the scale (full-scale in-degree kept); otherwise the
    count is recomputed from the probabilities at the scaled sizes.
    Weights: Normal(87.8, 8.78) pA, inhibitory x(-g), L4E->L23E doubled.
    Delays: Normal(1.5, 0.75) ms (E), Normal(0.75, 0.375) ms (I), >= dt.
    Poisson background: K_ext inputs at bg_rate_hz, weight 87.8 pA.
    Initial V ~ Normal(V_init_mean, V_init_sd) (the paper does not state one)."""
    if spec is None:
        spec = NetSpec(name="microcircuit_%g" % scale, seeds=[seed], weight_dtype=weight_dtype)
    base = len(spec.pops)
    sizes = [max(2, int(round(n * scale))) for n in MC_SIZES]
    j = 87.8
    for k in range(8):
        par = LifParams(V_init_mean=V_init_mean, V_init_sd=V_init_sd,
                        poisson=Poisson(n_inputs=MC_KEXT[k], rate_hz=bg_rate_hz, weight=j))
        spec.pops.append(Population(MC_NAMES[k], LIF, sizes[k], par, instance=instance))
    for t in range(8):
        for s in range(8):
            p = MC_PROB[t][s]
            if p == 0:
                continue
            if keep_indegree:
                K = int(round(microcircuit_synapse_count(p, MC_SIZES[s], MC_SIZES[t]) * sizes[t] / MC_SIZES[t]))
            else:
                K = microcircuit_synapse_count(p, sizes[s], sizes[t])
            if K == 0:
                continue
            exc = (s % 2 == 0)
            w = j if exc else -g * j
            if s == 2 and t == 0:  # L4E -> L23E
                w = 2.0 * j
            wd = Dist("normal", w, abs(0.1 * w))
            dd = Dist("normal", 1.5, 0.75) if exc else Dist("normal", 0.75, 0.375)
            spec.conns.append(Connection(base + s, base + t, TOTAL, K, wd, dd))
    return spec


# ----------------------------------------------------------------- config 2
def balanced_adex(n: int = 1_000_000, indegree: int = 1000, seed: int = 1,
                  weight_dtype: str = "bf16", rk_tol: float = 1e-10,
                  poisson_rate_hz: float = 20000.0, poisson_weight: float = 0.1,
                  w_ex: float = 0.05, w_in: float = 0.35, d_lo: float = 1.0, d_hi: float = 2.0,
                  V_init_sd: float = 0.0) -> NetSpec:
    """Balanced E/I network of AdEx neurons with exponential conductances."""
    n_e = (n * 4) // 5
    n_i = n - n_e
    k_e = (indegree * 4) // 5
    k_i = indegree - k_e
    par = AeifParams(rk_tol=rk_tol, V_init_sd=V_init_sd,
                     poisson=Poisson(n_inputs=1.0, rate_hz=poisson_rate_hz, weight=poisson_weight, receptor=0))
    spec = NetSpec(name="balanced_adex_%d" % n, seeds=[seed], weight_dtype=weight_dtype)
    spec.pops = [Population("E", AEIF, n_e, par), Population("I", AEIF, n_i, replace(par))]
    for tgt in (0, 1):
        spec.conns.append(Connection(0, tgt, INDEGREE, k_e, Dist("const", w_ex), Dist("uniform", d_lo, d_hi), 0))
        spec.conns.append(Connection(1, tgt, INDEGREE, k_i, Dist("const", w_in), Dist("uniform", d_lo, d_hi), 1))
    return spec


# ----------------------------------------------------------------- config 3
def batched_microcircuits(n_instances: int = 64, seed: int = 3, scale_lo: float = 0.05,
                          scale_hi: float = 0.5, weight_dtype: str = "fp32",
                          first_instance_seed: int = 1000) -> NetSpec:
    """Independent microcircuit instances of random scale, inhibitory factor g
    and background rate, batched into one handle (full-scale in-degree kept)."""
    rng = np.random.Generator(np.random.Philox(seed))
    scales = rng.uniform(scale_lo, scale_hi, n_instances)
    gs = rng.uniform(3.0, 6.0, n_instances)
    rates = rng.uniform(6.0, 10.0, n_instances)
    spec = NetSpec(name="batched_microcircuits_%d" % n_instances, seeds=[], weight_dtype=weight_dtype)
    for i in range(n_instances):
        spec.seeds.append(first_instance_seed + i)
        microcircuit(scale=float(scales[i]), g=float(gs[i]), bg_rate_hz=float(rates[i]), instance=i,
                     spec=spec, weight_dtype=weight_dtype)
    return spec


# ----------------------------------------------------------------- config 4
@dataclass
class Request:
    arrival_s: float
    n: int
    indegree: int
    bio_time_ms: float
    seed: int


def served_requests(rate_per_s: float = 20.0, duration_s: float = 60.0, seed: int = 4,
                    n_lo: int = 10_000, n_hi: int = 200_000, k_lo: int = 100, k_hi: int = 1000,
                    t_lo_ms: float = 100.0, t_hi_ms: float = 2000.0) -> List[Request]:
    """Poisson arrival stream of balanced LIF network requests."""
    rng = np.random.Generator(np.random.Philox(seed))
    out: List[Request] = []
    t = 0.0
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        n = int(rng.integers(n_lo, n_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        T = float(rng.uniform(t_lo_ms, t_hi_ms))
        out.append(Request(arrival_s=t, n=n, indegree=k, bio_time_ms=round(T, 1), seed=10_000 + i))
        i += 1
    return out


def request_net(req: Request, spec: Optional[NetSpec] = None, instance: int = 0) -> NetSpec:
    """The balanced LIF network of one served request (config-0 neurons, weights
    and drive) as instance `instance` of `spec`."""
    one = balanced_lif(n=req.n, indegree=req.indegree, seed=req.seed)
    if spec is None:
        return one
    base = len(spec.pops)
    for p in one.pops:
        spec.pops.append(replace(p, instance=instance))
    for c in one.conns:
        spec.conns.append(replace(c, src=c.src + base, tgt=c.tgt + base))
    spec.seeds.append(req.seed)
    return spec


def instance_spec(spec: NetSpec, instance: int) -> NetSpec:
    """The populations and connections of one instance of a batched spec, as a
    standalone network with that instance's seed (same random streams)."""
    pops = spec.instance_pops(instance)
    remap = {p: i for i, p in enumerate(pops)}
    one = NetSpec(name="%s_instance%d" % (spec.name, instance), dt=spec.dt, seeds=[spec.seeds[instance]],
                  weight_dtype=spec.weight_dtype)
    one.pops = [replace(spec.pops[p], instance=0) for p in pops]
    one.conns = [replace(c, src=remap[c.src], tgt=remap[c.tgt]) for c in spec.conns if c.src in remap]
    return one
