"""Benchmark: full-scale cortical microcircuit on one GB300 (real-time factor
and synaptic events/s), printed as one JSON line.

A bench step is one second of biological time (10,000 simulation steps of
dt = 0.1 ms) of the 8-population microcircuit (77,169 LIF neurons,
298,880,968 synapses, Poisson background), run through the C ABI
(ngb_simulate): per simulation step the LIF update (Poisson drive, exact
integration, threshold/reset, spike compaction) and the spike delivery into
the targets' input ring, in the step loop the autotuner picks (the
target-owned persistent kernel on this network).  The network is built on the
device before the timed region.  The CSR (2.4 GB) is larger than L2 and is
streamed per spike; the state and ring (~21 MB) stay resident by design.

The same line carries, under "variants", the other configurations measured
once per run: BF16 weights, 64 batched microcircuit instances against each
instance alone (both autotuned), the served request stream (60 s of Poisson
arrivals) with p50/p99 latency against each request alone, and the
1e6-neuron AdEx network's real-time factor.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C++, one core) on the same
workload: it builds the same network and simulates a bounded sample of
simulation steps per bench step.  Under torchrun (N > 1) every rank runs an
independent replica with its own seed (the path has no exchange step), and
value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "real-time factor & synaptic events/s; batched/served vs plain at stated tol"
UNIT = "synaptic events/s"
DELIVERY = {1: "ring", 2: "spike_buffer"}
LOOPS = {0: "graph", 1: "persistent", 2: "fused", 3: "pipelined", 4: "persistent_pipelined",
         5: "pipelined_one_kernel", 6: "target_owned", 7: "graph_tiled"}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean of two launches) from one ncu
# capture of the full-size microcircuit with FP32 weights in this configuration (delivery scheme, step loop);
# a kernel or configuration without a capture reports null
NCU_TRAFFIC = {("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "graph", "k_update_lif"): 2483840,
               ("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "graph", "k_deliver"): 3033728,
               ("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "pipelined", "k_update_lif"): 3171200,
               ("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "pipelined", "k_deliver"): 3112960,
               ("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "pipelined_one_kernel", "k_step_pipe"):
                   6284672,
               # one launch = one bench step (10,000 simulation steps): the reads of one 1,000-step launch
               # after 2,000 steps, scaled by the steps, plus the launch's copy-out of ring and state (writes)
               ("potjans_diesmann_microcircuit_full_scale", "fp32", "ring", "target_owned", "k_owned"): 12764709120}
SIM_STEPS_PER_BENCH_STEP = 10_000  # 1 s of biological time at dt = 0.1 ms
# AdEx update (exponential conductances): FP32 and FP64 operations per Runge-Kutta attempt, counted by ncu
# (FADD + FMUL + 2 FFMA; DADD + DMUL + 2 DFMA) over one launch on the 2e5-neuron network of the same recipe,
# 2.0 attempts per neuron and step: 1.85e8 FP32 and 1.0e6 FP64 operations for 4e5 attempts
ADEX_FP32_FLOPS_PER_ATTEMPT = 462.5
ADEX_FP64_FLOPS_PER_ATTEMPT = 2.5
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x (multiply + add) x maximum SM clock


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--weights", choices=["fp32", "bf16", "fp16"], default="fp32")
    ap.add_argument("--sim-steps", type=int, default=SIM_STEPS_PER_BENCH_STEP,
                    help="simulation steps per bench step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=2000,
                    help="oracle simulation steps timed for the CPU baseline")
    ap.add_argument("--profile-steps", type=int, default=2000)
    ap.add_argument("--no-variant", action="store_true", help="skip the BF16-weight variant")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched, served and AdEx measurements of the default line")
    ap.add_argument("--delivery", choices=["auto", "ring", "spike_buffer"], default="auto",
                    help="spike delivery scheme (auto: chosen at finalisation, and by the autotuner at step 0)")
    ap.add_argument("--mode", choices=["auto", "graph", "persistent", "fused", "pipelined", "persistent_pipelined",
                                       "pipelined_one_kernel", "target_owned", "tiled"],
                    default="auto",
                    help="step loop: autotuned (default), per-step kernels in CUDA graphs, the persistent kernel, "
                         "the fused update + delivery kernels, the pipelined loop (delivery beside the next "
                         "step's update, two-stream CUDA graphs), the pipelined persistent kernel (one grid "
                         "barrier per step), the one-kernel pipelined loop, or the target-owned persistent "
                         "kernel (rings in shared memory, spikes exchanged through mailboxes)")
    ap.add_argument("--paper-n", type=str, default="1000000",
                    help="neurons of the paper's balanced network (comma-separated for a sweep)")
    ap.add_argument("--paper-ce", type=str, default="800",
                    help="excitatory in-degree(s) of the paper's balanced network (comma-separated for a sweep)")
    ap.add_argument("--workload", choices=["microcircuit", "small", "batched", "adex", "paper", "serve", "request",
                                           "precision", "validate", "stdp"],
                    default="microcircuit",
                    help="microcircuit: the benchmark line; batched: 64 microcircuit instances vs the plain path; "
                         "adex: the 1e6-neuron AdEx network; serve: the served request stream")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--req-n", type=int, default=200_000, help="neurons of the single-request workload")
    ap.add_argument("--req-k", type=int, default=1000, help="in-degree of the single-request workload")
    ap.add_argument("--adex-n", type=int, default=1_000_000, help="neurons of the AdEx workload")
    ap.add_argument("--adex-ctl32", action="store_true", help="AdEx step-size control in FP32")
    ap.add_argument("--stdp-n", type=int, default=100_000, help="neurons of the STDP workload (in-degree 1000)")
    ap.add_argument("--serve-duration", type=float, default=60.0)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="microcircuit scale (population sizes and per-pathway counts); 1.0 is the benchmark")
    return ap.parse_args()


def reduce_over_ranks(pg, seconds: float, events: float, device: str = "cuda"):
    """Whole-job figures over independent replicas (one network per rank, no
    collective on the data path): the slowest rank's time and the sum of the
    ranks' synaptic events.  pg is torch.distributed (or None for one rank)."""
    if pg is None:
        return seconds, events
    import torch
    t = torch.tensor([seconds, float(events)], dtype=torch.float64, device=device)
    tmax = t.clone()
    pg.all_reduce(tmax, op=pg.ReduceOp.MAX)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_index, "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.2)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _spec(weights: str, seed: int, scale: float = 1.0):
    from paper_2007_14236_gb300 import workloads as W
    return W.microcircuit(scale=scale, seed=seed, weight_dtype=weights)


def _cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return "%s %s" % (platform.machine(), model)


def cpu_baseline(weights: str, sample_steps: int, seed: int = 1):
    """The oracle (one core) on the full-scale microcircuit: build (untimed), a
    short untimed warm-up past the onset transient, then `sample_steps` timed
    simulation steps; events/s of that sample."""
    import oracle
    spec = _spec(weights, seed)
    t0 = time.perf_counter()
    net = oracle.OracleNet(spec)
    net.finalize()
    build_s = time.perf_counter() - t0
    net.simulate(500)
    e0 = net.events
    t1 = time.perf_counter()
    net.simulate(sample_steps)
    dt_s = time.perf_counter() - t1
    ev = net.events - e0
    bio_s = sample_steps * spec.dt * 1e-3
    return {"value": ev / dt_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "full-scale microcircuit, %d simulation steps (%.0f ms biological) after a 500-step "
                      "warm-up; single-threaded C++ oracle on %s; build %.1f s untimed"
                      % (sample_steps, bio_s * 1e3, _cpu_info(), build_s),
            "real_time_factor": dt_s / bio_s}


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    spec = _spec(a.weights, 1)
    net = oracle.OracleNet(spec)
    net.finalize()
    per_step = 100  # simulation steps (10 ms biological) per bench step
    net.simulate(500)
    for _ in range(a.warmup):
        net.simulate(per_step)
    e0 = net.events
    t0 = time.perf_counter()
    for _ in range(a.steps):
        net.simulate(per_step)
    wall = time.perf_counter() - t0
    ev = net.events - e0
    bio_s = a.steps * per_step * spec.dt * 1e-3
    value = ev / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": wall * 1e3 / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "potjans_diesmann_microcircuit_full_scale", "neurons": 77169,
                       "synapses": 298880968, "dt_ms": 0.1, "bio_ms_per_step": per_step * 0.1,
                       "weights": a.weights},
            "real_time_factor": wall / bio_s,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "full-scale microcircuit, %d x %d simulation steps after a 500-step "
                                       "warm-up, single-threaded C++ oracle on %s"
                                       % (a.steps, per_step, _cpu_info())},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batched_variant(n_instances: int, sim_steps: int, weights: str = "fp32", delivery: str = "auto",
                    mode: str = "auto", plain_sample: int = 8):
    """Config 3: independent microcircuit instances of random scale advanced in
    the same kernels, against the plain path (a sample of the instances, each
    alone in its own handle).  Both sides are autotuned before timing (the
    tuning is not timed) and run the same simulation steps after a 1,000-step
    warm-up; events/s of each."""
    import numpy as np
    from paper_2007_14236_gb300 import ngb, workloads as W
    spec = W.batched_microcircuits(n_instances=n_instances, weight_dtype=weights)
    t0 = time.perf_counter()
    sim = ngb.from_spec(spec, drain_steps=sim_steps, record_capacity=16_000_000, delivery=delivery)
    sim.finalize()
    build_s = time.perf_counter() - t0
    if mode == "auto":
        sim.autotune(500)
    st = sim.stats()
    sim.simulate(1000)
    e0 = sim.stats()["events"]
    t1 = time.perf_counter()
    sim.simulate(sim_steps)
    wall = time.perf_counter() - t1
    ev = sim.stats()["events"] - e0
    batched = ev / wall
    mode_used = LOOPS[sim.stats()["mode"]]
    sim_delivery = sim.stats()["delivery"]
    # per-kernel CUDA-event times of the per-step kernels on the batch
    ep0 = sim.stats()["events"]
    kms, nl = sim.simulate_profiled(300)
    evl = (sim.stats()["events"] - ep0) / max(1, nl[2])
    wbytes = 4 if weights == "fp32" else 2
    peak, _ = _peaks()
    us_d = 1e3 * kms[2] / max(1, nl[2])
    us_u = 1e3 * kms[0] / max(1, nl[0])
    kern = {"k_deliver": {"us_per_launch": us_d, "events_per_launch": evl,
                          "achieved_gbs": evl * (8 + wbytes) / (us_d * 1e-6) / 1e9,
                          "frac_of_measured_hbm": evl * (8 + wbytes) / (us_d * 1e-6) / 1e9 / peak},
            "k_update_lif": {"us_per_launch": us_u, "achieved_gbs": st["num_neurons"] * 32 / (us_u * 1e-6) / 1e9,
                             "frac_of_measured_hbm": st["num_neurons"] * 32 / (us_u * 1e-6) / 1e9 / peak}}
    sim.close()
    # plain path: a sample of instances, each alone, autotuned like the batch
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(n_instances, size=min(plain_sample, n_instances), replace=False).tolist())
    pw, pe = 0.0, 0
    plain_loops = []
    for i in sample:
        one = ngb.from_spec(W.instance_spec(spec, i), drain_steps=sim_steps, delivery=delivery)
        one.finalize()
        if mode == "auto":
            one.autotune(500)
        plain_loops.append(LOOPS[one.stats()["mode"]])
        one.simulate(1000)
        e1 = one.stats()["events"]
        t2 = time.perf_counter()
        one.simulate(sim_steps)
        pw += time.perf_counter() - t2
        pe += one.stats()["events"] - e1
        one.close()
    plain = pe / pw
    return {"workload": "batched_microcircuits", "instances": n_instances, "neurons": st["num_neurons"],
            "synapses": st["num_synapses"], "build_s": build_s, "step_loop": mode_used,
            "delivery": DELIVERY[sim_delivery], "bio_s": sim_steps * 1e-4,
            "batched_events_per_s": batched, "plain_events_per_s": plain, "batched_vs_plain": batched / plain,
            "plain_sample": sample, "plain_step_loops": plain_loops, "kernels": kern}


def run_batched(a):
    print(json.dumps(batched_variant(a.instances, a.sim_steps, a.weights, a.delivery, a.mode)), flush=True)
    return 0


def adex_variant(n: int, sim_steps: int, steps: int, ctl32: bool = False, delivery: str = "auto",
                 mode: str = "auto", cpu: bool = True):
    """Config 2: n AdEx neurons (exponential conductances), in-degree 1000,
    BF16 weights, adaptive RK45 with FP64 step-size control (FP32 with
    ctl32): real-time factor over `steps` x `sim_steps` simulation steps after
    a 1,000-step warm-up, and the oracle's time on a bounded sample."""
    from paper_2007_14236_gb300 import ngb, workloads as W
    spec = W.balanced_adex(n=n, indegree=1000, seed=1, weight_dtype="bf16")
    for p in spec.pops:
        p.params.rk_control_fp32 = ctl32
    t0 = time.perf_counter()
    sim = ngb.from_spec(spec, drain_steps=sim_steps, delivery=delivery)
    sim.finalize()
    build_s = time.perf_counter() - t0
    if mode == "auto":
        sim.autotune(200)
    sim.simulate(1000)
    s0 = sim.stats()
    t1 = time.perf_counter()
    for _ in range(steps):
        sim.simulate(sim_steps)
    wall = time.perf_counter() - t1
    s1 = sim.stats()
    bio = steps * sim_steps * 1e-4
    ms, nl = sim.simulate_profiled(200)
    sim.close()
    # ALU roofline of the update kernel: FP32 operations per Runge-Kutta attempt of an exponential-conductance
    # neuron (ncu: FADD + FMUL + 2 FFMA per attempt of the update kernel on this network, 2e5 neurons), against
    # the FP32 peak from the unit counts and the clock (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz = 80.5 TFLOP/s)
    attempts = (s1["rk_substeps"] - s0["rk_substeps"]) / (steps * sim_steps)
    us_upd = 1e3 * ms[1] / max(1, nl[1])
    ach = attempts * ADEX_FP32_FLOPS_PER_ATTEMPT / (us_upd * 1e-6) / 1e12
    out = {"workload": "balanced_adex_%d" % n, "neurons": s1["num_neurons"], "synapses": s1["num_synapses"],
           "roofline": {"bound": "alu", "kernel": "k_update_aeif", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "peak_source": "derived",
                        "fp32_flops_per_rk_attempt": ADEX_FP32_FLOPS_PER_ATTEMPT,
                        "fp64_flops_per_rk_attempt": ADEX_FP64_FLOPS_PER_ATTEMPT, "rk_attempts_per_step": attempts},
           "build_s": build_s, "real_time_factor": wall / bio, "bio_s": bio,
           "spikes": s1["spikes"] - s0["spikes"], "events": s1["events"] - s0["events"],
           "rate_hz": (s1["spikes"] - s0["spikes"]) / n / bio,
           "rk_substeps_per_neuron_step": (s1["rk_substeps"] - s0["rk_substeps"]) / n / (bio * 1e4),
           "us_per_launch": {"k_update_aeif": 1e3 * ms[1] / max(1, nl[1]), "k_deliver": 1e3 * ms[2] / max(1, nl[2])},
           "step_loop": LOOPS[s1["mode"]], "delivery": DELIVERY[s1["delivery"]],
           "rk_control": "fp32" if ctl32 else "fp64", "cpu_baseline": None}
    if cpu:
        # the oracle (FP32-state replica at the same tolerance) on a bounded sample: 20,000 neurons of the
        # same network for 100 steps after 20; scaled per neuron-step to the full network
        import oracle
        n_s = 20_000
        small = W.balanced_adex(n=n_s, indegree=1000, seed=1, weight_dtype="bf16")
        for p in small.pops:
            p.params.rk_control_fp32 = ctl32
        o = oracle.OracleNet(small)
        o.finalize()
        o.simulate(20)
        c0 = time.perf_counter()
        o.simulate(100)
        cw = time.perf_counter() - c0
        out["cpu_baseline"] = {
            "real_time_factor": cw / 100 / n_s * n / 1e-4, "cores": 1, "kind": "oracle",
            "sample": "%d neurons of the same network (in-degree 1000), 100 steps after 20, single-threaded "
                      "C++ oracle on %s; scaled per neuron-step to %d neurons" % (n_s, _cpu_info(), n)}
    return out


def run_adex(a):
    print(json.dumps(adex_variant(a.adex_n, a.sim_steps, a.steps, a.adex_ctl32, a.delivery, a.mode,
                                  not a.no_cpu_baseline)), flush=True)
    return 0


def run_stdp(a):
    """Balanced LIF network with plastic excitatory-to-excitatory synapses
    (nearest-neighbour STDP, multiplicative), in-degree 1000, FP32 weights:
    real-time factor, synaptic events/s, and the potentiation + plastic
    delivery kernels against the HBM roofline."""
    from paper_2007_14236_gb300 import ngb, workloads as W
    n = a.stdp_n
    spec = W.stdp_net(n=n, indegree=1000, seed=1, mu=1.0, j_ex=25.0, rate_hz=32.0)
    t0 = time.perf_counter()
    sim = ngb.from_spec(spec, drain_steps=a.sim_steps)
    sim.finalize()
    build_s = time.perf_counter() - t0
    if a.mode == "auto":
        sim.autotune(200)
    sim.simulate(1000)
    s0 = sim.stats()
    t1 = time.perf_counter()
    for _ in range(a.steps):
        sim.simulate(a.sim_steps)
    wall = time.perf_counter() - t1
    s1 = sim.stats()
    bio = a.steps * a.sim_steps * 1e-4
    ev = s1["events"] - s0["events"]
    ms, nl = sim.simulate_profiled(500)
    s2 = sim.stats()
    ev_prof = s2["events"] - s1["events"]
    sim.close()
    # algorithmic bytes of the potentiation + delivery bracket per step: a static synaptic event reads its
    # target word and weight and adds into the input (12 B); a plastic one reads its target word and its
    # 8-byte weight-and-arrival word, the target's latest spike (4 B), adds into the input and writes the
    # 8-byte word back (28 B); every potentiation reads the index word and the weight-and-arrival word and
    # writes the weight (20 B).  Plastic fraction 0.64 (E -> E of 1000 inputs); potentiations per step =
    # excitatory spikes x 800 plastic inputs (estimated from the excitatory share of spikes, 0.8).
    spk_prof = (s2["spikes"] - s1["spikes"]) / 500.0
    events_step = ev_prof / 500.0
    pot_step = 0.8 * spk_prof * 800
    bytes_step = events_step * (0.36 * 12 + 0.64 * 28) + pot_step * 20
    us_del = 1e3 * ms[2] / max(1, nl[2])
    peak, peak_src = _peaks()
    achieved = bytes_step / (us_del * 1e-6) / 1e9
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        n_s = 10_000
        small = W.stdp_net(n=n_s, indegree=1000, seed=1, mu=1.0, j_ex=25.0, rate_hz=32.0)
        o = oracle.OracleNet(small)
        o.finalize()
        o.simulate(50)
        e0 = o.events
        c0 = time.perf_counter()
        o.simulate(200)
        cw = time.perf_counter() - c0
        cpu = {"value": (o.events - e0) / cw, "unit": "synaptic events/s", "cores": 1, "kind": "oracle",
               "sample": "%d-neuron network of the same recipe, 200 steps after 50, single-threaded C++ oracle "
                         "on %s" % (n_s, _cpu_info())}
    print(json.dumps({"workload": "stdp_balanced_lif_%d" % n, "neurons": s1["num_neurons"],
                      "synapses": s1["num_synapses"], "build_s": build_s, "real_time_factor": wall / bio,
                      "synaptic_events_per_s": ev / wall, "rate_hz": (s1["spikes"] - s0["spikes"]) / n / bio,
                      "us_per_step": {"k_update_lif": 1e3 * ms[0] / max(1, nl[0]),
                                      "k_stdp_post+k_deliver": us_del},
                      "roofline": {"bound": "hbm", "kernel": "k_stdp_post+k_deliver", "achieved": achieved,
                                   "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                                   "algorithmic_bytes_per_step": bytes_step},
                      "step_loop": LOOPS[s1["mode"]], "delivery": DELIVERY[s1["delivery"]],
                      "cpu_baseline": cpu}), flush=True)
    return 0


def run_paper(a):
    """The paper's balanced network (AdEx with alpha-function conductances,
    in-degree CE + CE/4) over sizes and in-degrees (Sec. 3.2: the size sweep
    at 1,000 synapses per neuron, Fig. 10, and the synapse sweep at 30,000
    neurons, Fig. 11): time per biological second, synaptic events/s and the
    mean rate, each point beside the oracle on a bounded sample (the same
    in-degree, 10,000 neurons, or 3,000 above 5,000 inputs per neuron; 100
    steps after 500, scaled per neuron to the point's size); the paper's
    figures on one RTX 2080 Ti (about 70 s per biological second at 1e6
    neurons x 1,000 synapses; 30.7 Hz) as context."""
    from paper_2007_14236_gb300 import ngb, workloads as W
    sizes = [int(x) for x in a.paper_n.split(",")]
    ces = [int(x) for x in str(a.paper_ce).split(",")]
    out = []
    for ce in ces:
        for n in sizes:
            n_ex = (n * 4) // 5
            spec = W.paper_balanced(n_ex=n_ex, ce=ce, seed=1, weight_dtype=a.weights, rk_control_fp32=a.adex_ctl32)
            t0 = time.perf_counter()
            sim = ngb.from_spec(spec, drain_steps=a.sim_steps, record_spikes=False, delivery=a.delivery)
            sim.finalize()
            build_s = time.perf_counter() - t0
            if a.mode == "auto":
                sim.autotune(200)
            sim.simulate(1000)  # 100 ms: past the onset transient
            s0 = sim.stats()
            t1 = time.perf_counter()
            for _ in range(a.steps):
                sim.simulate(a.sim_steps)
            wall = time.perf_counter() - t1
            s1 = sim.stats()
            ms, nl = sim.simulate_profiled(100)
            nn = s1["num_neurons"]
            bio = a.steps * a.sim_steps * spec.dt * 1e-3
            row = {"neurons": nn, "in_degree": ce + ce // 4, "synapses": s1["num_synapses"], "build_s": build_s,
                   "real_time_factor": wall / bio, "events_per_s": (s1["events"] - s0["events"]) / wall,
                   "rate_hz": (s1["spikes"] - s0["spikes"]) / nn / bio,
                   "rk_substeps_per_neuron_step": (s1["rk_substeps"] - s0["rk_substeps"]) / nn / (bio / spec.dt * 1e3),
                   "us_per_launch": {"k_update_aeif": 1e3 * ms[1] / max(1, nl[1]),
                                     "k_deliver": 1e3 * ms[2] / max(1, nl[2])},
                   "step_loop": LOOPS[s1["mode"]], "delivery": DELIVERY[s1["delivery"]]}
            sim.close()
            if not a.no_cpu_baseline:
                import oracle
                n_s = 10_000 if ce + ce // 4 <= 5000 else 3_000
                small = W.paper_balanced(n_ex=(n_s * 4) // 5, ce=ce, seed=1, weight_dtype=a.weights)
                o = oracle.OracleNet(small)
                o.finalize()
                o.simulate(500)
                e0 = o.events
                c0 = time.perf_counter()
                o.simulate(100)
                cw = time.perf_counter() - c0
                row["cpu_baseline"] = {
                    "s_per_bio_s": cw / 0.01 * nn / small.num_neurons(), "events_per_s": (o.events - e0) / cw,
                    "cores": 1, "kind": "oracle",
                    "sample": "%d neurons of the same network (same in-degree), 100 steps after 500, single-threaded "
                              "C++ oracle on %s; scaled per neuron to %d neurons" % (small.num_neurons(), _cpu_info(),
                                                                                   nn)}
            print(json.dumps(row), flush=True)
            out.append(row)
    line = {"workload": "paper_balanced_alpha", "weights": a.weights, "rk_control": "fp32" if a.adex_ctl32 else "fp64",
            "bio_s_per_point": a.steps * a.sim_steps * 1e-4, "points": out,
            "paper": {"s_per_bio_s_1e6_rtx2080ti": 70.0, "rate_hz": 30.7}}
    print(json.dumps(line), flush=True)
    return 0


def _pop_stats(ids, steps, spec, t_lo, t_hi):
    """Per-population mean rate (Hz) and mean CV of inter-spike intervals."""
    import numpy as np
    offs = np.cumsum([0] + [p.n for p in spec.pops])
    m = (steps >= t_lo) & (steps < t_hi)
    ids, steps = ids[m], steps[m]
    dur = (t_hi - t_lo) * spec.dt * 1e-3
    out = []
    for k in range(len(spec.pops)):
        sel = (ids >= offs[k]) & (ids < offs[k + 1])
        rate = np.count_nonzero(sel) / spec.pops[k].n / dur
        cvs = []
        pid, pst = ids[sel], steps[sel]
        order = np.lexsort((pst, pid))
        pid, pst = pid[order], pst[order]
        for nrn in np.unique(pid):
            isi = np.diff(pst[pid == nrn])
            if len(isi) >= 3:
                cvs.append(isi.std() / isi.mean())
        out.append((rate, float(np.mean(cvs)) if cvs else float("nan")))
    return out


def _oracle_job(job):
    """Spawned worker of the precision report: the oracle run of one network
    (spec, steps, input steps, receptors) -> spikes and the FP64 sums of the
    first input steps."""
    spec, steps, n_in, R = job
    import oracle
    o = oracle.OracleNet(spec, track_abs=n_in > 0)
    o.finalize()
    inputs = []
    for _ in range(n_in):
        for r in range(R):
            _, ab, ex = o.input(r, 0)
            inputs.append((ex, ab))
        o.simulate(1)
    o.simulate(steps - n_in)
    ids, st = o.spikes()
    return ids, st, inputs


def run_precision(a):
    """Precision report: for each network, the FP32-weight, BF16-weight and
    FP16-weight GPU runs against the oracle (FP32 weights) on the same seeds:
    the per-step synaptic input of the first 20 steps of the FP32 path against
    the oracle's FP64 sum (relative to the summed magnitudes of the
    contributing weights), and per-population rates and mean CV ISI over 2 s
    after a 0.5 s transient, for three seeds (the oracle runs in parallel
    worker processes)."""
    import multiprocessing as mp
    import numpy as np
    from paper_2007_14236_gb300 import ngb, workloads as W
    T0, T = 5000, 25000
    n_in = 20
    seeds = (1, 2, 3)
    cases = {
        "microcircuit_full_scale": lambda s, wd: W.microcircuit(scale=1.0, seed=s, weight_dtype=wd),
        "balanced_lif_1000": lambda s, wd: W.balanced_lif(n=1000, indegree=100, seed=s, weight_dtype=wd),
        "balanced_adex_20000_driven": lambda s, wd: W.balanced_adex(n=20000, indegree=1000, seed=s, weight_dtype=wd,
                                                                    poisson_weight=4.0, w_ex=2.0, w_in=4.0),
        "paper_balanced_alpha_2500": lambda s, wd: W.paper_balanced(n_ex=2000, ce=200, seed=s, weight_dtype=wd),
    }
    jobs, keys = [], []
    for name, mk in cases.items():
        for s in seeds:
            spec = mk(s, "fp32")
            R = 2 if any(p.model != W.LIF for p in spec.pops) else 1
            jobs.append((spec, T, n_in if s == seeds[0] else 0, R))
            keys.append((name, s))
    pool = mp.get_context("spawn").Pool(max(1, min(len(jobs), (os.cpu_count() or 2) - 1)))
    res = pool.map_async(_oracle_job, jobs, chunksize=1)
    gpu = {}
    for name, mk in cases.items():
        for s in seeds:
            for wd in ("fp32", "bf16", "fp16"):
                spec = mk(s, wd)
                R = 2 if any(p.model != W.LIF for p in spec.pops) else 1
                kw = dict(record_capacity=8_000_000, drain_steps=5000)
                if name.startswith("microcircuit"):
                    kw.update(steps_per_graph=100, drain_steps=10_000)
                g = ngb.from_spec(spec, **kw)
                g.finalize()
                g.autotune(500)
                gin = []
                if wd == "fp32" and s == seeds[0]:
                    for _ in range(n_in):
                        for r in range(R):
                            gin.append(g.input(r, 0).astype(np.float64))
                        g.simulate(1)
                g.simulate(T - g.stats()["steps"])
                ids, st = g.spikes()
                gpu[(name, s, wd)] = (ids, st, gin, LOOPS[g.stats()["mode"]])
                g.close()
    ora = dict(zip(keys, res.get()))
    pool.close()
    pool.join()

    def rel(x, y):
        return abs(x - y) / y if y > 0 else (0.0 if x == 0 else float("inf"))
    report = {}
    for name, mk in cases.items():
        spec = mk(seeds[0], "fp32")
        ids0, st0, oin = ora[(name, seeds[0])]
        gin = gpu[(name, seeds[0], "fp32")][2]
        err = 0.0
        for g_, (ex, ab) in zip(gin, oin):
            nz = ab > 0
            if np.any(nz):
                err = max(err, float(np.max(np.abs(g_[nz] - ex[nz]) / ab[nz])))
        row = {"input_rel_error_max_fp32": err, "seeds": list(seeds), "stats_window_s": [T0 * 1e-4, T * 1e-4],
               "step_loop": gpu[(name, seeds[0], "fp32")][3]}
        so_all = {s: _pop_stats(*ora[(name, s)][:2], spec, T0, T) for s in seeds}
        row["rates_hz_oracle_seed1"] = [round(x[0], 3) for x in so_all[seeds[0]]]
        for wd in ("fp32", "bf16", "fp16"):
            rmax, cmax = 0.0, 0.0
            for s in seeds:
                sg = _pop_stats(*gpu[(name, s, wd)][:2], spec, T0, T)
                so = so_all[s]
                rmax = max(rmax, max(rel(x[0], y[0]) for x, y in zip(sg, so)))
                cmax = max(cmax, max(abs(x[1] - y[1]) for x, y in zip(sg, so) if y[1] == y[1]))
            row["rate_rel_error_max_" + wd] = rmax
            row["cv_isi_abs_error_max_" + wd] = cmax
        report[name] = row
    print(json.dumps({"workload": "precision_report", "steps": T, "stats_window_steps": [T0, T], "cases": report}),
          flush=True)
    return 0


def run_validate(a):
    """The paper's equivalence test (Sec. 3.1) with the oracle in the
    reference simulator's role: the microcircuit at a reduced scale simulated
    with several seeds on the GPU and by the oracle; per population, the KL
    divergences of the smoothed firing-rate, CV ISI and correlation
    distributions for GPU-oracle pairs and for oracle-oracle pairs (different
    seeds in every pair)."""
    import numpy as np
    import oracle
    from paper_2007_14236_gb300 import ngb, validate as V, workloads as W
    n_seeds, T, T0 = 4, 11_000, 1_000  # 1.1 s, the first 0.1 s discarded
    gpu_stats, ora_stats = [], []
    for seed in range(1, n_seeds + 1):
        spec = W.microcircuit(scale=a.scale if a.scale != 1.0 else 0.1, seed=seed, weight_dtype=a.weights)
        bounds = np.cumsum([0] + [p.n for p in spec.pops])
        g = ngb.from_spec(spec, delivery=a.delivery, record_capacity=8_000_000, drain_steps=T)
        g.simulate(T)
        gpu_stats.append(V.population_statistics(*g.spikes(), bounds, T0, T, spec.dt))
        g.close()
        o = oracle.OracleNet(spec)
        o.finalize()
        o.simulate(T)
        ora_stats.append(V.population_statistics(*o.spikes(), bounds, T0, T, spec.dt))
    go = [V.compare(gpu_stats[i], ora_stats[(i + 1) % n_seeds]) for i in range(n_seeds)]
    oo = [V.compare(ora_stats[i], ora_stats[(i + 1) % n_seeds]) for i in range(n_seeds)]
    print(json.dumps({"workload": "validation_microcircuit", "scale": a.scale if a.scale != 1.0 else 0.1,
                      "seeds": n_seeds, "bio_s": T * 1e-4, "discarded_s": T0 * 1e-4, "populations": W.MC_NAMES,
                      "kl_gpu_vs_oracle": V.mean_std(go), "kl_oracle_vs_oracle": V.mean_std(oo)}), flush=True)
    return 0


def run_small(a):
    """Config 0: the 1,000-neuron balanced LIF network, 100 ms of biological
    time per bench step, beside the oracle on the host for the same 100 ms."""
    from paper_2007_14236_gb300 import ngb, workloads as W
    spec = W.balanced_lif(n=1000, indegree=100, seed=1)
    sim = ngb.from_spec(spec, drain_steps=1000, delivery=a.delivery)
    sim.finalize()
    if a.mode == "auto":
        sim.autotune(500)
    sim.simulate(1000)
    s0 = sim.stats()
    t1 = time.perf_counter()
    for _ in range(a.steps):
        sim.simulate(1000)
    wall = time.perf_counter() - t1
    s1 = sim.stats()
    sim.close()
    bio = a.steps * 0.1
    out = {"workload": "balanced_lif_1000", "neurons": 1000, "synapses": s1["num_synapses"],
           "real_time_factor": wall / bio, "events_per_s": (s1["events"] - s0["events"]) / wall,
           "rate_hz": (s1["spikes"] - s0["spikes"]) / 1000 / bio, "step_loop": LOOPS[s1["mode"]],
           "delivery": DELIVERY[s1["delivery"]]}
    if not a.no_cpu_baseline:
        import oracle
        o = oracle.OracleNet(spec)
        o.finalize()
        c0 = time.perf_counter()
        o.simulate(1000)
        cw = time.perf_counter() - c0
        out["cpu_baseline"] = {"real_time_factor": cw / 0.1, "events_per_s": o.events / cw, "cores": 1,
                               "kind": "oracle", "sample": "the whole 100 ms run, single-threaded C++ oracle on %s"
                                                           % _cpu_info()}
    print(json.dumps(out), flush=True)
    return 0


def run_request(a):
    """One served-request network alone (balanced LIF, config-0 neurons and
    weights) at a given size and in-degree: the high-load delivery case."""
    from paper_2007_14236_gb300 import ngb, workloads as W
    spec = W.balanced_lif(n=a.req_n, indegree=a.req_k, seed=7, weight_dtype=a.weights)
    sim = ngb.from_spec(spec, drain_steps=a.sim_steps, record_spikes=False, delivery=a.delivery)
    sim.finalize()
    if a.mode == "auto":
        sim.autotune(300)
    sim.simulate(1000)
    s0 = sim.stats()
    t1 = time.perf_counter()
    for _ in range(a.steps):
        sim.simulate(a.sim_steps)
    wall = time.perf_counter() - t1
    s1 = sim.stats()
    ep0 = s1["events"]
    kms, nl = sim.simulate_profiled(200)
    evl = (sim.stats()["events"] - ep0) / max(1, nl[2])
    peak, _ = _peaks()
    us_d = 1e3 * kms[2] / max(1, nl[2])
    bio = a.steps * a.sim_steps * 1e-4
    ev_b = 12 if a.weights == "fp32" else 10  # target index + weight + ring add per synaptic event
    n_steps = a.steps * a.sim_steps
    # the whole step of the loop that ran (update 32 B per neuron + delivery per event) over its wall time
    step_bytes = 32 * a.req_n + ev_b * (s1["events"] - s0["events"]) / n_steps
    step_gbs = step_bytes / (wall / n_steps) / 1e9
    print(json.dumps({"workload": "request_n%d_k%d" % (a.req_n, a.req_k), "synapses": s1["num_synapses"],
                      "weights": a.weights,
                      "events_per_s": (s1["events"] - s0["events"]) / wall, "real_time_factor": wall / bio,
                      "rate_hz": (s1["spikes"] - s0["spikes"]) / a.req_n / bio,
                      "us_per_step": 1e6 * wall / n_steps,
                      "step_roofline": {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_gbs,
                                        "frac_of_measured_hbm": step_gbs / peak},
                      "per_step_kernels": {"k_deliver": {"us_per_launch": us_d, "events_per_launch": evl,
                                                         "achieved_gbs": evl * ev_b / (us_d * 1e-6) / 1e9,
                                                         "frac_of_measured_hbm":
                                                             evl * ev_b / (us_d * 1e-6) / 1e9 / peak},
                                           "k_update_lif_us": 1e3 * kms[0] / max(1, nl[0])},
                      "step_loop": LOOPS[s1["mode"]],
                      "delivery": DELIVERY[s1["delivery"]]}), flush=True)
    return 0


def served_variant(duration_s: float, delivery: str = "auto", plain_sample: int = 30):
    """Config 4: the served request stream (Poisson arrivals at 20/s over
    duration_s seconds) through one serving handle, with p50/p99 completion
    latency, against the plain path: a sample of the requests, each alone in
    its own handle, (a) end to end through the library's default choices
    (build, simulate, read back) and (b) autotuned, the simulation alone timed.
    served_vs_plain divides by (b), the faster plain figure."""
    import numpy as np
    from paper_2007_14236_gb300 import ngb, serve, workloads as W
    reqs = W.served_requests(duration_s=duration_s)
    srv = serve.Server(8_000_000, 4_000_000_000, 8_000_000, ring_slots=32, delivery=delivery)
    sdelivery = DELIVERY[srv.sim.stats()["delivery"]]
    done, summary = srv.run(reqs)
    srv.close()
    summary["delivery"] = sdelivery
    rng = np.random.default_rng(0)
    sample = rng.choice(len(reqs), size=min(plain_sample, len(reqs)), replace=False)
    pw, pe, tw, te = 0.0, 0, 0.0, 0
    for i in sample:
        r = reqs[int(i)]
        w, ev, _, _ = serve.run_alone(r)
        pw += w
        pe += ev
        one = ngb.from_spec(W.request_net(r), drain_steps=1000, record_spikes=False, delivery=delivery)
        one.finalize()
        one.autotune(300)
        steps = int(round(r.bio_time_ms / 0.1))
        t0 = time.perf_counter()
        one.simulate(steps)
        tw += time.perf_counter() - t0
        te += one.stats()["events"]
        one.close()
    summary.update({"workload": "served_requests", "arrival_rate_per_s": 20.0, "window_s": duration_s,
                    "plain_e2e_events_per_s": pe / pw, "plain_tuned_events_per_s": te / tw,
                    "served_vs_plain": summary["events_per_s"] / (te / tw),
                    "served_vs_plain_e2e": summary["events_per_s"] / (pe / pw), "plain_sample": len(sample)})
    return summary


def run_serve(a):
    print(json.dumps(served_variant(a.serve_duration, a.delivery)), flush=True)
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    if a.mode in ("persistent", "fused", "pipelined", "persistent_pipelined", "pipelined_one_kernel", "target_owned",
                  "tiled"):
        os.environ["NGB_MODE"] = a.mode  # read by the library when a network is finalised
    if a.workload != "microcircuit":
        return {"small": run_small, "batched": run_batched, "adex": run_adex, "paper": run_paper,
                "serve": run_serve, "request": run_request, "precision": run_precision,
                "validate": run_validate, "stdp": run_stdp}[a.workload](a)
    ws, rank, local = _dist()
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    from paper_2007_14236_gb300 import ngb
    ngb.load()
    stream = torch.cuda.Stream()
    spec = _spec(a.weights, 1 + rank, a.scale)
    t0 = time.perf_counter()
    sim = ngb.from_spec(spec, device=local, stream=stream.cuda_stream, steps_per_graph=100,
                        drain_steps=a.sim_steps, record_capacity=4_000_000, delivery=a.delivery)
    sim.finalize()
    build_s = time.perf_counter() - t0
    tune_s = 0.0
    if a.mode == "auto":
        t1 = time.perf_counter()
        sim.autotune(1000)
        tune_s = time.perf_counter() - t1
    st0 = sim.stats()
    mode = LOOPS[st0["mode"]]

    for _ in range(a.warmup):
        sim.simulate(a.sim_steps)

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region (device clock)
    gpu_idx = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if ws > 1 else 0]
    barrier()
    sampler = ClockSampler(gpu_idx)
    ev_before = sim.stats()["events"]
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for _ in range(a.steps):
        sim.simulate(a.sim_steps)
    e_end.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e_start.elapsed_time(e_end)
    events = sim.stats()["events"] - ev_before
    ms, events = reduce_over_ranks(pg, ms, events)
    bio_s_rank = a.steps * a.sim_steps * spec.dt * 1e-3
    value = events / (ms * 1e-3)
    rtf = (ms * 1e-3) / bio_s_rank

    # ---------------------------------------------------------------- end to end (host buffers)
    barrier()
    ev_b = sim.stats()["events"]
    t_now = sim.stats()["steps"]
    d2h = 0
    h0 = time.perf_counter()
    for _ in range(a.steps):
        sim.simulate(a.sim_steps)
        ids, stp = sim.spikes(t0=t_now, t1=t_now + a.sim_steps)  # spike record read back into host buffers
        d2h += ids.size * (4 + 8)
        t_now += a.sim_steps
    barrier()
    e2e_s = time.perf_counter() - h0
    e2e_events = sim.stats()["events"] - ev_b
    e2e_s, e2e_events = reduce_over_ranks(pg, e2e_s, e2e_events)

    # ---------------------------------------------------------------- per-kernel times (CUDA events)
    ev_p0 = sim.stats()["events"]
    kms, nlaunch = sim.simulate_profiled(a.profile_steps)
    ev_p = sim.stats()["events"] - ev_p0
    N = st0["num_neurons"]
    lif_bytes = N * 32  # y, I, refractory read+write (24 B) + ring slot read and zero (8 B)
    wbytes = 4 if a.weights == "fp32" else 2
    spikes_per_step = None
    ev_per_launch = ev_p / max(1, nlaunch[2])
    deliver_bytes = ev_per_launch * (4 + wbytes + 4)
    if mode == "fused":
        # one launch per step updates the neurons and delivers their spikes; entry 2 is the step-counter tick
        kern = {
            "k_step_lif": {"launches": int(nlaunch[0]), "ms_total": float(kms[0]),
                           "us_per_launch": 1e3 * float(kms[0]) / max(1, nlaunch[0]),
                           "algorithmic_bytes_per_launch": lif_bytes + deliver_bytes,
                           "events_per_launch": ev_per_launch},
            "k_tick_add": {"launches": int(nlaunch[2]), "ms_total": float(kms[2]),
                           "us_per_launch": 1e3 * float(kms[2]) / max(1, nlaunch[2]),
                           "algorithmic_bytes_per_launch": 16},
        }
    else:
        kern = {
            "k_update_lif": {"launches": int(nlaunch[0]), "ms_total": float(kms[0]),
                             "us_per_launch": 1e3 * float(kms[0]) / max(1, nlaunch[0]),
                             "algorithmic_bytes_per_launch": lif_bytes},
            "k_deliver": {"launches": int(nlaunch[2]), "ms_total": float(kms[2]),
                          "us_per_launch": 1e3 * float(kms[2]) / max(1, nlaunch[2]),
                          "algorithmic_bytes_per_launch": deliver_bytes,
                          "events_per_launch": ev_per_launch},
        }
    peak, peak_kind = _peaks()
    if mode in ("persistent", "persistent_pipelined", "target_owned"):
        # one launch per bench step (sim_steps steps); its duration from the timed region's events
        ev_step = events / max(1, ws) / a.steps
        bytes_launch = a.sim_steps * lif_bytes + ev_step * (4 + wbytes + 4)
        us_launch = ms / a.steps * 1e3
        dom = "k_owned" if mode == "target_owned" else "k_persistent"
        kern[dom] = {"launches": a.steps, "ms_total": ms, "us_per_launch": us_launch,
                     "algorithmic_bytes_per_launch": bytes_launch, "steps_per_launch": a.sim_steps,
                     "grid": st0["launch_grid"]}
    elif mode == "pipelined_one_kernel":
        # one launch per simulation step, back to back in the stream (chained by programmatic dependent
        # launch): its average duration from the timed region's events
        ev_step = events / max(1, ws) / (a.steps * a.sim_steps)
        n_launch = a.steps * a.sim_steps
        kern["k_step_pipe"] = {"launches": n_launch, "ms_total": ms, "us_per_launch": ms * 1e3 / n_launch,
                               "algorithmic_bytes_per_launch": lif_bytes + ev_step * (4 + wbytes + 4),
                               "grid": st0["launch_grid"]}
        dom = "k_step_pipe"
    else:
        dom = max(kern, key=lambda k: kern[k]["ms_total"])
    ach = kern[dom]["algorithmic_bytes_per_launch"] / (kern[dom]["us_per_launch"] * 1e-6) / 1e9
    workload = ("potjans_diesmann_microcircuit_full_scale" if a.scale == 1.0 else
                "potjans_diesmann_microcircuit_scale_%g" % a.scale)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind,
                "traffic": NCU_TRAFFIC.get((workload, a.weights, DELIVERY[st0["delivery"]], mode, dom))}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Philox network and Poisson drive)",
        "config": {"workload": "potjans_diesmann_microcircuit_full_scale" if a.scale == 1.0 else
                   "potjans_diesmann_microcircuit_scale_%g" % a.scale, "neurons": N,
                   "synapses": st0["num_synapses"], "dt_ms": spec.dt, "bio_s_per_step": a.sim_steps * spec.dt * 1e-3,
                   "weights": a.weights, "parallelism": "replicas" if ws > 1 else "single",
                   "step_loop": mode, "launch_grid": st0["launch_grid"], "delivery": DELIVERY[st0["delivery"]],
                   "l2": "CSR (%.1f GB) larger than L2 and streamed per spike; state and %s stay resident"
                         % (st0["num_synapses"] * (4 + wbytes) / 1e9,
                            "ring" if st0["delivery"] == 1 else "input slot and pending spikes")},
        "real_time_factor": rtf,
        "build_s": build_s,
        "autotune_s": tune_s,
        "gpu_launches": int(a.steps if mode in ("persistent", "persistent_pipelined", "target_owned") else
                            a.steps * (a.sim_steps + (a.sim_steps + 99) // 100) if mode == "fused" else
                            a.steps * (2 * a.sim_steps + (a.sim_steps + 99) // 100) if mode == "pipelined" else
                            a.steps * (a.sim_steps + 2 * ((a.sim_steps + 99) // 100)) if mode == "pipelined_one_kernel"
                            else
                            a.steps * a.sim_steps * 2),
        "e2e": {"value": e2e_events / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(d2h / a.steps), "real_time_factor": e2e_s / bio_s_rank},
        "roofline": roofline,
        "kernels": kern,
        "clocks": clocks,
    }
    sim.close()
    torch.cuda.synchronize()

    if rank == 0 and ws == 1 and not a.no_variant and a.weights == "fp32":
        v = ngb.from_spec(_spec("bf16", 1), device=local, stream=stream.cuda_stream, steps_per_graph=100,
                          drain_steps=10_000, record_capacity=4_000_000, delivery=a.delivery)
        v.finalize()
        if a.mode == "auto":
            v.autotune(1000)
        v.simulate(a.sim_steps)
        e0 = v.stats()["events"]
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(max(1, a.steps // 2)):
            v.simulate(a.sim_steps)
        s1.record(stream)
        torch.cuda.synchronize()
        vms = s0.elapsed_time(s1)
        vb = max(1, a.steps // 2) * a.sim_steps * spec.dt * 1e-3
        line["variants"] = {"bf16_weights": {"value": (v.stats()["events"] - e0) / (vms * 1e-3),
                                             "real_time_factor": vms * 1e-3 / vb,
                                             "step_loop": LOOPS[v.stats()["mode"]]}}
        v.close()

    if rank == 0 and ws == 1 and not a.no_variants:
        # the other configurations, each measured once per run: batched and served throughput against the
        # plain path, and the AdEx network's real-time factor
        line.setdefault("variants", {})
        b = batched_variant(64, 5000, "fp32", a.delivery, a.mode)
        line["variants"]["batched_64_microcircuits"] = {
            k: b[k] for k in ("batched_events_per_s", "plain_events_per_s", "batched_vs_plain", "step_loop",
                              "delivery", "neurons", "synapses", "bio_s", "plain_step_loops", "kernels")}
        v = served_variant(a.serve_duration, a.delivery)
        line["variants"]["served_requests"] = {
            k: v[k] for k in ("requests", "window_s", "events_per_s", "plain_tuned_events_per_s",
                              "plain_e2e_events_per_s", "served_vs_plain", "served_vs_plain_e2e", "p50_latency_s",
                              "p99_latency_s", "max_active", "wall_s", "delivery")}
        x = adex_variant(1_000_000, 10_000, 1, False, a.delivery, a.mode, cpu=not a.no_cpu_baseline)
        line["variants"]["adex_1e6_config2"] = {
            k: x[k] for k in ("real_time_factor", "rate_hz", "rk_substeps_per_neuron_step", "us_per_launch",
                              "step_loop", "delivery", "rk_control", "cpu_baseline", "neurons", "synapses",
                              "roofline")}

    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a.weights, a.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
