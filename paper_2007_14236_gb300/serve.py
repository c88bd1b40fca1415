"""Continuous-batching request server over the C ABI.

A request is an independent network to simulate for a given biological time
(the served workload: balanced LIF networks of random size and in-degree).
The server keeps one serving handle (ngb_reserve) whose pools hold every
admitted network's state and connectivity on the device; all active networks
advance together in the same kernels.  At every chunk boundary it

  * retires the networks whose biological time is reached (their spikes are
    read back first) -- their pool ranges become free;
  * admits waiting requests in arrival order while their footprint (neurons,
    synapses, delay groups) fits the free pool capacity: the network is built
    on the device (ngb_commit_instance) and starts at the current step;
  * advances all active networks to the next completion or chunk end.

Arrival times are honoured either in real time (the loop sleeps until the
next arrival when idle) or in trace time (idle gaps are skipped; the clock
otherwise advances with the measured wall time), which keeps the queueing
behaviour without waiting through idle periods.  Latency = completion time -
arrival time.  Because every network draws its random numbers from its own key
with network-local ids and steps, its result does not depend on what else is
served with it (bit-identical in deterministic mode).
"""
from __future__ import annotations

import argparse
import json
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import ngb as _ngb
from . import workloads as W


@dataclass
class Done:
    req: W.Request
    admit_s: float
    done_s: float
    latency_s: float
    spikes: int
    ids: Optional[np.ndarray] = None
    steps: Optional[np.ndarray] = None


def footprint(spec: W.NetSpec) -> Dict[str, int]:
    """Pool demand of a network: neurons, synapses and an upper bound of its
    (source, delay) groups."""
    n = spec.num_neurons()
    k = spec.num_synapses()
    groups = 0
    for p_i, p in enumerate(spec.pops):
        out = [c for c in spec.conns if c.src == p_i]
        if not out:
            continue
        per_source = 0
        for c in out:
            if c.delay.kind == "const":
                per_source += 1
            else:
                hi = c.delay.p0 + 6 * c.delay.p1 if c.delay.kind == "normal" else c.delay.p1
                per_source += int(hi / spec.dt) + 2
        groups += p.n * per_source
    return {"neurons": n, "synapses": k, "groups": min(groups, k)}


class Server:
    def __init__(self, max_neurons: int, max_synapses: int, max_groups: int, ring_slots: int = 32,
                 chunk_steps: int = 1000, deterministic: bool = False, keep_spikes: bool = False,
                 weight_dtype: str = "fp32", device: int = 0, delivery: str = "auto"):
        # spikes are recorded only when the caller keeps them; the counters count them either way
        self.sim = _ngb.Simulator(dt_ms=0.1, seed=0, weight_dtype=weight_dtype, device=device,
                                  deterministic=deterministic, record_spikes=keep_spikes, drain_steps=chunk_steps,
                                  record_capacity=max(1 << 22, max_neurons * chunk_steps // 20), delivery=delivery)
        self.sim.reserve(max_neurons, max_synapses, max_groups, ring_slots, 1)
        self.sim.finalize()
        self.cap = {"neurons": max_neurons, "synapses": max_synapses, "groups": max_groups}
        self.used = {"neurons": 0, "synapses": 0, "groups": 0}
        self.chunk = chunk_steps
        self.keep = keep_spikes
        self.step = 0

    def _fits(self, fp):
        return all(self.used[k] + fp[k] <= self.cap[k] for k in fp)

    def run(self, requests: List[W.Request], realtime: bool = False, specs: Optional[List[W.NetSpec]] = None):
        """Serve the requests; returns (completed list, summary dict)."""
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival_s)
        queue = deque(order)
        waiting: deque = deque()
        active: Dict[int, dict] = {}
        built: Dict[int, tuple] = {}  # requests added as pending instances, waiting for room
        done: List[Done] = []
        ev0 = self.sim.stats()["events"]
        host = {"build_s": 0.0, "simulate_s": 0.0, "retire_s": 0.0}  # wall time by activity
        wall0 = time.perf_counter()
        clock = 0.0  # trace time, seconds since the first arrival window opened
        last_wall = wall0
        max_active = 0

        def now():
            nonlocal clock, last_wall
            w = time.perf_counter()
            clock += w - last_wall
            last_wall = w
            return clock

        while queue or waiting or active:
            t = now()
            while queue and requests[queue[0]].arrival_s <= t:
                waiting.append(queue.popleft())
            # admit in arrival order while the pools have room
            while waiting:
                i = waiting[0]
                spec = specs[i] if specs else W.request_net(requests[i])
                fp = footprint(spec)
                if not self._fits(fp):
                    break
                tb = time.perf_counter()
                if i not in built:
                    built[i] = self.sim.add_spec_instance(spec)
                inst, pops = built[i]
                try:
                    self.sim.commit(inst)
                except _ngb.NgbError as e:
                    if e.code == -3:  # pool fragmentation: retry after the next retirements
                        break
                    raise
                finally:
                    host["build_s"] += time.perf_counter() - tb
                del built[i]
                waiting.popleft()
                for k in fp:
                    self.used[k] += fp[k]
                t0, _ = self.sim.instance_info(inst)
                steps = int(round(requests[i].bio_time_ms / 0.1))
                active[inst] = {"i": i, "pops": pops, "t0": t0, "end": t0 + steps, "fp": fp, "admit": now()}
            max_active = max(max_active, len(active))
            if not active:
                if queue:
                    nxt = requests[queue[0]].arrival_s
                    if realtime:
                        time.sleep(max(0.0, nxt - now()))
                    else:
                        clock = max(clock, nxt)
                continue
            adv = min(self.chunk, min(a["end"] for a in active.values()) - self.step)
            ts = time.perf_counter()
            self.sim.simulate(adv)
            host["simulate_s"] += time.perf_counter() - ts
            self.step += adv
            tr = time.perf_counter()
            for inst in [k for k, a in active.items() if a["end"] <= self.step]:
                a = active.pop(inst)
                ids_all, st_all = [], []
                n_spk = 0
                local = 0  # network-local id of the population's first neuron
                for p in a["pops"]:
                    off, n = self.sim.population_range(p)
                    if self.keep:
                        ids, st = self.sim.spikes(pop=p, t0=a["t0"], t1=a["end"])
                        n_spk += len(ids)
                        ids_all.append(ids + local)
                        st_all.append(st - a["t0"])
                    local += n
                self.sim.retire(inst)
                for k in a["fp"]:
                    self.used[k] -= a["fp"][k]
                tdone = now()
                req = requests[a["i"]]
                d = Done(req, a["admit"], tdone, tdone - req.arrival_s, n_spk)
                if self.keep:
                    ids = np.concatenate(ids_all) if ids_all else np.zeros(0, np.int64)
                    st = np.concatenate(st_all) if st_all else np.zeros(0, np.int64)
                    o = np.lexsort((ids, st))
                    d.ids, d.steps = ids[o], st[o]
                done.append(d)
            host["retire_s"] += time.perf_counter() - tr
        wall = time.perf_counter() - wall0
        events = self.sim.stats()["events"] - ev0
        lat = np.array([d.latency_s for d in done]) if done else np.zeros(1)
        summary = {"requests": len(done), "wall_s": wall, "trace_s": clock, "events": int(events),
                   "events_per_s": events / wall if wall > 0 else 0.0,
                   "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                   "max_active": max_active, "realtime": realtime, "steps": self.step}
        summary.update(host)
        return done, summary

    def close(self):
        self.sim.close()


def run_alone(req: W.Request, spec: Optional[W.NetSpec] = None, deterministic: bool = False,
              keep_spikes: bool = False):
    """The plain path: the request's network alone in its own handle (build,
    simulate, read spikes).  Returns (wall seconds, events, ids, steps)."""
    spec = spec or W.request_net(req)
    t0 = time.perf_counter()
    sim = _ngb.from_spec(spec, deterministic=deterministic, drain_steps=1000, record_spikes=keep_spikes,
                         record_capacity=max(1 << 22, spec.num_neurons() * 50))
    steps = int(round(req.bio_time_ms / 0.1))
    sim.simulate(steps)
    ids, st = sim.spikes(t0=0, t1=steps)
    wall = time.perf_counter() - t0
    ev = sim.stats()["events"]
    sim.close()
    return wall, ev, (ids if keep_spikes else None), (st if keep_spikes else None)


def main():
    ap = argparse.ArgumentParser(description="served request stream (Poisson arrivals of balanced LIF networks)")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--realtime", action="store_true")
    ap.add_argument("--max-neurons", type=int, default=8_000_000)
    ap.add_argument("--max-synapses", type=int, default=4_000_000_000)
    ap.add_argument("--alone-sample", type=int, default=40, help="requests also run alone (plain path)")
    a = ap.parse_args()
    reqs = W.served_requests(rate_per_s=a.rate, duration_s=a.duration, seed=a.seed)
    srv = Server(a.max_neurons, a.max_synapses, a.max_neurons, ring_slots=32)
    done, summary = srv.run(reqs, realtime=a.realtime)
    srv.close()
    rng = np.random.default_rng(0)
    sample = rng.choice(len(reqs), size=min(a.alone_sample, len(reqs)), replace=False)
    alone_wall, alone_ev = 0.0, 0
    for i in sample:
        w, ev, _, _ = run_alone(reqs[int(i)])
        alone_wall += w
        alone_ev += ev
    summary["plain_events_per_s"] = alone_ev / alone_wall if alone_wall > 0 else 0.0
    summary["served_vs_plain"] = summary["events_per_s"] / summary["plain_events_per_s"] if alone_wall else None
    summary["plain_sample"] = len(sample)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
