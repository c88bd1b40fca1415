"""Python binding of the C ABI in include/ngb.h (argument marshalling only).

Every step of the simulation runs in the CUDA library libngb.so; this module
only converts Python values to the C structures and back.  Importing it loads
the library and raises if it has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Tuple

import numpy as np

from . import build as _build
from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "STATE", -3: "OOM", -4: "CUDA", -5: "TIMEOUT", -6: "OVERFLOW"}
WEIGHT_DTYPES = {"fp32": 0, "bf16": 1, "fp16": 2}
MODELS = {W.LIF: 0, W.AEIF: 1, W.AEIF_ALPHA: 2, W.AEIF_BETA: 3}
RULES = {W.INDEGREE: 0, W.TOTAL: 1, W.OUTDEGREE: 2, W.ONE_TO_ONE: 3, W.ALL_TO_ALL: 4}
DISTS = {"const": 0, "normal": 1, "uniform": 2}
DELIVERY = {"auto": 0, "ring": 1, "spike_buffer": 2}
VARS = {"V_m": 0, "I_syn": 1, "w": 1, "g_ex": 2, "g_in": 3, "refractory": 4, "h": 5, "dg_ex": 6, "dg_in": 7,
        "g_0": 2, "g_1": 3, "g_2": 8, "g_3": 9, "x_0": 6, "x_1": 7, "x_2": 10, "x_3": 11}


class SimConfig(C.Structure):
    _fields_ = [("dt_ms", C.c_double), ("seed", C.c_uint64), ("weight_dtype", C.c_int32), ("device", C.c_int32),
                ("stream", C.c_void_p), ("deterministic", C.c_int32), ("record_spikes", C.c_int32),
                ("record_capacity", C.c_int64), ("steps_per_graph", C.c_int32), ("drain_steps", C.c_int32),
                ("delivery", C.c_int32), ("pad_", C.c_int32)]


class PoissonDrive(C.Structure):
    _fields_ = [("n_inputs", C.c_double), ("rate_hz", C.c_double), ("weight", C.c_double),
                ("receptor", C.c_int32), ("pad_", C.c_int32)]


class LifParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("tau_m_ms", "C_m_pF", "E_L_mV", "V_reset_mV", "V_th_mV", "t_ref_ms",
                                          "tau_syn_ms", "I_e_pA", "V_init_mean_mV", "V_init_sd_mV")] + \
               [("poisson", PoissonDrive)]


class AeifParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("C_m_pF", "g_L_nS", "E_L_mV", "V_T_mV", "Delta_T_mV", "a_nS", "b_pA",
                                          "tau_w_ms", "V_peak_mV", "V_reset_mV", "E_ex_mV", "E_in_mV",
                                          "tau_ex_ms", "tau_in_ms", "I_e_pA", "V_init_mean_mV",
                                          "V_init_sd_mV", "w_init_pA", "rk_tol", "rk_h_min_ms",
                                          "rk_h_init_ms")] + \
               [("rk_max_substeps", C.c_int64), ("rk_control_fp32", C.c_int32), ("pad_", C.c_int32),
                ("poisson", PoissonDrive), ("n_ports", C.c_int32), ("pad2_", C.c_int32),
                ("E_rev_mV", C.c_double * 4), ("tau_rise_ms", C.c_double * 4), ("tau_decay_ms", C.c_double * 4)]


class StdpParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("tau_plus_ms", "tau_minus_ms", "lambda_", "alpha", "mu_plus", "mu_minus",
                                          "W_max")]


class ConnSpec(C.Structure):
    _fields_ = [("rule", C.c_int32), ("allow_autapses", C.c_int32), ("K", C.c_int64)]


class DistSpec(C.Structure):
    _fields_ = [("dist", C.c_int32), ("pad_", C.c_int32), ("p0", C.c_double), ("p1", C.c_double)]


class SynSpec(C.Structure):
    _fields_ = [("weight", DistSpec), ("delay_ms", DistSpec), ("receptor", C.c_int32), ("pad_", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("steps", "spikes", "events", "rk_substeps", "num_neurons", "num_synapses",
                                         "num_groups", "ring_slots", "max_delay_steps", "device_bytes", "mode",
                                         "launch_grid", "delivery", "hot_steps")]


_lib = None

# every symbol the header declares (checked by the tests)
EXPORTS = ["ngb_create", "ngb_destroy", "ngb_last_error", "ngb_add_instance", "ngb_add_population",
           "ngb_add_population_in", "ngb_connect", "ngb_connect_stdp", "ngb_finalize", "ngb_simulate", "ngb_simulate_profiled",
           "ngb_get_spikes", "ngb_get_stats", "ngb_population_range", "ngb_get_state", "ngb_get_input",
           "ngb_get_src_ptr", "ngb_get_synapses", "ngb_autotune", "ngb_deliver_spikes_noalloc",
           "ngb_reserve", "ngb_commit_instance", "ngb_retire_instance", "ngb_instance_info",
           "ngb_eval_step_factor"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libngb.so (building it with nvcc first if allowed and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libngb.so is not built (run __graft_entry__.build())")
    L = C.CDLL(path)
    P = C.c_void_p
    L.ngb_create.argtypes = [C.POINTER(P), C.POINTER(SimConfig)]
    L.ngb_destroy.argtypes = [P]
    L.ngb_last_error.argtypes = [P]
    L.ngb_last_error.restype = C.c_char_p
    L.ngb_add_instance.argtypes = [P, C.c_uint64, C.POINTER(C.c_int32)]
    L.ngb_add_population.argtypes = [P, C.c_int32, C.c_int64, P, C.POINTER(C.c_int32)]
    L.ngb_add_population_in.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, P, C.POINTER(C.c_int32)]
    L.ngb_connect.argtypes = [P, C.c_int32, C.c_int32, C.POINTER(ConnSpec), C.POINTER(SynSpec)]
    L.ngb_connect_stdp.argtypes = [P, C.c_int32, C.c_int32, C.POINTER(ConnSpec), C.POINTER(SynSpec),
                                   C.POINTER(StdpParams)]
    L.ngb_finalize.argtypes = [P]
    L.ngb_simulate.argtypes = [P, C.c_int64]
    L.ngb_simulate_profiled.argtypes = [P, C.c_int64, P, P]
    L.ngb_get_spikes.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, P, P, C.c_int64, C.POINTER(C.c_int64)]
    L.ngb_get_stats.argtypes = [P, C.POINTER(Stats)]
    L.ngb_population_range.argtypes = [P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.ngb_get_state.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, P]
    L.ngb_get_input.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, C.c_int64, P]
    L.ngb_get_src_ptr.argtypes = [P, P]
    L.ngb_get_synapses.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P]
    L.ngb_autotune.argtypes = [P, C.c_int64, C.POINTER(C.c_int32)]
    L.ngb_reserve.argtypes = [P, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32]
    L.ngb_commit_instance.argtypes = [P, C.c_int32]
    L.ngb_retire_instance.argtypes = [P, C.c_int32]
    L.ngb_instance_info.argtypes = [P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    L.ngb_eval_step_factor.argtypes = [P, C.c_int64, C.c_int32, P]
    for name in EXPORTS:
        if name not in ("ngb_last_error",):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class NgbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _check(rc: int, h=None):
    if rc != OK:
        raise NgbError(rc, load().ngb_last_error(h).decode())
    return rc


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def eval_step_factor(r: np.ndarray, k: int) -> np.ndarray:
    """The GPU's Runge-Kutta step-size factor r^(-1/k) (k = 4 or 5) for each ratio in r."""
    r = np.ascontiguousarray(r, dtype=np.float32)
    out = np.zeros_like(r)
    _check(load().ngb_eval_step_factor(_ptr(r), r.size, k, _ptr(out)))
    return out


def _poisson(p: W.Poisson) -> PoissonDrive:
    return PoissonDrive(p.n_inputs, p.rate_hz, p.weight, p.receptor, 0)


def lif_params(p: W.LifParams) -> LifParams:
    return LifParams(p.tau_m, p.C_m, p.E_L, p.V_reset, p.V_th, p.t_ref, p.tau_syn, p.I_e, p.V_init_mean,
                     p.V_init_sd, _poisson(p.poisson))


def aeif_params(p: W.AeifParams) -> AeifParams:
    q = AeifParams(p.C_m, p.g_L, p.E_L, p.V_T, p.Delta_T, p.a, p.b, p.tau_w, p.V_peak, p.V_reset, p.E_ex, p.E_in,
                   p.tau_ex, p.tau_in, p.I_e, p.V_init_mean, p.V_init_sd, p.w_init, p.rk_tol, p.rk_h_min,
                   p.rk_h_init, int(p.rk_max_substeps), int(p.rk_control_fp32), 0, _poisson(p.poisson))
    ports = list(p.ports or [])
    q.n_ports = len(ports)
    for k, (E, tr, td) in enumerate(ports[:4]):
        q.E_rev_mV[k], q.tau_rise_ms[k], q.tau_decay_ms[k] = E, tr, td
    return q


class Simulator:
    """A handle of the C library."""

    def __init__(self, dt_ms: float = 0.1, seed: int = 1, weight_dtype: str = "fp32", device: int = 0,
                 stream: Optional[int] = None, deterministic: bool = False, record_spikes: bool = True,
                 record_capacity: int = 0, steps_per_graph: int = 0, drain_steps: int = 0,
                 delivery: str = "auto"):
        L = load()
        cfg = SimConfig(dt_ms, seed, WEIGHT_DTYPES[weight_dtype], device, stream, int(deterministic),
                        int(record_spikes), record_capacity, steps_per_graph, drain_steps, DELIVERY[delivery], 0)
        h = C.c_void_p()
        _check(L.ngb_create(C.byref(h), C.byref(cfg)))
        self.h = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "h", None):
            load().ngb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        return _check(rc, self.h)

    # ---- construction
    def add_instance(self, seed: int) -> int:
        out = C.c_int32()
        self._c(load().ngb_add_instance(self.h, seed, C.byref(out)))
        return out.value

    def add_population(self, model: str, n: int, params, instance: int = 0) -> int:
        out = C.c_int32()
        par = lif_params(params) if model == W.LIF else aeif_params(params)
        self._c(load().ngb_add_population_in(self.h, instance, MODELS[model], n, C.cast(C.byref(par), C.c_void_p),
                                             C.byref(out)))
        return out.value

    def connect(self, src: int, tgt: int, rule: str, K: int, weight: W.Dist, delay: W.Dist, receptor: int = 0,
                allow_autapses: bool = True, stdp: Optional[W.Stdp] = None):
        conn = ConnSpec(RULES[rule], int(allow_autapses), K)
        syn = SynSpec(DistSpec(DISTS[weight.kind], 0, weight.p0, weight.p1),
                      DistSpec(DISTS[delay.kind], 0, delay.p0, delay.p1), receptor, 0)
        if stdp is None:
            self._c(load().ngb_connect(self.h, src, tgt, C.byref(conn), C.byref(syn)))
        else:
            q = StdpParams(stdp.tau_plus, stdp.tau_minus, stdp.lam, stdp.alpha, stdp.mu_plus, stdp.mu_minus,
                           stdp.W_max)
            self._c(load().ngb_connect_stdp(self.h, src, tgt, C.byref(conn), C.byref(syn), C.byref(q)))

    def finalize(self):
        self._c(load().ngb_finalize(self.h))

    # ---- running
    def simulate(self, steps: int):
        self._c(load().ngb_simulate(self.h, steps))

    def simulate_profiled(self, steps: int) -> Tuple[np.ndarray, np.ndarray]:
        ms = np.zeros(3, dtype=np.float64)
        n = np.zeros(3, dtype=np.int64)
        self._c(load().ngb_simulate_profiled(self.h, steps, _ptr(ms), _ptr(n)))
        return ms, n

    # ---- continuous batching (serving handles)
    def reserve(self, max_neurons: int, max_synapses: int, max_groups: int, ring_slots: int = 64,
                receptors: int = 1):
        self._c(load().ngb_reserve(self.h, max_neurons, max_synapses, max_groups, ring_slots, receptors))

    def commit(self, instance: int):
        self._c(load().ngb_commit_instance(self.h, instance))

    def retire(self, instance: int):
        self._c(load().ngb_retire_instance(self.h, instance))

    def instance_info(self, instance: int):
        t0 = C.c_int64()
        st = C.c_int32()
        self._c(load().ngb_instance_info(self.h, instance, C.byref(t0), C.byref(st)))
        return t0.value, st.value

    def add_spec_instance(self, spec: W.NetSpec) -> Tuple[int, list]:
        """Add the single-instance network `spec` as a new pending instance;
        returns (instance id, population ids)."""
        inst = self.add_instance(spec.seeds[0])
        pops = [self.add_population(p.model, p.n, p.params, instance=inst) for p in spec.pops]
        for c in spec.conns:
            self.connect(pops[c.src], pops[c.tgt], c.rule, c.K, c.weight, c.delay, c.receptor, c.allow_autapses)
        return inst, pops

    def autotune(self, trial_steps: int = 0) -> int:
        """Pick the step loop, delivery grid and (at step 0) delivery scheme by
        timing them; the state is restored."""
        g = C.c_int32()
        self._c(load().ngb_autotune(self.h, trial_steps, C.byref(g)))
        return g.value

    # ---- results / introspection
    def spikes(self, pop: int = -1, t0: int = 0, t1: int = 2**62):
        n = C.c_int64()
        self._c(load().ngb_get_spikes(self.h, pop, t0, t1, None, None, 0, C.byref(n)))
        ids = np.zeros(n.value, dtype=np.int32)
        st = np.zeros(n.value, dtype=np.int64)
        self._c(load().ngb_get_spikes(self.h, pop, t0, t1, _ptr(ids), _ptr(st), n.value, C.byref(n)))
        return ids.astype(np.int64), st

    def stats(self) -> dict:
        s = Stats()
        self._c(load().ngb_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def population_range(self, pop: int):
        off = C.c_int64()
        n = C.c_int64()
        self._c(load().ngb_population_range(self.h, pop, C.byref(off), C.byref(n)))
        return off.value, n.value

    def state(self, var: str, first: int = 0, n: Optional[int] = None) -> np.ndarray:
        if n is None:
            n = self.stats()["num_neurons"] - first
        out = np.zeros(n, dtype=np.float32)
        self._c(load().ngb_get_state(self.h, VARS[var], first, n, _ptr(out)))
        return out

    def input(self, receptor: int = 0, step_offset: int = 0, first: int = 0, n: Optional[int] = None):
        if n is None:
            n = self.stats()["num_neurons"] - first
        out = np.zeros(n, dtype=np.float32)
        self._c(load().ngb_get_input(self.h, receptor, step_offset, first, n, _ptr(out)))
        return out

    def src_ptr(self) -> np.ndarray:
        out = np.zeros(self.stats()["num_neurons"] + 1, dtype=np.uint64)
        self._c(load().ngb_get_src_ptr(self.h, _ptr(out)))
        return out

    def synapses(self, first: int = 0, n: Optional[int] = None):
        if n is None:
            n = self.stats()["num_synapses"] - first
        tgt = np.zeros(n, dtype=np.uint32)
        rc = np.zeros(n, dtype=np.uint8)
        w = np.zeros(n, dtype=np.float32)
        d = np.zeros(n, dtype=np.uint16)
        self._c(load().ngb_get_synapses(self.h, first, n, _ptr(tgt), _ptr(rc), _ptr(w), _ptr(d)))
        return dict(tgt=tgt, receptor=rc, weight=w, delay=d)


def from_spec(spec: W.NetSpec, **kw) -> Simulator:
    """Build a Simulator from a workloads.NetSpec (instances, populations, connections in order)."""
    sim = Simulator(dt_ms=spec.dt, seed=spec.seeds[0], weight_dtype=spec.weight_dtype, **kw)
    for s in spec.seeds[1:]:
        sim.add_instance(s)
    for p in spec.pops:
        sim.add_population(p.model, p.n, p.params, instance=p.instance)
    for c in spec.conns:
        sim.connect(c.src, c.tgt, c.rule, c.K, c.weight, c.delay, c.receptor, c.allow_autapses, c.stdp)
    return sim
