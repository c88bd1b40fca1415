"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
use this package.  It loads oracle/_build/libngb_oracle.so (built on demand by
oracle/build.py) and marshals arguments; all arithmetic is in ngb_oracle.cpp.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_VAR = {"V_m": 0, "I_syn": 1, "w": 1, "g_ex": 2, "g_in": 3, "refractory": 4, "h": 5, "dg_ex": 6, "dg_in": 7,
        "g_0": 2, "g_1": 3, "g_2": 8, "g_3": 9, "x_0": 6, "x_1": 7, "x_2": 10, "x_3": 11}


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = C.CDLL(path)
    P = C.c_void_p
    L.ora_last_error.restype = C.c_char_p
    L.ora_create.restype = P
    L.ora_create.argtypes = [C.c_double, C.c_uint64, C.c_int32, C.c_int32, C.c_int32]
    L.ora_destroy.argtypes = [P]
    L.ora_add_instance.argtypes = [P, C.c_uint64]
    L.ora_add_population.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, C.POINTER(C.c_double)]
    L.ora_connect.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                              C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double, C.c_int32]
    L.ora_set_stdp.argtypes = [P, C.c_int32, C.POINTER(C.c_double)]
    L.ora_finalize.argtypes = [P]
    L.ora_simulate.argtypes = [P, C.c_int64]
    L.ora_inject.argtypes = [P, C.c_int64, C.c_int32, C.c_int64, C.c_double]
    for name in ("ora_num_neurons", "ora_num_synapses", "ora_ring_length", "ora_steps_done", "ora_events",
                 "ora_num_spikes", "ora_rk_substeps", "ora_rk_cap_hits"):
        f = getattr(L, name)
        f.restype = C.c_int64
        f.argtypes = [P]
    L.ora_pop_offset.restype = C.c_int64
    L.ora_pop_offset.argtypes = [P, C.c_int32]
    L.ora_get_csr.argtypes = [P, P, P, P, P, P]
    L.ora_get_state.argtypes = [P, C.c_int32, P]
    L.ora_get_input.argtypes = [P, C.c_int32, C.c_int64, P, P, P]
    L.ora_get_spikes.argtypes = [P, P, P]
    L.ora_rows_for_sources.restype = C.c_int64
    L.ora_rows_for_sources.argtypes = [P, C.c_int64, P, C.c_int64, P, P, P, P, P]
    L.ora_philox4x32_10.argtypes = [P, P, P]
    L.ora_poisson_inversion.restype = C.c_int32
    L.ora_poisson_inversion.argtypes = [C.c_double, C.c_uint32]
    L.ora_lif_propagators.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, P]
    L.ora_cash_karp_tableau.argtypes = [P, P, P, P]
    L.ora_round_weight.restype = C.c_float
    L.ora_round_weight.argtypes = [C.c_float, C.c_int32]
    L.ora_normal_from_words.restype = C.c_double
    L.ora_normal_from_words.argtypes = [P]
    L.ora_step_factor_root.restype = C.c_float
    L.ora_step_factor_root.argtypes = [C.c_float, C.c_int32]
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc):
    if rc < 0:
        raise RuntimeError("oracle: " + lib().ora_last_error().decode())
    return rc


# ----------------------------------------------------------- building blocks
def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson_inversion(lam: float, x: int) -> int:
    return int(lib().ora_poisson_inversion(lam, x))


def lif_propagators(tau_m, C_m, tau_syn, h):
    out = np.zeros(4)
    lib().ora_lif_propagators(tau_m, C_m, tau_syn, h, _ptr(out))
    return dict(P11=out[0], P21=out[1], P22=out[2], P20=out[3])


def cash_karp_tableau():
    c = np.zeros(6); a = np.zeros(36); b5 = np.zeros(6); b4 = np.zeros(6)
    lib().ora_cash_karp_tableau(_ptr(c), _ptr(a), _ptr(b5), _ptr(b4))
    return c, a.reshape(6, 6), b5, b4


def round_weight(w: float, prec: int) -> float:
    return float(lib().ora_round_weight(w, prec))


def step_factor_root(r: float, k: int) -> float:
    return float(lib().ora_step_factor_root(r, k))


def normal_from_words(words) -> float:
    w = np.asarray(words, dtype=np.uint32)
    return float(lib().ora_normal_from_words(_ptr(w)))


# ----------------------------------------------------------------- networks
_PREC = {"fp32": 0, "bf16": 1, "fp16": 2}
_DIST = {"const": 0, "normal": 1, "uniform": 2}


def _lif_vec(p):
    return [p.tau_m, p.C_m, p.E_L, p.V_reset, p.V_th, p.t_ref, p.tau_syn, p.I_e, p.V_init_mean,
            p.V_init_sd, p.poisson.n_inputs, p.poisson.rate_hz, p.poisson.weight, p.poisson.receptor]


def _aeif_vec(p, fp64):
    v = [p.C_m, p.g_L, p.E_L, p.V_T, p.Delta_T, p.a, p.b, p.tau_w, p.V_peak, p.V_reset, p.E_ex, p.E_in,
         p.tau_ex, p.tau_in, p.I_e, p.V_init_mean, p.V_init_sd, p.w_init, p.rk_tol, p.rk_h_min,
         p.rk_h_init, float(p.rk_max_substeps), p.poisson.n_inputs, p.poisson.rate_hz, p.poisson.weight,
         p.poisson.receptor, 1.0 if fp64 else 0.0]
    # beta multisynapse ports: count, E_rev[4], tau_rise[4], tau_decay[4]
    ports = list(p.ports or [])
    pad = ports + [(0.0, 1.0, 1.0)] * (4 - len(ports))
    v += [float(len(ports))] + [q[0] for q in pad] + [q[1] for q in pad] + [q[2] for q in pad]
    return v


class OracleNet:
    """One oracle network built from a workloads.NetSpec."""

    def __init__(self, spec, deterministic: bool = False, track_abs: bool = False, adex_fp64: bool = False):
        L = lib()
        self.spec = spec
        self.h = L.ora_create(spec.dt, spec.seeds[0], _PREC[spec.weight_dtype], int(deterministic),
                              int(track_abs))
        if not self.h:
            raise RuntimeError("oracle: " + L.ora_last_error().decode())
        for s in spec.seeds[1:]:
            _check(L.ora_add_instance(self.h, s))
        for p in spec.pops:
            if p.model == "lif_psc_exp":
                v = np.array(_lif_vec(p.params), dtype=np.float64)
                _check(L.ora_add_population(self.h, p.instance, 0, p.n, v.ctypes.data_as(C.POINTER(C.c_double))))
            else:
                v = np.array(_aeif_vec(p.params, adex_fp64), dtype=np.float64)
                model = {"aeif_cond_alpha": 2, "aeif_cond_beta": 3}.get(p.model, 1)
                _check(L.ora_add_population(self.h, p.instance, model, p.n,
                                            v.ctypes.data_as(C.POINTER(C.c_double))))
        for c in spec.conns:
            rule = {"fixed_indegree": 0, "fixed_total_number": 1, "fixed_outdegree": 2, "one_to_one": 3,
                    "all_to_all": 4}[c.rule]
            call = _check(L.ora_connect(self.h, c.src, c.tgt, rule, c.K, int(c.allow_autapses), _DIST[c.weight.kind],
                                 c.weight.p0, c.weight.p1, _DIST[c.delay.kind], c.delay.p0, c.delay.p1,
                                 c.receptor))
            if c.stdp is not None:
                q = c.stdp
                v = np.array([q.tau_plus, q.tau_minus, q.lam, q.alpha, q.mu_plus, q.mu_minus, q.W_max], dtype=np.float64)
                _check(L.ora_set_stdp(self.h, call, v.ctypes.data_as(C.POINTER(C.c_double))))

    def __del__(self):
        if getattr(self, "h", None):
            lib().ora_destroy(self.h)
            self.h = None

    # -- running
    def finalize(self):
        _check(lib().ora_finalize(self.h))

    def simulate(self, steps: int):
        _check(lib().ora_simulate(self.h, steps))

    def inject(self, neuron: int, receptor: int, step_offset: int, value: float):
        _check(lib().ora_inject(self.h, neuron, receptor, step_offset, value))

    # -- introspection
    @property
    def N(self) -> int:
        return int(lib().ora_num_neurons(self.h))

    @property
    def num_synapses(self) -> int:
        return int(lib().ora_num_synapses(self.h))

    @property
    def ring_length(self) -> int:
        return int(lib().ora_ring_length(self.h))

    @property
    def steps(self) -> int:
        return int(lib().ora_steps_done(self.h))

    @property
    def events(self) -> int:
        return int(lib().ora_events(self.h))

    @property
    def rk_substeps(self) -> int:
        return int(lib().ora_rk_substeps(self.h))

    @property
    def rk_cap_hits(self) -> int:
        return int(lib().ora_rk_cap_hits(self.h))

    def pop_offset(self, pop: int) -> int:
        return int(lib().ora_pop_offset(self.h, pop))

    def csr(self):
        K = self.num_synapses
        src_ptr = np.zeros(self.N + 1, dtype=np.uint64)
        tgt = np.zeros(K, dtype=np.uint32)
        rc = np.zeros(K, dtype=np.uint8)
        w = np.zeros(K, dtype=np.float32)
        d = np.zeros(K, dtype=np.uint16)
        _check(lib().ora_get_csr(self.h, _ptr(src_ptr), _ptr(tgt), _ptr(rc), _ptr(w), _ptr(d)))
        return dict(src_ptr=src_ptr, tgt=tgt, receptor=rc, weight=w, delay=d)

    def state(self, var: str) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.float64)
        _check(lib().ora_get_state(self.h, _VAR[var], _ptr(out)))
        return out

    def input(self, receptor: int = 0, step_offset: int = 0):
        out = np.zeros(self.N, dtype=np.float32)
        ab = np.zeros(self.N, dtype=np.float64)
        ex = np.zeros(self.N, dtype=np.float64)
        _check(lib().ora_get_input(self.h, receptor, step_offset, _ptr(out), _ptr(ab), _ptr(ex)))
        return out, ab, ex

    def rows_for_sources(self, srcs):
        """Canonical CSR rows of the given global sources, drawn one by one."""
        srcs = np.ascontiguousarray(np.asarray(srcs, dtype=np.int64))
        n = int(lib().ora_rows_for_sources(self.h, len(srcs), _ptr(srcs), 0, None, None, None, None, None))
        _check(n)
        out = dict(src=np.zeros(n, dtype=np.uint32), tgt=np.zeros(n, dtype=np.uint32),
                   receptor=np.zeros(n, dtype=np.uint8), weight=np.zeros(n, dtype=np.float32),
                   delay=np.zeros(n, dtype=np.uint16))
        lib().ora_rows_for_sources(self.h, len(srcs), _ptr(srcs), n, _ptr(out["src"]), _ptr(out["tgt"]),
                                   _ptr(out["receptor"]), _ptr(out["weight"]), _ptr(out["delay"]))
        return out

    def spikes(self):
        n = int(lib().ora_num_spikes(self.h))
        ids = np.zeros(n, dtype=np.int64)
        st = np.zeros(n, dtype=np.int64)
        _check(lib().ora_get_spikes(self.h, _ptr(ids), _ptr(st)))
        return ids, st
