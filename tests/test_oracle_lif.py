"""Pins of the oracle's LIF exact integration (Eqs. 1-2, Sec. 2.1) -- CPU only.

* The propagators equal the matrix exponential of the linear system (scipy's
  expm), including the constant-current column.
* Closed forms at grid points: membrane under constant current, the response
  to a single PSC (difference of exponentials), and the firing period under a
  suprathreshold current with the refractory period.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2007_14236_gb300 import workloads as W

TAU_M, C_M, TAU_S, DT = 10.0, 250.0, 0.5, 0.1


def _single(I_e=0.0, **kw):
    par = W.LifParams(I_e=I_e, **kw)
    spec = W.NetSpec(name="single", seeds=[1], pops=[W.Population("n", W.LIF, 1, par)])
    net = oracle.OracleNet(spec)
    net.finalize()
    return net, par


def test_propagators_equal_matrix_exponential():
    linalg = pytest.importorskip("scipy.linalg")
    for tau_m, C, tau_s, h in [(10.0, 250.0, 0.5, 0.1), (20.0, 200.0, 2.0, 0.05), (5.0, 100.0, 7.0, 0.3)]:
        P = oracle.lif_propagators(tau_m, C, tau_s, h)
        # state (I, y, I_e): dI/dt = -I/tau_s, dy/dt = I/C - y/tau_m + I_e/C, dI_e/dt = 0
        A = np.array([[-1.0 / tau_s, 0.0, 0.0], [1.0 / C, -1.0 / tau_m, 1.0 / C], [0.0, 0.0, 0.0]])
        E = linalg.expm(A * h)
        assert P["P11"] == pytest.approx(E[0, 0], rel=1e-13)
        assert P["P21"] == pytest.approx(E[1, 0], rel=1e-12)
        assert P["P22"] == pytest.approx(E[1, 1], rel=1e-13)
        assert P["P20"] == pytest.approx(E[1, 2], rel=1e-12)
    # equal time constants: the limit form h/C * exp(-h/tau)
    P = oracle.lif_propagators(4.0, 100.0, 4.0, 0.1)
    A = np.array([[-0.25, 0.0], [0.01, -0.25]])
    assert P["P21"] == pytest.approx(linalg.expm(A * 0.1)[1, 0], rel=1e-12)


def test_constant_current_closed_form():
    I_e = 300.0  # R I_e = 12 mV < 15 mV: subthreshold
    net, par = _single(I_e=I_e)
    R = TAU_M / C_M
    for k in range(1, 401):
        net.simulate(1)
        V = net.state("V_m")[0]
        exact = par.E_L + R * I_e * (1.0 - math.exp(-k * DT / TAU_M))
        assert abs(V - exact) < 2e-5 * abs(par.E_L) + 1e-4, (k, V, exact)


def test_single_psc_closed_form():
    w = 150.0
    net, par = _single()
    net.inject(0, 0, 0, w)  # consumed by the update of step 0
    net.simulate(1)
    assert net.state("I_syn")[0] == pytest.approx(w, rel=1e-7)
    assert net.state("V_m")[0] == pytest.approx(par.E_L, abs=1e-6)
    amp = (w / C_M) * TAU_M * TAU_S / (TAU_M - TAU_S)
    peak_t = TAU_M * TAU_S / (TAU_M - TAU_S) * math.log(TAU_M / TAU_S)
    best = (-1.0, 0)
    for k in range(1, 300):
        net.simulate(1)
        t = k * DT
        y_exact = amp * (math.exp(-t / TAU_M) - math.exp(-t / TAU_S))
        I_exact = w * math.exp(-t / TAU_S)
        y = net.state("V_m")[0] - par.E_L
        assert abs(y - y_exact) < 1e-5 * amp + 1e-6, (k, y, y_exact)
        assert abs(net.state("I_syn")[0] - I_exact) < 1e-6 * w, k
        best = max(best, (y, k))
    # the grid maximum sits next to the analytic peak time
    assert abs(best[1] * DT - peak_t) <= DT


def test_firing_period_with_refractoriness():
    I_e = 500.0  # R I_e = 20 mV > theta = 15 mV
    net, par = _single(I_e=I_e)
    R = TAU_M / C_M
    theta = par.V_th - par.E_L
    # first k with R I_e (1 - exp(-k h / tau_m)) >= theta
    k_star = next(k for k in range(1, 10000) if R * I_e * (1 - math.exp(-k * DT / TAU_M)) >= theta)
    margin = min(abs(R * I_e * (1 - math.exp(-k * DT / TAU_M)) - theta) for k in (k_star - 1, k_star))
    assert margin > 1e-3  # the grid decision is not a rounding tie
    ref_steps = int(round(par.t_ref / DT))
    net.simulate(2000)
    ids, steps = net.spikes()
    assert len(steps) > 5
    assert steps[0] == k_star - 1
    isi = np.diff(steps)
    assert np.all(isi == ref_steps + k_star), (isi[:5], ref_steps, k_star)
    # analytic period (continuous time) lies within one step of the grid period
    period = par.t_ref + TAU_M * math.log(R * I_e / (R * I_e - theta))
    assert abs(isi[0] * DT - period) <= DT


def test_refractory_holds_v_and_current_keeps_decaying():
    net, par = _single(I_e=500.0)
    # run to the first spike
    while len(net.spikes()[0]) == 0:
        net.simulate(1)
    I_at_spike = net.state("I_syn")[0]
    for _ in range(5):
        net.simulate(1)
        assert net.state("V_m")[0] == pytest.approx(par.V_reset, abs=1e-6)
    assert net.state("refractory")[0] == int(round(par.t_ref / DT)) - 5
    assert I_at_spike == 0.0
