"""Pins for oracle/membrane.py: Table 2 gate values, textbook HH-1952 resting values,
exactness of Rush-Larsen for a frozen potential, alpha partition, reversal potentials."""
import numpy as np
import pytest

from oracle import membrane
from synth.configs import table2

from helpers import paper_values


def test_gates_at_phi_M0_match_table2():
    p = table2()
    V = 1e3 * (p["phi_M0"] - p["phi_rest"])           # -2.74 mV
    n, m, h = membrane.hh_steady_state(np.array([V]))[:, 0]
    # Table 2: n0 = 0.276, m0 = 0.0379, h0 = 0.688 (printed to 3 significant digits)
    g = paper_values()["table2_initial_gates"]
    assert abs(n - g["n0"]) < 1.5e-3 and abs(m - g["m0"]) < 5e-4 and abs(h - g["h0"]) < 1.5e-3


def test_textbook_resting_values():
    # HH-1952 at V = 0 (rest): n_inf = 0.3177, m_inf = 0.0529, h_inf = 0.5961
    n, m, h = membrane.hh_steady_state(np.array([0.0]))[:, 0]
    assert abs(n - 0.31768) < 5e-5 and abs(m - 0.05293) < 5e-5 and abs(h - 0.59612) < 5e-5
    a, b = membrane.hh_rates(np.array([0.0]))
    np.testing.assert_allclose(a[:, 0], [0.1 / (np.e - 1), 2.5 / (np.exp(2.5) - 1), 0.07], rtol=1e-14)
    np.testing.assert_allclose(b[:, 0], [0.125, 4.0, 1 / (np.exp(3.0) + 1)], rtol=1e-14)


def test_removable_singularities():
    a, _ = membrane.hh_rates(np.array([10.0, 25.0, 10.0 + 1e-9, 25.0 - 1e-9]))
    assert abs(a[0, 0] - 0.1) < 1e-15 and abs(a[1, 1] - 1.0) < 1e-15
    assert abs(a[0, 2] - 0.1) < 1e-10 and abs(a[1, 3] - 1.0) < 1e-9


def test_rush_larsen_is_exact_for_frozen_potential():
    rng = np.random.default_rng(0)
    phi = rng.uniform(-0.09, 0.03, 50)
    w0 = rng.uniform(0, 1, (3, 50))
    dt = 5e-5
    w25 = membrane.rush_larsen(w0, phi, -0.065, dt, 25)
    w1 = membrane.rush_larsen(w0, phi, -0.065, dt, 1)
    np.testing.assert_allclose(w25, w1, rtol=1e-13, atol=1e-15)
    # independent check: fine RK4 of dw/dt = a(1-w) - b w
    V = 1e3 * (phi + 0.065)
    a, b = membrane.hh_rates(V)
    w = w0.copy()
    hs = 1e3 * dt / 2000
    f = lambda w: a * (1 - w) - b * w
    for _ in range(2000):
        k1 = f(w); k2 = f(w + hs / 2 * k1); k3 = f(w + hs / 2 * k2); k4 = f(w + hs * k3)
        w = w + hs / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    np.testing.assert_allclose(w25, w, rtol=1e-11, atol=1e-13)


def test_alpha_partition_and_reversal():
    p = table2()
    c = np.array([[12.0, 100.0], [125.0, 4.0], [137.0, 104.0]])
    a = membrane.alpha_split(p["D"], p["z"], c)
    np.testing.assert_allclose(a.sum(axis=0), 1.0, rtol=0, atol=1e-15)
    assert np.all((a >= 0) & (a <= 1))
    E = membrane.reversal_potential(p["R"], p["T"], p["F"], np.array(p["z"]), c[:, 0], c[:, 1])
    psi = p["R"] * p["T"] / p["F"]
    np.testing.assert_allclose(E, [psi * np.log(100 / 12), psi * np.log(4 / 125), -psi * np.log(104 / 137)])
    # leak rest potential of the 2D workload (g_Na, g_K, g_Cl) = (0.2, 0.8, 0): -60.22 mV
    assert abs(1e3 * (0.2 * E[0] + 0.8 * E[1]) - (-60.22)) < 0.01


def test_stimulus_shapes():
    assert membrane.stimulus_conductance(1, 40.0, 0.5e-3, 0.0, 1e-3, 0, 0) == 40.0
    assert membrane.stimulus_conductance(1, 40.0, 1e-3, 0.0, 1e-3, 0, 0) == 0.0
    g = membrane.stimulus_conductance(2, 40.0, 12e-3, 0, 0, 2e-3, 10e-3)
    assert abs(g - 40.0 * np.exp(-1.0)) < 1e-12
