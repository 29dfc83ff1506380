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


def test_pump_half_saturation_and_limits():
    """Each saturating factor of j_pump is 1/2 at its threshold and tends to 1 far above it, so
    j = rho/4 at ([Na]_i, [K]_e) = (P_Na, P_K) and j -> rho for large concentrations; j grows
    with both concentrations."""
    p = table2()
    rho, PNa, PK = p["rho_pump"], p["P_Na"], p["P_K"]
    assert membrane.pump_flux(PNa, PK, rho, PNa, PK) == pytest.approx(rho / 4, rel=1e-15)
    assert membrane.pump_flux(1e9, 1e12, rho, PNa, PK) == pytest.approx(rho, rel=1e-9)
    c = np.linspace(1.0, 50.0, 40)
    assert np.all(np.diff(membrane.pump_flux(c, 4.0, rho, PNa, PK)) > 0)
    assert np.all(np.diff(membrane.pump_flux(12.0, c, rho, PNa, PK)) > 0)


def test_kir_factor_special_values():
    """f_Kir at phi_M = E_K^0 (so D = B), dphi_K = -0.0185 V (so C = 2) and [K]_e = [K]_e^0 is
    (1 + e^0.433)/2; it scales with sqrt([K]_e / [K]_e^0); it falls as dphi_K rises (inward
    rectification: the K conductance is largest for hyperpolarised membranes)."""
    EK0, cK0 = -0.0889, 4.0
    assert membrane.kir_factor(cK0, -0.0185, EK0, EK0, cK0) == pytest.approx((1 + np.exp(0.433)) / 2, rel=1e-14)
    f1 = membrane.kir_factor(cK0, 0.01, -0.07, EK0, cK0)
    assert membrane.kir_factor(4 * cK0, 0.01, -0.07, EK0, cK0) == pytest.approx(2 * f1, rel=1e-14)
    d = np.linspace(-0.05, 0.05, 41)
    assert np.all(np.diff(membrane.kir_factor(cK0, d, -0.07, EK0, cK0)) < 0)


def test_kir_pump_is_electrogenic():
    """With every leak conductance zero the Kir-Na/K currents are the pump's alone:
    I_Na = 3 F z_Na j, I_K = -2 F z_K j, I_Cl = 0, so the net current is F j (one charge out per
    cycle) and I_Na / I_K = -3/2 (3 Na out, 2 K in)."""
    from oracle import problem, system
    from synth import make_config
    cfg = make_config(7)
    pb, s0 = problem.from_config(cfg)
    pb.facet_gleak = np.zeros_like(pb.facet_gleak)
    mf = system.membrane_fields(pb, s0)
    I = system.channel_currents(pb, mf, s0.t)
    j = membrane.pump_flux(s0.c_i[0, 0], s0.c_e[1, 0], pb.rho_pump, pb.P_Na, pb.P_K)
    np.testing.assert_allclose(I.sum(axis=0), pb.F * j, rtol=1e-14)
    np.testing.assert_allclose(I[0] / I[1], -1.5, rtol=1e-14)
    assert np.all(I[2] == 0)
