"""Membrane models at the membrane nodes (Sections 2.4 and 3.2).

All membrane coefficients are nodal: they are evaluated at the membrane vertices
(as the paper does for the gating ODE, Section 3.3) and enter the facet
integrals as P1 functions.

* reversal potential  E_k = RT/(F z_k) ln([k]_e/[k]_i)                      (Section 2.4.1)
* capacitive split    alpha_r^k = D_r^k z_k^2 [k]_r / sum_l D_r^l z_l^2 [l]_r   (Section 2.2)
* C_r^k = alpha_r^k C_m / (F z_k)                                            (Eq. 3.6)
* Hodgkin-Huxley gates by N_ode Rush-Larsen substeps with phi_M frozen at phi_M^{n-1} (Section 3.2)
* channel driving terms q = G(w) (phi_M - E_k): leak G = 1, HH Na m^3 h, HH K n^4 (Eq. 2.15)
* Kir-Na/K (Section 2.4.2): the K leak is rectified by f_Kir([K]_e, phi_M - E_K, phi_M), and a
  Na/K pump of flux density j_pump([Na]_i, [K]_e) adds 3 F z_Na j_pump to the Na current and
  -2 F z_K j_pump to the K current. E_K^0 and [K]_e^0 are the t = 0 values (the uniform
  initial concentrations).

The HH-1952 rates are not printed in the paper (Section 2.4.1 cites HH-1952);
the reading used is the textbook set in the modern sign convention with
V = phi_M - phi_rest in mV and rates in 1/ms. Pinned by
tests/test_oracle_membrane.py (steady-state gates reproduce Table 2's m0, h0,
n0 at phi_M^0; Rush-Larsen substeps equal the closed-form step; alpha sums to 1).
"""
from __future__ import annotations

import numpy as np


def reversal_potential(R, T, F, z, c_i, c_e):
    return (R * T / (F * z)) * np.log(c_e / c_i)


def alpha_split(D, z, c):
    """c: (n_ions, n) concentrations of one region at the membrane nodes."""
    w = (np.asarray(D)[:, None] * np.asarray(z)[:, None] ** 2) * c
    return w / w.sum(axis=0, keepdims=True)


def _vtrap(x):
    """x / (exp(x) - 1), continuous at 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-6
    out[~small] = x[~small] / np.expm1(x[~small])
    xs = x[small]
    out[small] = 1.0 - xs / 2.0 + xs * xs / 12.0
    return out


def hh_rates(V):
    """(alpha, beta) for gates (n, m, h); V in mV relative to rest, rates in 1/ms."""
    a_n = 0.1 * _vtrap((10.0 - V) / 10.0)
    b_n = 0.125 * np.exp(-V / 80.0)
    a_m = 1.0 * _vtrap((25.0 - V) / 10.0)
    b_m = 4.0 * np.exp(-V / 18.0)
    a_h = 0.07 * np.exp(-V / 20.0)
    b_h = 1.0 / (np.exp((30.0 - V) / 10.0) + 1.0)
    return np.stack([a_n, a_m, a_h]), np.stack([b_n, b_m, b_h])


def hh_steady_state(V):
    a, b = hh_rates(V)
    return a / (a + b)


def rush_larsen(w, phi_M, phi_rest, dt, n_ode):
    """N_ode Rush-Larsen substeps of dt/N_ode for dw/dt = a(1-w) - b w, phi_M frozen.

    w: (3, n) gates (n, m, h); phi_M, phi_rest in volts; dt in seconds.
    """
    V = 1e3 * (phi_M - phi_rest)
    a, b = hh_rates(V)
    winf = a / (a + b)
    h = 1e3 * dt / n_ode
    decay = np.exp(-(a + b) * h)
    w = np.array(w, dtype=np.float64, copy=True)
    for _ in range(n_ode):
        w = winf + (w - winf) * decay
    return w


def stimulus_conductance(kind, gbar, t, t0, t1, a, tau):
    """g_stim^Na(t): 0 (none), gbar on [t0, t1) (window), gbar exp(-(t mod tau)/a) (Model A)."""
    if kind == 0:
        return 0.0
    if kind == 1:
        return gbar if (t0 <= t < t1) else 0.0
    if kind == 2:
        return gbar * np.exp(-np.mod(t, tau) / a)
    raise ValueError(kind)


def kir_factor(cKe, dphi_K, phi_M, E_K0, cKe0):
    """f_Kir of Section 2.4.2 (potentials in volts, concentrations in mol/m^3):
    A B / (C D) sqrt([K]_e / [K]_e^0) with A = 1 + e^0.433, B = 1 + e^{-(0.1186 + E_K^0)/0.0441},
    C = 1 + e^{(dphi_K + 0.0185)/0.0425}, D = 1 + e^{-(0.1186 + phi_M)/0.0441}, dphi_K = phi_M - E_K."""
    A = 1.0 + np.exp(0.433)
    B = 1.0 + np.exp(-(0.1186 + E_K0) / 0.0441)
    C = 1.0 + np.exp((dphi_K + 0.0185) / 0.0425)
    D = 1.0 + np.exp(-(0.1186 + phi_M) / 0.0441)
    return A * B / (C * D) * np.sqrt(cKe / cKe0)


def pump_flux(cNa_i, cK_e, rho, P_Na, P_K):
    """Na/K pump flux density (mol/(m^2 s)) of Section 2.4.2:
    rho [Na]_i^1.5 / ([Na]_i^1.5 + P_Na^1.5) * [K]_e / ([K]_e + P_K)."""
    a = cNa_i ** 1.5
    return rho * a / (a + P_Na ** 1.5) * cK_e / (cK_e + P_K)
