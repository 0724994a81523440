"""Pins of the FP64 integration oracle (oracle/integrate.py) against what the
mathematics fixes, independent of the oracle's own formulas:

* Phi(dt) = int_0^dt exp(uA) du satisfies A Phi = exp(dt A) - I;
* no forces, no thermostat, p = 0: a particle moves with the flow,
  q(t) = exp(tA) q0 modulo the lattice, its fractional coordinates fixed
  within a period and mapped by M at the remap of Sec. 2.2;
* no forces, no thermostat: p(t) = exp(-tA) p0 (closed form, eigenbasis of the
  symmetric A), and positions converge at second order to the closed-form
  solution q(t) = exp(tA) q0 + V diag(sinh(t lam)/lam) V^T p0;
* A = 0, no thermostat (velocity Verlet): energy error O(dt^2) and exact time
  reversibility;
* no forces under Lees-Edwards shear (A^2 = 0): the closed form
  p = (I - tA) p0, q = (I + tA) q0 + t p0, across the centred remap;
* isokinetic thermostat: |p|^2 stays at its initial value.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import integrate as OI
from paper_1412_3784_gb300 import workloads as W


def _flow_system(k=3, seed=2, rc=0.05, vac=0):
    """General KR flow; rc tiny: no pairs, zero forces."""
    ser = W.StrainSeries(W.M_GENERAL, k, seed, rc=rc, vacancies=vac)
    return ser, ser.workload(0.0)


def test_phi_satisfies_its_defining_identity():
    ser, _ = _flow_system()
    for dt in (0.001, 0.05, 0.3):
        P = OI.phi(ser.A, dt)
        E = oracle.expm(ser.A, dt)
        assert np.abs(ser.A @ P - (E - np.eye(3))).max() <= 1e-13
        # and reduces to dt I for A = 0
        assert np.abs(OI.phi(np.zeros((3, 3)), dt) - dt * np.eye(3)).max() == 0.0


def test_affine_motion_follows_the_flow_across_the_remap():
    """p = 0, no forces: q(t) = exp((t - t0) A) q0 modulo the lattice of time t;
    within a period the fractional coordinates stay fixed, and at the remap
    (L_T = L0 M, the same lattice) they become M s mod 1."""
    ser, w = _flow_system()
    p0 = np.zeros((w.n, 3))
    lat0 = oracle.lattice(w.A, w.L0, w.T, w.t)
    s0, q0 = oracle.wrap(lat0["L"], lat0["Linv"], w.q)
    dt = ser.period / 37.0
    q, p, t = OI.integrate(w, p0, dt, 30, thermostat=False)      # t = 0.81 T: no remap yet
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    s, _ = oracle.wrap(lat["L"], lat["Linv"], q)
    d = s - s0
    d -= np.rint(d)
    assert np.abs(d).max() <= 1e-12
    q, p, t = OI.integrate(w, p0, dt, 53, thermostat=False)      # t = 1.43 T: one remap
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    d = (q - q0 @ oracle.expm(w.A, t - w.t).T) @ lat["Linv"].T
    d -= np.rint(d)
    assert np.abs(d).max() <= 1e-11
    s, _ = oracle.wrap(lat["L"], lat["Linv"], q)
    d = s - (s0 @ np.asarray(w.M, dtype=np.float64).T)             # s' = M s mod 1 after the remap
    d -= np.rint(d)
    assert np.abs(d).max() <= 1e-11
    assert np.abs(p).max() == 0.0


def _closed_form(ser, q0, p0, t):
    """Exact solution without forces: p = V e^{-t lam} V^T p0,
    q = e^{tA} q0 + V diag(sinh(t lam) / lam) V^T p0 (A = V diag(lam) V^T)."""
    lam, V = np.linalg.eigh(ser.A)
    p = (V @ np.diag(np.exp(-t * lam)) @ V.T @ p0.T).T
    g = np.where(np.abs(lam) > 0, np.sinh(t * lam) / np.where(lam == 0, 1, lam), t)
    q = (V @ np.diag(np.exp(t * lam)) @ V.T @ q0.T).T + (V @ np.diag(g) @ V.T @ p0.T).T
    return q, p


def test_free_flight_momenta_exact_positions_second_order():
    ser, w = _flow_system(k=2)
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=(w.n, 3))
    lat0 = oracle.lattice(w.A, w.L0, w.T, w.t)
    _, q0 = oracle.wrap(lat0["L"], lat0["Linv"], w.q)
    t_end = 0.8 * ser.period
    errs = []
    for m in (40, 80, 160):
        q, p, t = OI.integrate(w, p0, t_end / m, m, thermostat=False)
        qe, pe = _closed_form(ser, q0, p0, t)
        assert np.abs(p - pe).max() <= 1e-12 * np.abs(pe).max()
        lat = oracle.lattice(w.A, w.L0, w.T, t)
        d = (q - qe) @ lat["Linv"].T            # compare modulo the lattice
        d -= np.rint(d)
        errs.append(np.abs(d @ lat["L"].T).max())
    assert errs[0] > 0
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_free_flight_under_shear_closed_form():
    """Lees-Edwards shear (A = g e_x e_y^T, A^2 = 0), no forces, no thermostat:
    p(t) = (I - tA) p0 and q(t) = (I + tA) q0 + t p0 exactly, modulo the
    lattice; the splitting is exact here (every propagator is a polynomial of
    degree one in A), and the centred remap of Sec. 2.2 is crossed."""
    sh = W.shear_series(k=2, seed=3, rate=0.9)
    w = replace(sh.workload(0.3 * sh.period), rc=0.05)
    rng = np.random.default_rng(12)
    p0 = 0.01 * rng.normal(size=(w.n, 3))
    lat0 = oracle.lattice(w.A, w.L0, w.T, w.t, centered=True)
    _, q0 = oracle.wrap(lat0["L"], lat0["Linv"], w.q)
    dt, m = sh.period / 17.0, 20                      # crosses t = T/2 (the remap)
    q, p, t = OI.integrate(w, p0, dt, m, thermostat=False)
    tt = t - w.t
    pe = p0 @ (np.eye(3) - tt * w.A).T
    qe = q0 @ (np.eye(3) + tt * w.A).T + tt * p0
    assert np.abs(p - pe).max() <= 1e-14
    lat = oracle.lattice(w.A, w.L0, w.T, t, centered=True)
    d = (q - qe) @ lat["Linv"].T
    d -= np.rint(d)
    assert np.abs(d @ lat["L"].T).max() <= 1e-12


def _equilibrium(kind, seed=11):
    rng = np.random.default_rng(seed)
    s, side, delta = W.perturbed_fcc(4, 0.8442, rng)
    L0 = side * np.eye(3)
    q = s @ L0.T + delta
    return W.Workload(name="rest", A=np.zeros((3, 3)), L0=L0, M=np.eye(3, dtype=np.int64), T=1.0, t=0.0,
                      q=q, kind=kind, rc=W.WCA_RC if kind == W.POT_WCA else 2.5)


def test_velocity_verlet_energy_error_is_second_order():
    """WCA (force continuous at the cut-off): the energy error after a fixed
    time falls about fourfold per halving of dt."""
    w = _equilibrium(W.POT_WCA)
    p0 = W.maxwell_momenta(w.n, 0.7, seed=3)
    e0 = OI.energy(w, w.q, p0, 0.0)
    err = []
    for dt, m in ((0.004, 50), (0.002, 100), (0.001, 200)):
        q, p, t = OI.integrate(w, p0, dt, m, thermostat=False)
        err.append(abs(OI.energy(w, q, p, t) - e0))
    assert err[0] / abs(e0) < 1e-3
    assert 2.8 < err[0] / err[1] < 5.0 and 2.8 < err[1] / err[2] < 5.0, err


def test_velocity_verlet_is_time_reversible():
    w = _equilibrium(W.POT_LJ)
    p0 = W.maxwell_momenta(w.n, 0.7, seed=5)
    q1, p1, t1 = OI.integrate(w, p0, 0.003, 40, thermostat=False)
    from dataclasses import replace
    q2, p2, _ = OI.integrate(replace(w, q=q1, t=t1), -p1, 0.003, 40, thermostat=False)
    L = w.L0
    d = (q2 - w.q) @ np.linalg.inv(L).T
    d -= np.rint(d)
    assert np.abs(d @ L.T).max() <= 1e-9
    assert np.abs(p2 + p0).max() <= 1e-9


def test_isokinetic_thermostat_holds_the_kinetic_energy():
    ser = W.StrainSeries(W.M_GENERAL, 4, 7, kind=W.POT_WCA)
    w = ser.workload(0.1 * ser.period)
    p0 = W.maxwell_momenta(w.n, 1.0, seed=8)
    q, p, t = OI.integrate(w, p0, 0.003, 30, thermostat=True)
    assert abs(np.sum(p * p) / np.sum(p0 * p0) - 1.0) <= 1e-12
    assert abs(t - (w.t + 30 * 0.003)) <= 1e-15
