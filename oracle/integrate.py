"""FP64 CPU oracle for time integration under the flow.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product path never does.

What it computes.  Sec. 2.1 gives the periodic images of a particle (q, p) in
a flow u(x) = A x as (q + L_t n, p + A L_t n): in peculiar momenta p - A q all
images carry the same momentum, and the images of the positions are the
lattice of Sec. 2.1 / 2.2 (L_t = exp(A (t mod T)) L0).  The paper does not
state an integrator; the reading used here (and by the library) is the SLLOD
system for unit mass in peculiar momenta p,

    dq/dt = p + A q,     dp/dt = F(q, t) - A p   (- alpha p with a thermostat),

stepped by a symmetric splitting with h = dt / 2:

    p <- exp(-A h) (s p + h F)                      s: the previous rescale
    p <- sqrt(K0 / |p|^2) p          (isokinetic thermostat only)
    q <- exp(A dt) q + Phi(dt) p,    Phi(dt) = int_0^dt exp(uA) du
    t <- t0 + k dt;  q <- L_t frac(L_t^-1 q)        (unit cell of Sec. 2)
    F <- F(q, t)                                    (the force oracle, FP64)
    p <- h F + exp(-A h) p;  s = sqrt(K0 / |p|^2) (or 1); at the end p <- s p

K0 = |p0|^2.  With F = 0 and no thermostat the momentum part is exact,
p(t) = exp(-tA) p0, and with p = 0 a particle moves with the box,
q(t) = L_t s at fixed s; with A = 0 the step is velocity Verlet.

exp(A tau) is the oracle's expm (symmetric eigen-decomposition or Pade);
Phi is its defining power series  sum_k dt^(k+1) A^k / (k+1)!.
"""
from __future__ import annotations

import math

import numpy as np

from . import evaluate, expm, lattice, wrap


def phi(A, dt, terms=60):
    """Phi(dt) = int_0^dt exp(uA) du = sum_{k>=0} dt^(k+1) A^k / (k+1)!."""
    A = np.asarray(A, dtype=np.float64)
    if np.abs(A).sum(axis=0).max() * dt > 4.0:
        raise ValueError("dt |A| too large for the series")
    out = np.zeros((3, 3))
    term = dt * np.eye(3)                    # dt^(k+1) A^k / (k+1)!, k = 0
    for k in range(terms):
        out = out + term
        term = term @ A * (dt / (k + 2))
    return out


def forces(w, q, t, method="ds"):
    """FP64 forces of the workload's potential at positions q and time t."""
    from dataclasses import replace
    return evaluate(replace(w, q=np.ascontiguousarray(q), t=float(t)), method).F


def trajectory(w, p0, dt, nsteps, thermostat=True, method="ds"):
    """The steps above from w.q, p0 at time w.t, yielding after each step
    (k, q, p, t): q wrapped into the unit cell at t = w.t + k dt, p the peculiar
    momenta before the final rescale."""
    centered = bool(getattr(w, "remap", 0))
    E = expm(w.A, dt)
    Eh = expm(w.A, -0.5 * dt)
    Ph = phi(w.A, dt)
    h = 0.5 * dt
    lat = lattice(w.A, w.L0, w.T, w.t, centered)
    _, q = wrap(lat["L"], lat["Linv"], np.asarray(w.q, dtype=np.float64))
    p = np.array(p0, dtype=np.float64, copy=True)
    k0 = float(np.sum(p * p))
    F = forces(w, q, w.t, method)
    scale = 1.0
    t = w.t
    for k in range(nsteps):
        p = (scale * p + h * F) @ Eh.T
        if thermostat:
            p = p * math.sqrt(k0 / float(np.sum(p * p)))
        q = q @ E.T + p @ Ph.T
        t = w.t + (k + 1) * dt
        lat = lattice(w.A, w.L0, w.T, t, centered)
        _, q = wrap(lat["L"], lat["Linv"], q)
        F = forces(w, q, t, method)
        p = h * F + p @ Eh.T
        scale = math.sqrt(k0 / float(np.sum(p * p))) if thermostat else 1.0
        yield k + 1, q, p, t, scale


def integrate(w, p0, dt, nsteps, thermostat=True, method="ds"):
    """The steps above from w.q, p0 at time w.t.  Returns (q, p, t): q wrapped
    into the unit cell at t = w.t + nsteps dt, p the peculiar momenta."""
    lat = lattice(w.A, w.L0, w.T, w.t, bool(getattr(w, "remap", 0)))
    _, q = wrap(lat["L"], lat["Linv"], np.asarray(w.q, dtype=np.float64))
    p, t, scale = np.array(p0, dtype=np.float64, copy=True), w.t, 1.0
    for _, q, p, t, scale in trajectory(w, p0, dt, nsteps, thermostat, method):
        pass
    return q, scale * p, t


def energy(w, q, p, t, method="ds"):
    """U + |p|^2 / 2 at (q, p, t)."""
    from dataclasses import replace
    r = evaluate(replace(w, q=np.ascontiguousarray(q), t=float(t)), method)
    return float(r.U) + 0.5 * float(np.sum(p * p))
