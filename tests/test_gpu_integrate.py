"""Time integration under the flow through the C ABI (nemd_integrate) against
the FP64 integration oracle, and its invariants on the device."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import integrate as OI
from paper_1412_3784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

DS, DO = 0, 1


def _ctx(w):
    ctx = nemd.Context(0)
    ctx.set_flow(w.A, w.L0, w.M, w.T)
    ctx.set_potential(nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ, w.eps, w.sigma, w.shift)
    if getattr(w, "remap", 0):
        ctx.set_option(nemd.NEMD_OPT_REMAP, 1)
    return ctx


def run_gpu(w, p0, dt, nsteps, variant, thermostat=1, kernel=2, graph=1):
    ctx = _ctx(w)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, kernel)
    ctx.set_option(nemd.NEMD_OPT_INT_GRAPH, graph)
    q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(p0)).cuda()
    ctx.integrate(q, p, w.t, dt, nsteps, variant, w.rc, thermostat)
    ctx.sync()
    out = q.cpu().numpy(), p.cpu().numpy()
    ctx.close()
    return out


def lattice_at(w, t):
    return oracle.lattice(w.A, w.L0, w.T, t, centered=bool(getattr(w, "remap", 0)))


def pos_err(w, t, qa, qb):
    """max |qa - qb| modulo the lattice of time t."""
    lat = lattice_at(w, t)
    d = (qa - qb) @ lat["Linv"].T
    d -= np.rint(d)
    return float(np.abs(d @ lat["L"].T).max())


@pytest.mark.parametrize("variant", [DS, DO])
def test_trajectory_matches_the_oracle(variant):
    """N = 4000 WCA under the general flow, isokinetic, 25 steps from t = 0.3 T."""
    ser = W.StrainSeries(W.M_GENERAL, 10, 21, kind=W.POT_WCA)
    w = ser.workload(0.3 * ser.period)
    p0 = W.maxwell_momenta(w.n, 1.0, seed=22)
    dt, m = 0.004, 25
    qg, pg = run_gpu(w, p0, dt, m, variant)
    qo, po, t = OI.integrate(w, p0, dt, m, thermostat=True)
    assert pos_err(w, t, qg, qo) <= 2e-5
    assert np.abs(pg - po).max() <= 1e-4 * np.abs(po).max()
    assert abs(np.sum(pg * pg) / np.sum(p0 * p0) - 1.0) <= 1e-12      # isokinetic on the device


def test_trajectory_across_the_remap_lj():
    """N = 4000 LJ, 20 steps across t = T (the lattice jumps from L0 M to L0)."""
    ser = W.StrainSeries(W.M_GENERAL, 10, 23)
    dt, m = 0.005, 20
    w = ser.workload(ser.period - 10.5 * dt)
    p0 = W.maxwell_momenta(w.n, 0.8, seed=24)
    qg, pg = run_gpu(w, p0, dt, m, DO)
    qo, po, t = OI.integrate(w, p0, dt, m, thermostat=True)
    assert t > ser.period
    assert pos_err(w, t, qg, qo) <= 2e-5
    assert np.abs(pg - po).max() <= 1e-4 * np.abs(po).max()


def test_shear_flow_trajectory():
    """Lees-Edwards shear remapped half way (NEMD_OPT_REMAP = 1), 20 steps."""
    sh = W.shear_series(k=10, seed=25)
    w = sh.workload(0.45 * sh.period)
    p0 = W.maxwell_momenta(w.n, 1.0, seed=26)
    qg, pg = run_gpu(w, p0, 0.004, 20, DS)
    qo, po, t = OI.integrate(w, p0, 0.004, 20, thermostat=True)
    assert pos_err(w, t, qg, qo) <= 2e-5
    assert np.abs(pg - po).max() <= 1e-4 * np.abs(po).max()


def test_free_flight_follows_the_flow_exactly():
    """No pairs (rc tiny and momenta too small for any two particles to come
    within it), no thermostat: p(t) = exp(-tA) p0 to rounding, and with p0 = 0
    the positions move with the flow, q = exp(tA) q0 mod L."""
    ser = W.StrainSeries(W.M_GENERAL, 4, 27, rc=0.05)
    w = ser.workload(0.0)
    rng = np.random.default_rng(28)
    p0 = 0.01 * rng.normal(size=(w.n, 3))
    dt, m = ser.period / 29.0, 40
    qg, pg = run_gpu(w, p0, dt, m, DO, thermostat=0)
    pe = p0 @ oracle.expm(w.A, -m * dt).T
    assert np.abs(pg - pe).max() <= 1e-11 * np.abs(pe).max()
    qg, pg = run_gpu(w, np.zeros_like(p0), dt, m, DS, thermostat=0)
    lat0 = lattice_at(w, 0.0)
    _, q0 = oracle.wrap(lat0["L"], lat0["Linv"], w.q)
    assert pos_err(w, m * dt, qg, q0 @ oracle.expm(w.A, m * dt).T) <= 1e-10
    assert np.abs(pg).max() == 0.0


def test_energy_is_conserved_without_flow_or_thermostat():
    """A = 0, LJ N = 4000, velocity Verlet for 200 steps of dt = 0.002."""
    w = W.config_equilibrium_wca()
    w = replace(w, kind=W.POT_LJ, rc=2.5)
    p0 = W.maxwell_momenta(w.n, 0.7, seed=29)
    e0 = OI.energy(w, w.q, p0, 0.0)
    qg, pg = run_gpu(w, p0, 0.002, 200, DO, thermostat=0)
    e1 = OI.energy(w, qg, pg, 200 * 0.002)
    assert abs(e1 - e0) <= 1e-3 * abs(e0)


def test_repeats_bit_for_bit_and_validates_arguments():
    """Two runs, and the replayed step graph against launching every step,
    agree bit for bit; bad arguments are refused."""
    ser = W.StrainSeries(W.M_GENERAL, 6, 30, kind=W.POT_WCA)
    w = ser.workload(0.2)
    p0 = W.maxwell_momenta(w.n, 1.0, seed=31)
    a = run_gpu(w, p0, 0.004, 10, DO)
    b = run_gpu(w, p0, 0.004, 10, DO)
    c = run_gpu(w, p0, 0.004, 10, DO, graph=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    for m in (0, 1, 2, 3):
        d = run_gpu(w, p0, 0.004, m, DS)
        e = run_gpu(w, p0, 0.004, m, DS, graph=0)
        assert np.array_equal(d[0], e[0]) and np.array_equal(d[1], e[1])
    ctx = _ctx(w)
    q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(p0)).cuda()
    with pytest.raises(nemd.NemdError):
        ctx.integrate(q, p, 0.0, -0.01, 3, DO, w.rc)            # dt <= 0
    with pytest.raises(nemd.NemdError):
        ctx.integrate(torch.from_numpy(w.q.copy()), p, 0.0, 0.01, 3, DO, w.rc)   # host positions
    ctx.close()
