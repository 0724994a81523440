"""The Verlet list of nemd_integrate (nemd_set_verlet) through the C ABI.

* Every step of a 200-step trajectory under the general 3-D flow that crosses a
  remap: the pair set the list evaluates is bit-exact against the FP64 oracle's
  brute force on the GPU's own positions and time, with the list rebuilt only
  now and then (both cell-list variants build it).
* The trajectory with the list equals the one with the per-step cell list.
* Wrapping and image bookkeeping: positions moved by lattice vectors between
  calls give the same pairs.
"""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

DS, DO = 0, 1
DT = 0.004


def _ctx(w, skin, record=0):
    ctx = nemd.Context(0)
    ctx.set_flow(w.A, w.L0, w.M, w.T)
    ctx.set_potential(nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ, w.eps, w.sigma, w.shift)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
    ctx.set_option(nemd.NEMD_OPT_RECORD_PAIRS, record)
    ctx.set_verlet(skin)
    return ctx


def _brute_keys(w, q, t):
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    s, qp = oracle.wrap(lat["L"], lat["Linv"], q)
    r = oracle.brute(lat["L"], s, qp, w.rc, want_pairs=True)
    return oracle.canonical_pair_keys(r.pairs), r.npairs


@pytest.mark.parametrize("variant", [DS, DO])
def test_pair_sets_bit_exact_every_step_across_a_remap(variant):
    """N = 864 LJ (rc 2.5) under the general flow from t = 0.7 T: 200 steps of
    dt = 0.004 cross the remap at t = T."""
    w = W.config_flow(W.M_GENERAL, 6, 0.7, 51)
    p0 = W.maxwell_momenta(w.n, 1.0, 52)
    ctx = _ctx(w, 0.3, record=60 * w.n + 1000)
    q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(p0)).cuda()
    t = w.t
    crossed = False
    for k in range(200):
        ctx.integrate(q, p, t, DT, 1, variant, w.rc, 1)
        ctx.sync()
        t_new = w.t + (k + 1) * DT
        crossed |= int(t_new) != int(t)
        t = t_new
        ref, npairs = _brute_keys(w, q.cpu().numpy(), t)
        got = oracle.canonical_pair_keys(ctx.pairs())
        assert ctx.stats()["pairs"] == npairs, k
        assert np.array_equal(got, ref), k
    builds, steps, width, _ = ctx.verlet_stats()
    assert crossed
    assert 2 <= builds < steps // 3        # reused, and rebuilt (the remap at least)
    assert width > 0
    ctx.close()


def test_trajectory_equals_cell_list_trajectory():
    """30 steps with the list and with the per-step cell list from one state."""
    w = W.config_flow(W.M_GENERAL, 8, 0.2, 53)
    p0 = W.maxwell_momenta(w.n, 1.0, 54)
    out = []
    for skin in (0.0, 0.3):
        ctx = _ctx(w, skin)
        q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(p0)).cuda()
        ctx.integrate(q, p, w.t, DT, 30, nemd.NEMD_AUTO_HEURISTIC, w.rc, 1)
        ctx.sync()
        out.append((q.cpu().numpy(), p.cpu().numpy()))
        ctx.close()
    t = w.t + 30 * DT
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    d = (out[0][0] - out[1][0]) @ lat["Linv"].T
    d -= np.rint(d)
    assert np.abs(d @ lat["L"].T).max() < 1e-6
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-5 * np.abs(out[0][1]).max()


def test_images_follow_lattice_shifts_between_calls():
    """Positions moved by arbitrary lattice vectors between two calls give the
    same pair set as the oracle, and the list is kept (its images re-derived):
    a mildly strained crystal started at rest, small steps."""
    dt = 0.0005
    w = W.config_flow(W.M_GENERAL, 6, 0.05, 55)
    p0 = np.zeros((w.n, 3))
    ctx = _ctx(w, 0.4, record=60 * w.n + 1000)
    q = torch.from_numpy(np.ascontiguousarray(w.q)).cuda()
    p = torch.from_numpy(p0).cuda()
    ctx.integrate(q, p, w.t, dt, 1, DS, w.rc, 0)
    ctx.sync()
    t = w.t + dt
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    rng = np.random.default_rng(3)
    qs = q.cpu().numpy() + rng.integers(-2, 3, size=(w.n, 3)) @ lat["L"].T
    q.copy_(torch.from_numpy(qs))
    ctx.integrate(q, p, t, dt, 1, DS, w.rc, 0)
    ctx.sync()
    ref, _ = _brute_keys(w, q.cpu().numpy(), t + dt)
    assert np.array_equal(oracle.canonical_pair_keys(ctx.pairs()), ref)
    builds, steps, _, delta = ctx.verlet_stats()
    assert builds == 1 and steps == 4     # two evaluations per call, one build
    assert 0.0 < delta < 0.2
    ctx.close()
