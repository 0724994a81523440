"""Pins of the FP64 Verlet-list oracle (oracle/verlet.py) against brute force.

Along an oracle trajectory under the general 3-D flow that crosses a remap,
the skin list -- rebuilt by its rule (deformation bound and peculiar
displacements) and at the remap -- gives exactly the brute-force pair set of
the positions at every step.  A list that is never rebuilt does not: the pin
can fail.
"""
import numpy as np

import oracle
from oracle import integrate as OI
from oracle import verlet as OV
from paper_1412_3784_gb300 import workloads as W


def _trajectory(nsteps, t0, k=5, seed=41, dt=0.004):
    w = W.config_flow(W.M_GENERAL, k, t0, seed)
    p0 = W.maxwell_momenta(w.n, 1.0, seed + 1)
    return w, OI.trajectory(w, p0, dt, nsteps, thermostat=True)


def _brute_keys(w, q, t):
    lat = oracle.lattice(w.A, w.L0, w.T, t)
    s, qp = oracle.wrap(lat["L"], lat["Linv"], q)
    return oracle.canonical_pair_keys(oracle.brute(lat["L"], s, qp, w.rc, want_pairs=True).pairs), lat


def test_skin_list_equals_brute_force_at_every_step_across_a_remap():
    w, traj = _trajectory(120, 0.8)
    vl = OV.SkinList(w.rc, 0.3, w.A)
    lat0 = oracle.lattice(w.A, w.L0, w.T, w.t)
    vl.build(lat0["L"], lat0["Linv"], w.q, w.t)
    per = OV.period_index(w.t, w.T)
    crossed = False
    for _, q, _, t, _ in traj:
        ref, lat = _brute_keys(w, q, t)
        per_t = OV.period_index(t, w.T)
        remapped = per_t != per
        crossed |= remapped
        per = per_t
        if vl.must_rebuild(lat["L"], lat["Linv"], q, t, remapped):
            vl.build(lat["L"], lat["Linv"], q, t)
        assert np.array_equal(oracle.canonical_pair_keys(vl.pairs_at(lat["L"], lat["Linv"], q)), ref), t
    assert crossed                 # the trajectory went through a remap
    assert 3 <= vl.builds < 60     # the list was reused, and rebuilt more than at the remap


def test_stale_list_misses_pairs():
    """Without rebuilds the list loses pairs (the rebuild rule is what keeps it exact)."""
    w, traj = _trajectory(80, 0.1)
    vl = OV.SkinList(w.rc, 0.05, w.A)
    lat0 = oracle.lattice(w.A, w.L0, w.T, w.t)
    vl.build(lat0["L"], lat0["Linv"], w.q, w.t)
    differs = False
    for _, q, _, t, _ in traj:
        ref, lat = _brute_keys(w, q, t)
        got = oracle.canonical_pair_keys(vl.pairs_at(lat["L"], lat["Linv"], q))
        differs |= not np.array_equal(got, ref)
    assert differs


def test_images_follow_the_wrap():
    """A list built from one image of the positions gives the same pairs for
    positions moved by arbitrary lattice vectors (the images are re-derived)."""
    w = W.config_flow(W.M_GENERAL, 4, 0.37, 43)
    lat = oracle.lattice(w.A, w.L0, w.T, w.t)
    vl = OV.SkinList(w.rc, 0.2, w.A)
    vl.build(lat["L"], lat["Linv"], w.q, w.t)
    rng = np.random.default_rng(5)
    shifted = w.q + rng.integers(-2, 3, size=(w.n, 3)) @ lat["L"].T
    ref, _ = _brute_keys(w, w.q, w.t)
    assert np.array_equal(oracle.canonical_pair_keys(vl.pairs_at(lat["L"], lat["Linv"], shifted)), ref)
