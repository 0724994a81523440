"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  pair sets            bit-exact (i, j, n) against the oracle
  forces               max|dF| / max|F| <= 1e-5   (float32 pair arithmetic)
  energy, virial       rel <= 1e-9 in precise mode (accepted pairs in float64
                       or float-float, summed in float64 / float-float);
                       fast mode (float32 pair terms summed per particle in
                       float32, float64 across particles): the error is a few
                       float32 roundings per pair term times the sum's
                       condition number (sum of |terms| over |sum|), not a
                       function of N.  Row kernel (the pair sums without the
                       potential's constant factors, applied once per
                       particle in float64) <= 1e-6: worst measured 2.5e-7
                       (virial of the 2^21-particle system at t = 0.61 T),
                       7.9e-7 for F.  The other kernels (constant factors in
                       every float32 pair term) <= 3e-6: worst measured 1.4e-6
                       on the same system, 2.8e-7 on the smaller systems of
                       this file
  lattice              |L_gpu - L_oracle| <= 1e-13 |L|
"""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, mat_rel, rel, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DS, DO = 0, 1
F_TOL = 1e-5
UW_TOL_PRECISE = 1e-9
UW_TOL_FAST = 3e-6
UW_TOL_ROW = 1e-6


def keys(p):
    return oracle.canonical_pair_keys(p)


KERNELS = [(0, 16), (2, 32), (3, 32), (1, 16), (1, 4), (4, 32)]   # (kernel, group): plain, warp, warp-half,
#                                                                   grouped, row
DETERMINISTIC = [(0, 16), (2, 32), (4, 32)]          # kernels whose forces repeat bit for bit
MAIN = [(0, 16), (2, 32), (3, 32), (4, 32)]          # plain, warp, warp-half, row


def check_against(w, variant, ref, *, pairs=True, precise=True, kfac=1, kernel=(0, 16)):
    if pairs:
        g = run(w, variant, record=True, kfac=kfac, kernel=kernel)
        assert g["stats"]["pairs"] == ref.npairs
        assert np.array_equal(keys(g["pairs"]), keys(ref.pairs)), "pair sets differ"
    g = run(w, variant, kfac=kfac, kernel=kernel)
    assert g["stats"]["pairs"] == ref.npairs
    assert force_err(g["F"], ref.F) <= F_TOL
    uw = UW_TOL_ROW if kernel[0] == 4 else UW_TOL_FAST
    assert rel(g["U"], ref.U) <= uw
    assert mat_rel(g["W"], ref.W) <= uw
    if precise:
        gp = run(w, variant, precise=True, kfac=kfac, kernel=kernel)
        assert gp["stats"]["pairs"] == ref.npairs
        assert rel(gp["U"], ref.U) <= UW_TOL_PRECISE
        assert mat_rel(gp["W"], ref.W) <= UW_TOL_PRECISE
        assert force_err(gp["F"], ref.F) <= 1e-6
    return g


# ---------------------------------------------------------------- lattice ----

@pytest.mark.parametrize("M", [W.M_PLANAR, W.M_GENERAL])
def test_lattice_matches_oracle(M):
    for t in (0.0, 0.25, 0.6180339, W.NEAR_REMAP_T, 3.75):
        w = W.config_flow(M, 6, t, seed=9)
        g = run(w, DS)
        lat = g["lattice"]
        ref = oracle.lattice(w.A, w.L0, w.T, w.t)
        scale = np.abs(ref["L"]).max()
        assert np.abs(lat["L"] - ref["L"]).max() <= 1e-13 * scale
        assert np.abs(lat["Linv"] - ref["Linv"]).max() <= 1e-12 * np.abs(ref["Linv"]).max()
        assert np.allclose(lat["h"], ref["h"], rtol=1e-13)
        assert np.allclose(lat["R"], ref["R"], rtol=0, atol=1e-12 * scale)
        assert abs(lat["V"] - ref["V"]) <= 1e-12 * ref["V"]
        assert np.array_equal(lat["counts"], oracle.ds_counts(ref["L"], w.rc))
        g2 = run(w, DO)
        assert np.array_equal(g2["lattice"]["counts"], oracle.do_counts(ref["R"], w.rc))


# ------------------------------------------------------------- config 0 ----

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("variant", [DS, DO])
def test_config0_wca_equilibrium(variant, kernel):
    w = W.config_equilibrium_wca()
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    check_against(w, variant, ref, kernel=kernel)


# ------------------------------------------------------ flows at strains ----

@pytest.mark.parametrize("kernel", MAIN)
@pytest.mark.parametrize("i", [0, 17, 40, 63])
@pytest.mark.parametrize("variant", [DS, DO])
def test_planar_flow_strains(i, variant, kernel):
    w = W.config_planar(i, k=12)   # 6912 particles, several tiles and a ragged tail
    ref = oracle.evaluate(w, "do" if variant else "ds", want_pairs=True)
    check_against(w, variant, ref, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("t", [0.3, 0.71, W.NEAR_REMAP_T])
@pytest.mark.parametrize("variant", [DS, DO])
def test_general_flow_incl_max_skew(t, variant, kernel):
    w = W.config_general(t=t, k=11)   # 5324 particles
    ref = oracle.evaluate(w, "ds", want_pairs=True)
    check_against(w, variant, ref, kernel=kernel)


@pytest.mark.parametrize("kernel", MAIN)
@pytest.mark.parametrize("variant", [DS, DO])
def test_planar_config_full_size(variant, kernel):
    """The planar-flow configuration at its full size (N = 32000) at two strains."""
    for i in (9, 50):
        w = W.config_planar(i)
        ref = oracle.evaluate(w, "ds", want_pairs=True)
        check_against(w, variant, ref, precise=(i == 9), kernel=kernel)


# ------------------------------------------------------- tiny / ragged ----

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("kfac", [1, 2])
def test_tiny_skewed_boxes(seed, kfac, kernel):
    """Boxes with 1-3 cells per direction: multiple images of one partner."""
    rng = np.random.default_rng(500 + seed)
    rc = 1.3
    L, q = W.small_random_box(rng, 37 + 11 * seed, rc, 1.0, 3.2)
    w = W.Workload(name="tiny", A=np.zeros((3, 3)), L0=L, M=W.M_IDENTITY.copy(), T=1.0, t=0.0,
                   q=q, kind=W.POT_LJ, rc=rc)
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    for variant in (DS, DO):
        check_against(w, variant, ref, kfac=kfac, kernel=kernel)


def test_edge_cases_small_n():
    L = 9.0 * np.eye(3)
    base = dict(A=np.zeros((3, 3)), L0=L, M=W.M_IDENTITY.copy(), T=1.0, t=0.0, kind=W.POT_LJ, rc=2.5)
    # N = 0
    w0 = W.Workload(name="empty", q=np.zeros((0, 3)), **base)
    g = run(w0, DS)
    assert g["stats"]["pairs"] == 0 and g["U"] == 0.0 and np.all(g["W"] == 0)
    # N = 1: no pair, not even with its own images (h = 9 > rc)
    w1 = W.Workload(name="one", q=np.array([[1.0, 2.0, 3.0]]), **base)
    for v in (DS, DO):
        g = run(w1, v)
        assert g["stats"]["pairs"] == 0 and np.all(g["F"] == 0)
    # N = 2 across the periodic boundary: closed form
    r = 1.2
    w2 = W.Workload(name="two", q=np.array([[0.1, 4.0, 4.0], [0.1 - r, 4.0, 4.0]]), **base)
    for v in (DS, DO):
        g = run(w2, v, precise=True)
        u = 4 * (r ** -12 - r ** -6) - 4 * (2.5 ** -12 - 2.5 ** -6)
        assert g["stats"]["pairs"] == 1
        assert abs(g["U"] - u) < 1e-12
        du = -48 * r ** -13 + 24 * r ** -7
        assert abs(g["F"][0, 0] - (-du)) < 1e-5 * abs(du)


def face_positions(L, rc, faces, rng, interior=True):
    """Particles on the half-cell grid of one variant's cells (every interior
    face and centre; cell factor 1) with 30 % vacancies, each coordinate moved by 0, +-1 or +-2 units in the
    last place or +-2^-44 of the box: binning decisions at and a rounding either
    side of every face."""
    if faces == "ds":
        c = oracle.ds_counts(L, rc)
        axes = [np.arange(2 * c[a]) / (2.0 * c[a]) for a in range(3)]
        s = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
        q = s @ L.T
    else:
        Q, R = oracle.qr(L)
        l = oracle.do_counts(R, rc)
        axes = [np.arange(2 * l[a]) * (R[a, a] / (2.0 * l[a])) for a in range(3)]
        b = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
        q = b @ Q.T       # L s = Q R s = Q b
    # Interior faces only: a particle within a rounding of the unit cell's own
    # boundary (s = 0 or 1) is wrapped by L(t), which each side computes to
    # ~1e-15 relative on its own, so its canonical image (the n of its pairs)
    # may legitimately differ by a lattice vector between the two.
    sr = q @ np.linalg.inv(L).T
    keep = rng.random(len(q)) < 0.7
    if interior:
        keep &= np.abs(sr - np.rint(sr)).min(axis=1) > 1e-9
    q = q[keep]                          # (and vacancies: no symmetric cancellation of forces)
    ulp = np.spacing(np.abs(q) + 1e-300)
    kick = rng.choice(np.array([0.0, 1.0, -1.0, 2.0, -2.0]), size=q.shape) * ulp
    tiny = rng.choice(np.array([0.0, 1.0, -1.0]), size=q.shape) * (2.0 ** -44) * np.abs(L).max()
    use_tiny = rng.random(q.shape) < 0.3
    return np.ascontiguousarray(q + np.where(use_tiny, tiny, kick))


@pytest.mark.parametrize("kernel", DETERMINISTIC)
@pytest.mark.parametrize("faces", ["ds", "do"])
@pytest.mark.parametrize("frac", [0.0, 0.37, 0.999])
def test_particles_on_cell_and_brick_faces(frac, faces, kernel):
    """Particles on the faces of the dynamic size cells or the dynamic offset
    bricks of a general-flow box at three strains; both variants, both cell
    factors: exact pair set, forces, energy and virial against brute force."""
    rng = np.random.default_rng(int(frac * 1000) + (17 if faces == "ds" else 71))
    ser = W.general_series(k=10, seed=9)
    t = frac * ser.period
    L = oracle.lattice(ser.A, ser.L0, ser.period, t)["L"]
    q = face_positions(L, ser.rc, faces, rng)
    w = W.Workload(name="faces", A=ser.A, L0=ser.L0, M=ser.M, T=ser.period, t=t, q=q, kind=W.POT_LJ, rc=ser.rc)
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    assert ref.npairs > 0
    for kfac in (1, 2):
        for v in (DS, DO):
            check_against(w, v, ref, kfac=kfac, kernel=kernel, precise=(kfac == 1))


@pytest.mark.parametrize("faces", ["ds", "do"])
@pytest.mark.parametrize("frac", [0.0, 0.37])
def test_particles_on_unit_cell_faces(frac, faces):
    """The same grids including the unit cell's own faces (s = 0 = 1, a few
    units in the last place either side): the binning takes its float64 path
    there.  Which image of such a particle is canonical depends on the last
    bits of L(t), which the two sides compute independently, so the pair
    images n may differ by lattice vectors; everything else is unique: the
    (i, j) multiset, forces, energy and virial."""
    rng = np.random.default_rng(int(frac * 1000) + (19 if faces == "ds" else 73))
    ser = W.general_series(k=10, seed=9)
    t = frac * ser.period
    L = oracle.lattice(ser.A, ser.L0, ser.period, t)["L"]
    q = face_positions(L, ser.rc, faces, rng, interior=False)
    w = W.Workload(name="faces", A=ser.A, L0=ser.L0, M=ser.M, T=ser.period, t=t, q=q, kind=W.POT_LJ, rc=ser.rc)
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    ij_ref = np.sort(ref.pairs[:, 0].astype(np.int64) * w.n + ref.pairs[:, 1])
    for kfac in (1, 2):
        for v in (DS, DO):
            for kernel in DETERMINISTIC:
                g = run(w, v, record=True, kfac=kfac, kernel=kernel)
                assert g["stats"]["pairs"] == ref.npairs
                ij = np.sort(g["pairs"][:, 0].astype(np.int64) * w.n + g["pairs"][:, 1])
                assert np.array_equal(ij, ij_ref)
                g = run(w, v, kfac=kfac, kernel=kernel)
                assert force_err(g["F"], ref.F) <= F_TOL
                assert rel(g["U"], ref.U) <= UW_TOL_FAST and mat_rel(g["W"], ref.W) <= UW_TOL_FAST


@pytest.mark.parametrize("kernel", KERNELS)
def test_ragged_counts_and_empty_cells(kernel):
    """A dilute random system: many empty cells, uneven occupancy."""
    w = W.uniform_random(777, 30.0 * np.eye(3), seed=3)
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    for v in (DS, DO):
        check_against(w, v, ref, kernel=kernel)


@pytest.mark.parametrize("kernel", MAIN)
def test_crowded_cells(kernel):
    """A strained general-flow system with 200 of its particles packed into a
    cube of side 3 (local density ~7): cells of 40 to 200 particles, well past
    the 32 of a warp, beside cells of ordinary occupancy."""
    w = W.config_general(t=0.3, k=8)
    rng = np.random.default_rng(41)
    q = w.q.copy()
    q[:200] = q[500] + 3.0 * rng.random((200, 3))
    w = W.Workload(name="crowded", A=w.A, L0=w.L0, M=w.M, T=w.T, t=w.t, q=q, kind=w.kind, rc=w.rc)
    ref = oracle.evaluate(w, "brute", want_pairs=True)
    for v in (DS, DO):
        g = check_against(w, v, ref, kernel=kernel)
        assert g["stats"]["pairs"] == ref.npairs


# ------------------------------------------------------------ properties ----

@pytest.mark.parametrize("kernel", DETERMINISTIC)
def test_deterministic_repeat(kernel):
    w = W.config_planar(23, k=10)
    a = run(w, DO, kernel=kernel)
    b = run(w, DO, kernel=kernel)
    assert np.array_equal(a["F"], b["F"]) and a["U"] == b["U"]


def test_kernels_agree_bitwise_on_forces():
    """Same pair arithmetic and per-particle summation order in both kernels."""
    w = W.config_general(t=0.55, k=12)
    a = run(w, DO, kernel=(0, 16))
    for kern in ((1, 16), (2, 32), (3, 32)):
        b = run(w, DO, kernel=kern)
        assert a["stats"]["pairs"] == b["stats"]["pairs"]
        assert force_err(b["F"], a["F"]) <= 1e-6


def test_variants_agree_and_newton():
    w = W.config_general(t=0.45, k=12)
    a = run(w, DS)
    b = run(w, DO)
    assert a["stats"]["pairs"] == b["stats"]["pairs"]
    assert force_err(a["F"], b["F"]) <= 2 * F_TOL
    assert np.abs(a["F"].sum(0)).max() <= 1e-5 * np.abs(a["F"]).max() * np.sqrt(w.n)


def test_host_pointers_match_device():
    from paper_1412_3784_gb300 import nemd
    from gpu_util import make_ctx
    w = W.config_planar(5, k=8)
    g = run(w, DS)
    ctx = make_ctx(w, nemd, torch)
    F = np.zeros((w.n, 3), dtype=np.float32)
    U = np.zeros(1)
    Wv = np.zeros(9)
    ctx.set_state(np.ascontiguousarray(w.q), w.t)
    ctx.build_cells(DS, w.rc)
    ctx.compute_forces(F, U, Wv)
    assert np.array_equal(F.astype(np.float64), g["F"])
    assert U[0] == g["U"]
    ctx.close()


def test_auto_heuristic_picks_smaller_volume():
    from paper_1412_3784_gb300 import nemd
    for t in (0.0, 0.5, W.NEAR_REMAP_T):
        w = W.config_general(t=t, k=10)
        g = run(w, nemd.NEMD_AUTO_HEURISTIC)
        ref = oracle.evaluate(w, "ds")
        assert g["stats"]["pairs"] == ref.npairs
        lat = oracle.lattice(w.A, w.L0, w.T, w.t)
        c = oracle.ds_counts(lat["L"], w.rc)
        l = oracle.do_counts(lat["R"], w.rc)
        vds = 27 * lat["V"] / np.prod(c)
        avg = 27 + 14 / l[2] + 6 / l[1] - 4 / (l[1] * l[2])
        vdo = avg * lat["V"] / np.prod(l)
        assert g["stats"]["variant"] == (1 if vdo < vds else 0)


def test_do_stencil_size_matches_oracle():
    for t in (0.0, 0.37, W.NEAR_REMAP_T):
        w = W.config_general(t=t, k=10)
        g = run(w, DO)
        lat = oracle.lattice(w.A, w.L0, w.T, w.t)
        assert g["stats"]["stencil_cells"] == oracle.do_total_stencil_cells(lat["R"], w.rc)
        d = run(w, DS)
        c = oracle.ds_counts(lat["L"], w.rc)
        assert d["stats"]["stencil_cells"] == 27 * int(np.prod(c))


def test_async_host_io_matches_sync():
    """NEMD_OPT_ASYNC_HOST: host positions in, host F, U, W out over several
    states without synchronising, then one nemd_sync -- bitwise the results of
    the synchronising path."""
    from paper_1412_3784_gb300 import nemd
    from gpu_util import make_ctx
    states = [W.config_planar(i) for i in (3, 20, 41, 58)]
    ref = [run(w, DO, kernel=(2, 32)) for w in states]
    ctx = make_ctx(states[0], nemd, torch)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 2)
    ctx.set_option(nemd.NEMD_OPT_ASYNC_HOST, 1)
    qs = [torch.from_numpy(w.q).pin_memory() for w in states]
    Fs = [torch.empty((w.n, 3), dtype=torch.float32).pin_memory() for w in states]
    Us = [np.zeros(1) for _ in states]
    Ws = [np.zeros(9) for _ in states]
    for w, q, F, U, Wv in zip(states, qs, Fs, Us, Ws):
        ctx.set_state(q, w.t)
        ctx.build_cells(DO, w.rc)
        ctx.compute_forces(F, U, Wv)
    ctx.sync()
    for r, F, U, Wv in zip(ref, Fs, Us, Ws):
        assert np.array_equal(F.numpy().astype(np.float64), r["F"])
        assert U[0] == r["U"] and np.array_equal(Wv.reshape(3, 3), r["W"])
    ctx.close()
