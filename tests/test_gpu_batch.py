"""Batches of independent systems (nemd_batch_*): every system's results equal
those of a context running the same system alone with the same force kernel,
and the FP64 oracle's; graph replay, eager launches, options, host pointers,
per-system errors and two batches in flight on two streams."""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, kind_of, mat_rel, rel, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

VARIANTS = (nemd.NEMD_DS, nemd.NEMD_DO, nemd.NEMD_AUTO_HEURISTIC)


def spec(w, variant):
    return {"A": w.A, "L0": w.L0, "M": w.M, "T": w.T, "rc": w.rc, "n": w.n, "kind": kind_of(w),
            "eps": w.eps, "sigma": w.sigma, "shift": w.shift, "variant": variant}


def systems(nsys=9, seed=21, nmin=300, nmax=3000):
    ws = W.batched_systems(nsys=nsys, seed=seed, nmin=nmin, nmax=nmax)
    return ws, [VARIANTS[i % 3] for i in range(len(ws))]


def evaluate(b, ws, ts=None, q=None):
    if q is None:
        q = torch.from_numpy(np.concatenate([w.q for w in ws])).cuda()
    F = torch.zeros((b.ntot, 3), dtype=torch.float32, device="cuda")
    UW = torch.zeros((b.nsys, 10), dtype=torch.float64, device="cuda")
    b.set_state(q, [w.t for w in ws] if ts is None else ts)
    b.compute(F, UW)
    b.sync()
    return F.cpu().numpy().astype(np.float64), UW.cpu().numpy()


def test_batch_equals_single_contexts_and_oracle():
    ws, vs = systems()
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    F, UW = evaluate(b, ws)
    st, launches = b.stats()
    assert launches == 11
    for s, (w, v) in enumerate(zip(ws, vs)):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        one = run(w, v, kernel=(4, 32))
        # the batch's default force kernel (the row kernel) on the system alone
        assert st[s]["pairs"] == one["stats"]["pairs"], s
        assert st[s]["variant"] == one["stats"]["variant"]
        assert force_err(F[lo:hi], one["F"]) <= 1e-6, s
        assert rel(UW[s, 0], one["U"]) <= 1e-6
        assert mat_rel(UW[s, 1:].reshape(3, 3), one["W"]) <= 1e-6
        ref = oracle.evaluate(w, "ds")
        assert st[s]["pairs"] == ref.npairs
        assert force_err(F[lo:hi], ref.F) <= 1e-5, s
        assert rel(UW[s, 0], ref.U) <= 3e-6
        assert mat_rel(UW[s, 1:].reshape(3, 3), ref.W) <= 3e-6
        assert st[s]["status"] == 0
    b.close()


def test_replay_is_deterministic_and_equals_eager():
    ws, vs = systems(nsys=6, seed=22)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    F1, U1 = evaluate(b, ws)
    F2, U2 = evaluate(b, ws)
    assert np.array_equal(F1, F2) and np.array_equal(U1, U2)
    b.set_option(nemd.NEMD_BATCH_OPT_GRAPH, 0)
    F3, U3 = evaluate(b, ws)
    assert np.array_equal(F1, F3) and np.array_equal(U1, U3)
    b.close()


def test_strains_advance_each_system():
    """New times every step (the graph reads them from device memory)."""
    ws, vs = systems(nsys=5, seed=23)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    rng = np.random.default_rng(0)
    for _ in range(3):
        ts = [float(rng.uniform(0, w.T)) for w in ws]
        moved = [W.Workload(name=w.name, A=w.A, L0=w.L0, M=w.M, T=w.T, t=t, q=w.q, kind=w.kind, rc=w.rc)
                 for w, t in zip(ws, ts)]
        F, UW = evaluate(b, moved, ts=ts)
        st, _ = b.stats()
        for s, w in enumerate(moved):
            ref = oracle.evaluate(w, "ds")
            lo, hi = b.offsets[s], b.offsets[s + 1]
            assert st[s]["pairs"] == ref.npairs
            assert force_err(F[lo:hi], ref.F) <= 1e-5
            assert rel(UW[s, 0], ref.U) <= 3e-6
    b.close()


def test_two_batches_in_flight_on_two_streams():
    """Two batches of the same systems, each on its own CUDA stream, take the
    steps (new strains every step) in turn with no synchronisation between
    them (the form the bench times): every step's F and U, W equal those of
    one batch running the steps one after another."""
    ws, vs = systems(nsys=7, seed=27)
    specs = [spec(w, v) for w, v in zip(ws, vs)]
    q = torch.from_numpy(np.concatenate([w.q for w in ws])).cuda()
    rng = np.random.default_rng(1)
    steps = [[float(rng.uniform(0, w.T)) for w in ws] for _ in range(6)]

    one = nemd.Batch(specs)
    ref = []
    for ts in steps:
        F = torch.zeros((one.ntot, 3), dtype=torch.float32, device="cuda")
        UW = torch.zeros((one.nsys, 10), dtype=torch.float64, device="cuda")
        one.set_state(q, ts)
        one.compute(F, UW)
        one.sync()
        ref.append((F.cpu().numpy(), UW.cpu().numpy(), [x["pairs"] for x in one.stats()[0]]))
    one.close()

    streams = [torch.cuda.Stream() for _ in range(2)]
    bs = [nemd.Batch(specs, stream=st.cuda_stream) for st in streams]
    outs = [(torch.zeros((bs[0].ntot, 3), dtype=torch.float32, device="cuda"),
             torch.zeros((bs[0].nsys, 10), dtype=torch.float64, device="cuda")) for _ in steps]
    for i, ts in enumerate(steps):
        bs[i % 2].set_state(q, ts)
        bs[i % 2].compute(*outs[i])
    for b in bs:
        b.sync()
    torch.cuda.synchronize()
    for i, (F, UW) in enumerate(outs):
        assert np.array_equal(F.cpu().numpy(), ref[i][0]), i
        assert np.array_equal(UW.cpu().numpy(), ref[i][1]), i
    for k, b in enumerate(bs):
        assert [x["pairs"] for x in b.stats()[0]] == ref[len(steps) - 2 + k][2]
        b.close()
    # one system of the last step against the oracle
    moved = W.Workload(name=ws[0].name, A=ws[0].A, L0=ws[0].L0, M=ws[0].M, T=ws[0].T, t=steps[-1][0],
                       q=ws[0].q, kind=ws[0].kind, rc=ws[0].rc)
    o = oracle.evaluate(moved, "ds")
    assert ref[-1][2][0] == o.npairs
    assert force_err(ref[-1][0][:ws[0].n].astype(np.float64), o.F) <= 1e-5


def test_warp_kernel_option_agrees_with_row_kernel():
    """NEMD_BATCH_OPT_KERNEL = 2 (the warp kernel over the same chunk list)
    against the default row kernel: the same pairs per system, forces, U and W
    within float32 rounding of each other, and both against the oracle; the
    option changes the captured step (graph re-captured) and back."""
    ws, vs = systems(nsys=8, seed=28)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    F4, U4 = evaluate(b, ws)
    st4, l4 = b.stats()
    b.set_option(nemd.NEMD_BATCH_OPT_KERNEL, 2)
    F2, U2 = evaluate(b, ws)
    st2, l2 = b.stats()
    b.set_option(nemd.NEMD_BATCH_OPT_KERNEL, 4)
    F4b, U4b = evaluate(b, ws)
    assert l4 == l2 == 11
    assert np.array_equal(F4, F4b) and np.array_equal(U4, U4b)
    for s, w in enumerate(ws):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        ref = oracle.evaluate(w, "ds")
        assert st4[s]["pairs"] == st2[s]["pairs"] == ref.npairs, s
        # each within its own bar of the oracle (row 1e-6, warp 3e-6)
        assert force_err(F4[lo:hi], F2[lo:hi]) <= 3e-6, s
        assert rel(U4[s, 0], U2[s, 0]) <= 4e-6
        assert mat_rel(U4[s, 1:].reshape(3, 3), U2[s, 1:].reshape(3, 3)) <= 4e-6
        assert force_err(F2[lo:hi], ref.F) <= 1e-5, s
        assert rel(U2[s, 0], ref.U) <= 3e-6
    with pytest.raises(nemd.NemdError):
        b.set_option(nemd.NEMD_BATCH_OPT_KERNEL, 3)
    b.close()


@pytest.mark.parametrize("kfac,tile", [(2, 32), (1, 16), (2, 16)])
def test_cell_factor_and_tile_keep_results(kfac, tile):
    ws, vs = systems(nsys=6, seed=24)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    b.set_option(nemd.NEMD_BATCH_OPT_CELL_FACTOR, kfac)
    b.set_option(nemd.NEMD_BATCH_OPT_TILE, tile)
    F, UW = evaluate(b, ws)
    st, _ = b.stats()
    for s, w in enumerate(ws):
        ref = oracle.evaluate(w, "ds")
        lo, hi = b.offsets[s], b.offsets[s + 1]
        assert st[s]["pairs"] == ref.npairs and st[s]["cell_factor"] == kfac
        assert force_err(F[lo:hi], ref.F) <= 1e-5
        assert rel(UW[s, 0], ref.U) <= 3e-6
    b.close()


def test_autotune_picks_a_candidate_and_keeps_results():
    ws, vs = systems(nsys=6, seed=25)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    q = torch.from_numpy(np.concatenate([w.q for w in ws])).cuda()
    b.set_state(q, [w.t for w in ws])
    times = b.autotune(reps=2)
    assert len(times) == 4 and all(ms > 0 for _, ms in times)
    F, UW = evaluate(b, ws, q=q)
    st, _ = b.stats()
    best = min(times, key=lambda x: x[1])[0]
    assert st[0]["cell_factor"] == best["cell_factor"]
    for s, w in enumerate(ws):
        assert st[s]["pairs"] == oracle.evaluate(w, "ds").npairs
    b.close()


def test_host_pointers():
    ws, vs = systems(nsys=4, seed=26)
    b = nemd.Batch([spec(w, v) for w, v in zip(ws, vs)])
    Fd, UWd = evaluate(b, ws)
    qh = np.ascontiguousarray(np.concatenate([w.q for w in ws]))
    Fh = np.zeros((b.ntot, 3), dtype=np.float32)
    UWh = np.zeros((b.nsys, 10))
    b.set_state(qh, [w.t for w in ws])
    b.compute(Fh, UWh)
    assert np.array_equal(Fh.astype(np.float64), Fd) and np.array_equal(UWh, UWd)
    b.close()


def test_edge_systems_and_per_system_errors():
    """N = 0 and N = 1 systems; a system whose box is too small for its cut-off
    and one with a NaN position fail alone; the others are unaffected."""
    ws, vs = systems(nsys=3, seed=27)
    cube = 3.0 * np.eye(3)
    eq = dict(A=np.zeros((3, 3)), M=np.eye(3, dtype=np.int64), T=1.0, t=0.0, kind=W.POT_LJ, rc=2.5)
    empty = W.Workload(name="empty", L0=4 * cube, q=np.zeros((0, 3)), **eq)
    single = W.Workload(name="one", L0=4 * cube, q=np.array([[0.3, 0.2, 0.1]]), **eq)
    small = W.Workload(name="small", L0=0.6 * cube, q=np.random.default_rng(1).random((20, 3)), **eq)
    bad = W.Workload(name="nan", L0=4 * cube, q=np.random.default_rng(2).random((50, 3)) * 12, **eq)
    allw = [empty, ws[0], single, small, ws[1], bad, ws[2]]
    allv = [nemd.NEMD_DS, vs[0], nemd.NEMD_DO, nemd.NEMD_DS, vs[1], nemd.NEMD_DS, vs[2]]
    b = nemd.Batch([spec(w, v) for w, v in zip(allw, allv)])
    q = np.concatenate([w.q for w in allw])
    q[b.offsets[5] + 7, 1] = np.nan
    F = torch.zeros((b.ntot, 3), dtype=torch.float32, device="cuda")
    UW = torch.zeros((b.nsys, 10), dtype=torch.float64, device="cuda")
    b.set_state(torch.from_numpy(q).cuda(), [w.t for w in allw])
    b.compute(F, UW)
    status = b.sync(status=True)
    assert status[3] == 5                                 # box too small
    assert status[5] == 8                                 # non-finite position
    assert status[[0, 1, 2, 4, 6]].tolist() == [0, 0, 0, 0, 0]
    F = F.cpu().numpy().astype(np.float64)
    UW = UW.cpu().numpy()
    st, _ = b.stats()
    assert st[0]["pairs"] == 0 and st[2]["pairs"] == 0 and UW[0, 0] == 0.0 and UW[2, 0] == 0.0
    assert np.all(F[b.offsets[2]:b.offsets[3]] == 0.0)
    for s in (1, 4, 6):
        w = allw[s]
        ref = oracle.evaluate(w, "ds")
        assert st[s]["pairs"] == ref.npairs
        assert force_err(F[b.offsets[s]:b.offsets[s + 1]], ref.F) <= 1e-5
    # the next clean step clears the failed systems' status
    q[b.offsets[5] + 7, 1] = 0.5
    b.set_state(torch.from_numpy(q).cuda(), [w.t for w in allw])
    b.compute()
    status = b.sync(status=True)
    assert status[5] == 0 and status[3] == 5
    b.close()


def test_add_rejects_bad_systems():
    w = W.config_general(t=0.1, k=6)
    h = nemd._vp()
    assert nemd.nemd_batch_create(nemd.ctypes.byref(h), 0, None) == 0
    y = nemd.nemd_system()
    s = spec(w, nemd.NEMD_DS)
    y.A[:] = list(w.A.ravel())
    y.L0[:] = list(w.L0.ravel())
    M = w.M.copy()
    M[0, 0] += 1                                           # det M != 1
    y.M[:] = [int(x) for x in M.ravel()]
    y.T, y.eps, y.sigma, y.rc, y.n, y.kind, y.shift, y.variant = w.T, 1.0, 1.0, s["rc"], w.n, 0, 1, 0
    assert nemd.nemd_batch_add(h, nemd.ctypes.byref(y), None) == 2
    y.M[:] = [int(x) for x in w.M.ravel()]
    y.variant = nemd.NEMD_AUTO_LEARNED
    assert nemd.nemd_batch_add(h, nemd.ctypes.byref(y), None) == 1
    y.variant = 0
    y.kind = 1                                             # WCA with rc = 2.5
    assert nemd.nemd_batch_add(h, nemd.ctypes.byref(y), None) == 1
    y.kind = 0
    assert nemd.nemd_batch_finalize(h) == 1               # no systems yet
    assert nemd.nemd_batch_add(h, nemd.ctypes.byref(y), None) == 0
    assert nemd.nemd_batch_compute(h, None, None) == 6     # before set_state
    assert nemd.nemd_batch_finalize(h) == 0
    assert nemd.nemd_batch_add(h, nemd.ctypes.byref(y), None) == 6
    nemd.nemd_batch_destroy(h)
