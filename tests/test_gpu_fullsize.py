"""Parity at the full sizes of the measured workloads, in the launch
configurations the benchmark times: the whole evaluation is compared with the
FP64 oracle's cell list (exact pair counts, every force, U and W), plus the
bit-exact pair set of the N = 256,000 general-flow system at its most skewed
state."""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, kind_of, make_ctx, mat_rel, rel, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

F_TOL = 1e-5
UW_TOL_FAST = 3e-6    # warp kernel and the batch's per-particle float32 sums (worst measured 1.4e-6)
UW_TOL_ROW = 1e-6     # row kernel (worst measured 2.5e-7, the 2^21 system's virial)
UW_TOL_PRECISE = 1e-9
WARP = (2, 32)
ROW = (4, 32)


def evaluate(ctx, w, q, variant):
    F = torch.zeros((w.n, 3), dtype=torch.float32, device="cuda")
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    Wv = torch.zeros(9, dtype=torch.float64, device="cuda")
    ctx.set_state(q, w.t)
    ctx.build_cells(variant, w.rc)
    ctx.compute_forces(F, U, Wv)
    ctx.sync()
    return F.cpu().numpy().astype(np.float64), float(U.item()), Wv.cpu().numpy().reshape(3, 3), ctx.stats()


def check(F, U, Wm, st, ref, uw_tol=UW_TOL_FAST):
    assert st["pairs"] == ref.npairs
    assert force_err(F, ref.F) <= F_TOL
    assert rel(U, ref.U) <= uw_tol
    assert mat_rel(Wm, ref.W) <= uw_tol


@pytest.mark.parametrize("t", [0.37, W.NEAR_REMAP_T])
def test_general_n1m_bench_configuration(t):
    """N = 1,048,576 general flow: warp and row kernels, per-step variant by the volume rule."""
    ser = W.general_series(k=64)
    w = ser.workload(t)
    ref = oracle.evaluate(w, "ds")
    ctx = make_ctx(w, nemd, torch)
    q = torch.from_numpy(w.q).cuda()
    for kern in (2, 4):
        ctx.set_option(nemd.NEMD_OPT_KERNEL, kern)
        check(*evaluate(ctx, w, q, nemd.NEMD_AUTO_HEURISTIC), ref, UW_TOL_ROW if kern == 4 else UW_TOL_FAST)
    # the row kernel's precise mode (float-float energy and virial): 1e-9
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 1)
    check(*evaluate(ctx, w, q, nemd.NEMD_AUTO_HEURISTIC), ref, UW_TOL_PRECISE)
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 0)
    # the plain fixed-variant cell lists on the same state
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 0)
    for variant in (nemd.NEMD_DS, nemd.NEMD_DO):
        check(*evaluate(ctx, w, q, variant), ref)
    ctx.close()


def test_general_n2m_cell_factors():
    """N = 2^21 general flow (the learned selector's system) at both cell factors."""
    ser = W.general_series_2m()
    w = ser.workload(0.61 * ser.period)
    ref = oracle.evaluate(w, "ds")
    ctx = make_ctx(w, nemd, torch)
    q = torch.from_numpy(w.q).cuda()
    for kern in (2, 4):
        ctx.set_option(nemd.NEMD_OPT_KERNEL, kern)
        for kfac in (1, 2):
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, kfac)
            for variant in (nemd.NEMD_DS, nemd.NEMD_DO):
                F, U, Wm, st = evaluate(ctx, w, q, variant)
                assert st["cell_factor"] == kfac
                check(F, U, Wm, st, ref, UW_TOL_ROW if kern == 4 else UW_TOL_FAST)
    # precise mode on the row kernel, both cell lists: energy and virial to 1e-9
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
    ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 1)
    for variant in (nemd.NEMD_DS, nemd.NEMD_DO):
        check(*evaluate(ctx, w, q, variant), ref, UW_TOL_PRECISE)
    ctx.close()


def test_batched_256_systems():
    """The 256-system batch as the benchmark runs it (autotuned graph replay)."""
    ws = W.batched_systems()
    specs = [{"A": w.A, "L0": w.L0, "M": w.M, "T": w.T, "rc": w.rc, "n": w.n, "kind": kind_of(w),
              "variant": nemd.NEMD_AUTO_HEURISTIC} for w in ws]
    b = nemd.Batch(specs)
    q = torch.from_numpy(np.concatenate([w.q for w in ws])).cuda()
    b.set_state(q, [w.t for w in ws])
    b.autotune(reps=1)
    F = torch.zeros((b.ntot, 3), dtype=torch.float32, device="cuda")
    UW = torch.zeros((b.nsys, 10), dtype=torch.float64, device="cuda")
    b.compute(F, UW)
    b.sync()
    F = F.cpu().numpy().astype(np.float64)
    UW = UW.cpu().numpy()
    st, _ = b.stats()
    for s, w in enumerate(ws):
        ref = oracle.evaluate(w, "ds")
        lo, hi = b.offsets[s], b.offsets[s + 1]
        assert st[s]["pairs"] == ref.npairs, s
        assert force_err(F[lo:hi], ref.F) <= F_TOL, s
        assert rel(UW[s, 0], ref.U) <= UW_TOL_FAST, s
        assert mat_rel(UW[s, 1:].reshape(3, 3), ref.W) <= UW_TOL_FAST, s
    b.close()


def test_general_n256k_pair_set_at_max_skew():
    """Bit-exact (i, j, n) pair set of the N = 256,000 system just before the remap."""
    w = W.config_general(t=W.NEAR_REMAP_T, k=40)
    ref = oracle.evaluate(w, "ds", want_pairs=True)
    for variant in (0, 1):
        for kern in (WARP, ROW):
            g = run(w, variant, record=True, kernel=kern)
            assert g["stats"]["pairs"] == ref.npairs
            assert np.array_equal(oracle.canonical_pair_keys(g["pairs"]), oracle.canonical_pair_keys(ref.pairs))
            assert force_err(g["F"], ref.F) <= F_TOL
