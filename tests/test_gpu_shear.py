"""Lees-Edwards shear (Sec. 2.2) remapped half way through the period
(NEMD_OPT_REMAP = 1): the device lattice against the oracle, and pair sets,
forces, energy and virial of every kernel against the FP64 oracle across the
period, including the remap instant; a batch mixing shear and KR systems."""
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

KERNELS = [(0, 16), (2, 32), (3, 32), (4, 32)]
STRAINS = [0.0, 0.23, 0.4999999, 0.5, 0.77]


def test_lattice_centred_matches_oracle():
    ser = W.shear_series(k=8, rate=0.7)
    w = ser.workload(0.0)
    ctx = make_ctx(w, nemd, torch)
    for f in STRAINS + [1.31, -0.4]:
        t = f * ser.period
        q = torch.from_numpy(ser.positions(t)).cuda()
        ctx.set_state(q, t)
        lat = ctx.lattice()
        ref = oracle.lattice(ser.A, ser.L0, ser.period, t, centered=True)
        assert np.abs(lat["L"] - ref["L"]).max() <= 1e-13 * np.abs(ref["L"]).max()
        assert abs(ref["L"][0, 1] / ref["L"][1, 1]) <= 0.5 + 1e-12
    ctx.close()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("variant", [0, 1])
def test_shear_parity_across_the_period(variant, kernel):
    ser = W.shear_series(k=10, seed=8)          # N = 4000
    for f in STRAINS:
        w = ser.workload(f * ser.period)
        ref = oracle.evaluate(w, "ds", want_pairs=True)
        g = run(w, variant, record=True, kernel=kernel)
        assert g["stats"]["pairs"] == ref.npairs
        assert np.array_equal(oracle.canonical_pair_keys(g["pairs"]), oracle.canonical_pair_keys(ref.pairs))
        g = run(w, variant, kernel=kernel)
        assert g["stats"]["pairs"] == ref.npairs
        assert force_err(g["F"], ref.F) <= 1e-5
        assert rel(g["U"], ref.U) <= 3e-6 and mat_rel(g["W"], ref.W) <= 3e-6


def test_shear_full_size_config():
    """N = 32000 LJ under shear at the remap instant and half way between."""
    ser = W.shear_series(k=20)
    for f in (0.25, 0.5):
        w = ser.workload(f * ser.period)
        ref = oracle.evaluate(w, "ds")
        for variant in (0, 1):
            g = run(w, variant, kernel=(2, 32))
            assert g["stats"]["pairs"] == ref.npairs
            assert force_err(g["F"], ref.F) <= 1e-5
            assert rel(g["U"], ref.U) <= 3e-6


def test_batch_with_shear_systems():
    shear = [W.shear_series(k=k, seed=20 + k, rate=0.5 + 0.1 * k).workload(0.37 * k) for k in (6, 7, 8)]
    kr = W.batched_systems(nsys=3, seed=31, nmin=500, nmax=3000)
    ws = [shear[0], kr[0], shear[1], kr[1], shear[2], kr[2]]
    specs = [{"A": w.A, "L0": w.L0, "M": w.M, "T": w.T, "rc": w.rc, "n": w.n, "kind": kind_of(w),
              "variant": nemd.NEMD_AUTO_HEURISTIC, "remap": w.remap} for w in ws]
    b = nemd.Batch(specs)
    F = torch.zeros((b.ntot, 3), dtype=torch.float32, device="cuda")
    UW = torch.zeros((b.nsys, 10), dtype=torch.float64, device="cuda")
    b.set_state(torch.from_numpy(np.concatenate([w.q for w in ws])).cuda(), [w.t for w in ws])
    b.compute(F, UW)
    b.sync()
    F = F.cpu().numpy().astype(np.float64)
    UW = UW.cpu().numpy()
    st, _ = b.stats()
    for s, w in enumerate(ws):
        ref = oracle.evaluate(w, "ds")
        assert st[s]["pairs"] == ref.npairs
        assert force_err(F[b.offsets[s]:b.offsets[s + 1]], ref.F) <= 1e-5
        assert rel(UW[s, 0], ref.U) <= 3e-6
    b.close()
