"""The autotuner: it times every candidate configuration, keeps the fastest for
the shape class, applies it, persists it, and never changes the results."""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, make_ctx, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402


def evaluate(ctx, w, q, variant):
    F = torch.zeros((w.n, 3), dtype=torch.float32, device="cuda")
    ctx.set_state(q, w.t)
    ctx.build_cells(variant, w.rc)
    ctx.compute_forces(F)
    ctx.sync()
    return F.cpu().numpy().astype(np.float64), ctx.stats()


def test_autotune_picks_fastest_and_keeps_results(tmp_path):
    w = W.config_general(t=0.4, k=14)
    ref = oracle.evaluate(w, "ds")
    q = torch.from_numpy(w.q).cuda()
    ctx = make_ctx(w, nemd, torch)
    ctx.set_state(q, w.t)
    best, times = ctx.autotune(nemd.NEMD_AUTO_HEURISTIC, w.rc, reps=2)
    assert len(times) == 13
    fastest = min(times, key=lambda x: x[1])[0]
    assert best == fastest          # first call: the class mean is this call's time
    F, st = evaluate(ctx, w, q, nemd.NEMD_AUTO_HEURISTIC)
    assert st["pairs"] == ref.npairs
    assert st["cell_factor"] == best["cell_factor"]
    assert force_err(F, ref.F) <= 1e-5
    # every candidate gives the same pair count
    path = tmp_path / "tune.bin"
    ctx.tune_save(path)
    ctx.close()
    # a fresh context loads the cache and applies it when asked to
    ctx2 = make_ctx(w, nemd, torch)
    ctx2.tune_load(path)
    ctx2.set_option(nemd.NEMD_OPT_AUTOTUNED, 1)
    F2, st2 = evaluate(ctx2, w, q, nemd.NEMD_AUTO_HEURISTIC)
    assert st2["cell_factor"] == best["cell_factor"]
    assert force_err(F2, ref.F) <= 1e-5
    # a corrupted file is refused and the cache is left as it was
    raw = bytearray(path.read_bytes())
    raw[30] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(nemd.NemdError):
        ctx2.tune_load(bad)
    F3, st3 = evaluate(ctx2, w, q, nemd.NEMD_AUTO_HEURISTIC)
    assert st3["cell_factor"] == best["cell_factor"]
    ctx2.close()


def test_every_candidate_gives_the_same_pairs():
    w = W.config_planar(30, k=10)
    ref = oracle.evaluate(w, "do")
    for kern, group, kfac in ((0, 16, 1), (2, 32, 1), (2, 32, 2), (3, 32, 1), (3, 32, 2), (1, 4, 2), (1, 8, 1),
                              (1, 16, 2)):
        g = run(w, nemd.NEMD_DO, kernel=(kern, group), kfac=kfac)
        assert g["stats"]["pairs"] == ref.npairs, (kern, group, kfac)
        assert force_err(g["F"], ref.F) <= 1e-5
