"""The learned cell-list selector: its training kernels against the FP64 network
oracle, its training, its per-step device inference, and what it gains over the
paper's neighbourhood-volume rule on measured timings."""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import make_ctx

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402


def _ctx():
    ctx = nemd.Context(0)
    ctx.set_flow(np.zeros((3, 3)), 10 * np.eye(3), np.eye(3, dtype=np.int64), 1.0)
    return ctx


def test_gradient_kernels_match_fp64_oracle():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.2, size=oracle.MLP_PARAMS)
    Xn = rng.normal(size=(300, 12))
    Tn = rng.normal(size=(300, 4))
    ctx = _ctx()
    ctx.model_set_params(p.astype(np.float32), np.concatenate([np.zeros(12), np.ones(12), [0.0, 1.0]]))
    pf = p.astype(np.float32).astype(np.float64)   # the parameters the device holds
    g_gpu, loss_gpu = ctx.model_grad(Xn, Tn)
    loss, g, _ = oracle.mlp_loss_grad(pf, Xn.astype(np.float32).astype(np.float64),
                                      Tn.astype(np.float32).astype(np.float64))
    assert abs(loss_gpu - loss) <= 1e-5 * abs(loss)
    assert np.abs(g_gpu - g).max() <= 1e-4 * np.abs(g).max()
    ctx.close()


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(800, 12)).astype(np.float32)
    w = rng.normal(size=(12, 4))
    T = np.exp(0.5 * np.tanh(X @ w)).astype(np.float32)     # positive "times"
    ctx = _ctx()
    hist = ctx.model_train(X, T, steps=1500, batch=128, lr=3e-3, seed=5)
    assert hist[-50:].mean() < 0.1 * hist[:50].mean()
    Y = ctx.model_predict(X)
    _, norm = ctx.model_get_params()
    pred = np.exp(Y * norm[25] + norm[24] + X[:, 11:12])     # targets are ln(time / N), N = exp(x[11])
    assert np.mean(np.abs(np.log(pred) - np.log(T))) < 0.1
    ctx.close()


def test_device_inference_picks_argmin_of_predictions(tmp_path):
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(200, 12)).astype(np.float32)
    T = rng.uniform(0.5, 2.0, size=(200, 4)).astype(np.float32)
    w = W.config_general(t=0.62, k=10)
    ctx = make_ctx(w, nemd, torch)
    ctx.model_train(X, T, steps=200, batch=64, lr=3e-3, seed=3)
    path = tmp_path / "m.bin"
    ctx.model_save(path)
    ctx.close()
    ctx = make_ctx(w, nemd, torch)
    ctx.model_load(path)
    q = torch.from_numpy(w.q).cuda()
    ctx.set_state(q, w.t)
    f = ctx.features(w.rc)
    choice = int(np.argmin(ctx.model_predict(f[None, :])[0]))
    ctx.build_cells(nemd.NEMD_AUTO_LEARNED, w.rc)
    ctx.compute_forces()
    st = ctx.stats()
    assert st["variant"] == (choice & 1) and st["cell_factor"] == 1 + (choice >> 1)
    # features are the reduced lattice, density, cut-off and ln N
    lat = ctx.lattice()
    assert np.allclose(f[:9], (lat["L"] / lat["V"] ** (1 / 3)).ravel(), rtol=1e-6)
    assert abs(f[9] - w.n / lat["V"]) < 1e-6 and abs(f[10] - w.rc) < 1e-6
    assert abs(f[11] - np.log(w.n)) < 1e-5
    ctx.close()


def test_learned_choice_beats_volume_rule_on_held_out_strains():
    """Measured timings of the four options (cell list variant x cell factor) of
    the row kernel on strained LJ and WCA systems: the model, trained on two
    thirds of the strains, is judged on the others against the exhaustive
    choice, next to the paper's neighbourhood-volume rule (k = 1).  The rule
    counts cells; the row kernel's cost is not proportional to them (each lane
    searches only its own window along the row), and for WCA the rule often
    picks the dynamic offset list where the dynamic size one is faster."""
    rows_f, rows_t, rule = [], [], []
    series = (W.general_series(k=14, seed=11), W.planar_series(k=16, seed=12),
              W.StrainSeries(W.M_GENERAL, 14, 13, kind=W.POT_WCA), W.StrainSeries(W.M_PLANAR, 12, 14, kind=W.POT_WCA))
    for ser in series:
        ctx = make_ctx(ser.workload(0.0), nemd, torch)
        ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
        for i in range(24):
            t = (i + 0.5) / 24 * ser.period
            q = torch.from_numpy(ser.positions(t)).cuda()
            ctx.set_state(q, t)
            f, ms = ctx.time_options(ser.rc, reps=3)
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
            ctx.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
            ctx.compute_forces()
            rows_f.append(f)
            rows_t.append(ms)
            rule.append(ctx.stats()["variant"])     # option index of the rule at k = 1
        ctx.close()
    X = np.array(rows_f)
    T = np.array(rows_t)
    train = np.arange(len(X)) % 3 != 0
    test = ~train
    ctx = _ctx()
    ctx.model_train(X[train], T[train], steps=1500, batch=64, lr=3e-3, seed=7)
    pick = np.argmin(ctx.model_predict(X[test]), axis=1)
    best = T[test].min(axis=1)
    regret_learned = float((T[test][np.arange(test.sum()), pick] - best).sum())
    regret_rule = float((T[test][np.arange(test.sum()), np.array(rule)[test]] - best).sum())
    assert regret_learned < regret_rule
    ctx.close()
