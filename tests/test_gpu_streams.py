"""Independent evaluations on several contexts and streams (the form the bench
times): three contexts, each on its own CUDA stream, take the strains of one
period in turn, with no synchronisation between the strains.  Every strain's
F, U and W equal bit for bit those of one context evaluating the strains one
after another (each kernel sums in a fixed order), and one strain per
variant is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, mat_rel, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

S = 12   # strains of one period


def _ctx(ser, stream=None):
    ctx = nemd.Context(0, stream=stream)
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
    return ctx


def test_three_streams_equal_one_stream_bit_for_bit():
    ser = W.general_series(k=16)          # N = 16384, general flow
    ts = [i / S * ser.period for i in range(S)]
    qs = [torch.from_numpy(ser.positions(t)).cuda() for t in ts]

    def out():
        return (torch.zeros((ser.n, 3), dtype=torch.float32, device="cuda"),
                torch.zeros(1, dtype=torch.float64, device="cuda"),
                torch.zeros(9, dtype=torch.float64, device="cuda"))

    # one context, one stream, one strain after another
    one = _ctx(ser)
    ref = []
    for i in range(S):
        F, U, Wv = out()
        one.set_state(qs[i], ts[i])
        one.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
        one.compute_forces(F, U, Wv)
        one.sync()
        ref.append((F.cpu().numpy(), float(U.item()), Wv.cpu().numpy(), one.stats()["variant"]))
    one.close()

    # three contexts on three streams, strains in turn, results kept per strain
    streams = [torch.cuda.Stream() for _ in range(3)]
    ctxs = [_ctx(ser, s.cuda_stream) for s in streams]
    res = [out() for _ in range(S)]
    for i in range(S):
        c = ctxs[i % 3]
        c.set_state(qs[i], ts[i])
        c.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
        c.compute_forces(*res[i])
    for c in ctxs:
        c.sync()
    torch.cuda.synchronize()
    for i in range(S):
        F, U, Wv = res[i]
        assert np.array_equal(F.cpu().numpy(), ref[i][0]), i
        assert float(U.item()) == ref[i][1], i
        assert np.array_equal(Wv.cpu().numpy(), ref[i][2]), i
    for c in ctxs:
        c.close()

    # the oracle on one strain of each cell list the volume rule picked
    seen = set()
    for i in range(S):
        v = ref[i][3]
        if v in seen:
            continue
        seen.add(v)
        w = ser.workload(ts[i])
        o = oracle.evaluate(w, "ds")
        assert force_err(ref[i][0].astype(np.float64), o.F) <= 1e-5
        assert rel(ref[i][1], o.U) <= 1e-6
        assert mat_rel(ref[i][2].reshape(3, 3), o.W) <= 1e-6
