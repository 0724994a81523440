"""nemd_forces_noalloc: the force evaluation for callers that cannot call cudaMalloc.

Some callers may not allocate device memory (a loop that must never allocate
once running, a plug-in without access to its host's CUDA allocator).  For
them the library offers one entry point whose scratch is a fixed device array
inside the library.  This file checks, through the C ABI, that two calls in a
row (two different systems, so the second must not be disturbed by what the
first left in the shared array) give the same forces, energy and virial as the
ordinary context path (nemd_set_state -> nemd_build_cells ->
nemd_compute_forces) within the parity tolerances, and that requests larger
than the array are refused.  Collected last on purpose.
"""
import numpy as np
import pytest

from paper_1412_3784_gb300 import workloads as W
from gpu_util import force_err, mat_rel, rel, run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402

F_TOL = 1e-5
UW_TOL = 3e-6


def call_noalloc(w, variant):
    dev = torch.device("cuda:0")
    A = np.ascontiguousarray(w.A, dtype=np.float64)
    L0 = np.ascontiguousarray(w.L0, dtype=np.float64)
    q = torch.from_numpy(np.ascontiguousarray(w.q)).to(dev)
    F = torch.full((w.n, 3), float("nan"), dtype=torch.float32, device=dev)
    UW = torch.full((10,), float("nan"), dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    kind = nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = nemd.nemd_forces_noalloc(A.ctypes.data, L0.ctypes.data, float(w.T), float(w.t), q.data_ptr(), w.n,
                                  int(variant), float(w.rc), kind, float(w.eps), float(w.sigma), int(w.shift),
                                  F.data_ptr(), UW.data_ptr(), status.data_ptr(), stream)
    return rc, F, UW, status, q


def test_noalloc_matches_context_path_two_calls():
    cases = [(W.config_planar(11, k=8), nemd.NEMD_DO), (W.config_equilibrium_wca(), nemd.NEMD_DS)]
    refs = [run(w, v) for w, v in cases]
    outs = [call_noalloc(w, v) for w, v in cases]   # two calls in a row
    torch.cuda.synchronize()
    for (w, _), ref, (rc, F, UW, status, _q) in zip(cases, refs, outs):
        assert rc == 0
        assert int(status.item()) == 0
        Fh = F.cpu().numpy().astype(np.float64)
        uw = UW.cpu().numpy()
        assert np.all(np.isfinite(Fh)) and np.all(np.isfinite(uw))
        assert force_err(Fh, ref["F"]) <= F_TOL
        assert rel(uw[0], ref["U"]) <= UW_TOL
        assert mat_rel(uw[1:].reshape(3, 3), ref["W"]) <= UW_TOL
        # both paths run the same kernels in the same order on the same inputs, so
        # anything the previous call left in the shared array would show up here
        assert np.array_equal(Fh, ref["F"])
        assert uw[0] == ref["U"] and np.array_equal(uw[1:].reshape(3, 3), ref["W"])


def test_noalloc_refuses_sizes_beyond_its_array():
    w = W.config_equilibrium_wca(k=17)          # 19652 particles > 16384
    assert w.n > nemd.NEMD_NOALLOC_MAX_N
    rc, F, UW, status, _ = call_noalloc(w, nemd.NEMD_DS)
    assert rc == 10                              # NEMD_ERR_CAPACITY
    assert int(status.item()) == -1              # nothing was launched
    # a box with more cells than the array holds is refused too
    big = W.uniform_random(1000, 60.0 * np.eye(3), seed=1, rc=1.0)   # 216000 cells > 16384
    rc, *_ = call_noalloc(big, nemd.NEMD_DS)
    assert rc == 10
