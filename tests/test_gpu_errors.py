"""Error behaviour of the C ABI (each error is produced on the host side or by
an input the kernels turn into an error word; nothing here faults a GPU)."""
import numpy as np
import pytest

from paper_1412_3784_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3784_gb300 import nemd  # noqa: E402


def code_of(fn, *a):
    with pytest.raises(nemd.NemdError) as ei:
        fn(*a)
    return ei.value.code


def test_flow_validation():
    ctx = nemd.Context(0)
    A, _, _ = W.kr_flow(W.M_PLANAR)
    L0 = 20.0 * np.eye(3)
    bad_det = W.M_PLANAR.copy()
    bad_det[0, 0] = 3
    assert code_of(ctx.set_flow, A, L0, bad_det, 1.0) == 2            # NOT_SL3Z
    assert code_of(ctx.set_flow, 1.1 * A, L0, W.M_PLANAR, 1.0) == 3    # NOT_KR
    At = A.copy()
    At[0, 0] += 0.1
    assert code_of(ctx.set_flow, At, L0, W.M_PLANAR, 1.0) == 4        # TRACE
    assert code_of(ctx.set_flow, np.zeros((3, 3)), L0, W.M_PLANAR, 1.0) == 3  # A = 0 needs M = I
    assert code_of(ctx.set_flow, A, L0, W.M_PLANAR, -1.0) == 1
    ctx.set_flow(A, L0, W.M_PLANAR, 1.0)
    ctx.close()


def test_call_order():
    ctx = nemd.Context(0)
    q = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    assert code_of(ctx.set_state, q, 0.0) == 6
    ctx.set_flow(np.zeros((3, 3)), 10 * np.eye(3), np.eye(3, dtype=np.int64), 1.0)
    assert code_of(ctx.build_cells, 0, 2.5) == 6
    ctx.set_state(q, 0.0)
    assert code_of(ctx.compute_forces) == 6
    assert code_of(ctx.build_cells, 7, 2.5) == 1
    assert code_of(ctx.build_cells, 0, -1.0) == 1
    ctx.close()


def test_box_too_small_is_deferred_error():
    ctx = nemd.Context(0)
    ctx.set_flow(np.zeros((3, 3)), 4.0 * np.eye(3), np.eye(3, dtype=np.int64), 1.0)
    q = torch.rand((50, 3), dtype=torch.float64, device="cuda") * 4
    ctx.set_state(q, 0.0)
    ctx.build_cells(0, 5.0)      # h = 4 < rc = 5: no cell fits
    F = torch.zeros((50, 3), dtype=torch.float32, device="cuda")
    ctx.compute_forces(F)
    assert code_of(ctx.sync) == 5
    # the context stays usable
    ctx.set_state(q, 0.0)
    ctx.build_cells(0, 1.0)
    ctx.compute_forces(F)
    ctx.sync()
    ctx.close()


def test_nonfinite_positions():
    ctx = nemd.Context(0)
    ctx.set_flow(np.zeros((3, 3)), 10.0 * np.eye(3), np.eye(3, dtype=np.int64), 1.0)
    q = torch.rand((100, 3), dtype=torch.float64, device="cuda") * 10
    q[17, 1] = float("nan")
    ctx.set_state(q, 0.0)
    ctx.build_cells(0, 2.5)
    ctx.compute_forces()
    assert code_of(ctx.sync) == 8
    ctx.close()


def test_wca_cutoff_and_options():
    ctx = nemd.Context(0)
    ctx.set_flow(np.zeros((3, 3)), 10.0 * np.eye(3), np.eye(3, dtype=np.int64), 1.0)
    ctx.set_potential(nemd.NEMD_WCA, 1.0, 1.0, 1)
    q = torch.rand((10, 3), dtype=torch.float64, device="cuda") * 10
    ctx.set_state(q, 0.0)
    assert code_of(ctx.build_cells, 0, 2.5) == 1
    assert code_of(ctx.set_option, nemd.NEMD_OPT_CELL_FACTOR, 0) == 1
    assert code_of(ctx.set_option, 999, 1) == 12
    ctx.close()
