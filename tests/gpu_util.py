"""Helpers for the GPU tests: run one force evaluation through the C ABI."""
import numpy as np

from paper_1412_3784_gb300 import workloads as W


def kind_of(w):
    return 1 if w.kind == W.POT_WCA else 0


def make_ctx(w, nemd, torch):
    ctx = nemd.Context(0)
    ctx.set_flow(w.A, w.L0, w.M, w.T)
    ctx.set_potential(kind_of(w), w.eps, w.sigma, w.shift)
    ctx.set_option(nemd.NEMD_OPT_REMAP, getattr(w, "remap", 0))
    return ctx


def run(w, variant, *, precise=False, record=False, kfac=1, ctx=None, q=None, kernel=(0, 16)):
    """Evaluate workload w on cuda:0; returns dict with F (N,3) float64, U, W, stats, pairs."""
    import torch

    from paper_1412_3784_gb300 import nemd

    own = ctx is None
    if own:
        ctx = make_ctx(w, nemd, torch)
    dev = torch.device("cuda:0")
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 1 if precise else 0)
    ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, kfac)
    kern, group = kernel if isinstance(kernel, tuple) else (kernel, 16)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, kern)
    ctx.set_option(nemd.NEMD_OPT_GROUP, group)
    cap = 0
    if record:
        cap = int(w.n * 40 + 1000)
    ctx.set_option(nemd.NEMD_OPT_RECORD_PAIRS, cap)
    if q is None:
        q = torch.from_numpy(np.ascontiguousarray(w.q)).to(dev)
    F = torch.zeros((w.n, 3), dtype=torch.float32, device=dev)
    U = torch.zeros(1, dtype=torch.float64, device=dev)
    Wv = torch.zeros(9, dtype=torch.float64, device=dev)
    ctx.set_state(q, w.t)
    ctx.build_cells(variant, w.rc)
    ctx.compute_forces(F, U, Wv)
    ctx.sync()
    out = {"F": F.cpu().numpy().astype(np.float64), "U": float(U.item()),
           "W": Wv.cpu().numpy().reshape(3, 3), "stats": ctx.stats(), "lattice": ctx.lattice()}
    if record:
        out["pairs"] = ctx.pairs()
    ctx.set_option(nemd.NEMD_OPT_RECORD_PAIRS, 0)
    if own:
        ctx.close()
    return out


def force_err(F, Fref):
    return float(np.abs(F - Fref).max() / max(np.abs(Fref).max(), 1e-300))


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def mat_rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
