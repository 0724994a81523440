"""FP64 CPU oracle for the cell-list force evaluation (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product path never does.  The C code in
oracle.c states, per function, the passage of the paper it follows; the
time-integration oracle is in oracle/integrate.py.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_expm.argtypes = [_dp, ctypes.c_double, _dp]
        L.orc_expm.restype = None
        L.orc_lattice.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp]
        L.orc_lattice.restype = None
        L.orc_kr_residual.argtypes = [_dp, _dp, _i64p, ctypes.c_double]
        L.orc_kr_residual.restype = ctypes.c_double
        L.orc_heights.argtypes = [_dp, _dp]
        L.orc_qr.argtypes = [_dp, _dp, _dp]
        L.orc_wrap.argtypes = [_dp, _dp, ctypes.c_int64, _dp, _dp, _dp]
        L.orc_wrap.restype = None
        sig = [_dp, ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
               ctypes.c_int, _i32p, ctypes.c_int64, _dp, _dp, _i64p]
        L.orc_brute.argtypes = sig
        L.orc_brute.restype = ctypes.c_int64
        sig_c = [_dp, ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                 ctypes.c_double, ctypes.c_int, _i32p, ctypes.c_int64, _dp, _dp, _i64p]
        L.orc_cells_ds.argtypes = sig_c
        L.orc_cells_ds.restype = ctypes.c_int64
        L.orc_cells_do.argtypes = sig_c
        L.orc_cells_do.restype = ctypes.c_int64
        L.orc_ds_counts.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _i64p]
        L.orc_do_counts.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _i64p]
        L.orc_do_stencil.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _i64p, _i64p, ctypes.c_int64]
        L.orc_do_stencil.restype = ctypes.c_int64
        L.orc_do_fixed_count.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64]
        L.orc_do_fixed_count.restype = ctypes.c_int64
        L.orc_do_total_stencil_cells.argtypes = [_dp, ctypes.c_double, ctypes.c_int]
        L.orc_do_total_stencil_cells.restype = ctypes.c_int64
        L.orc_sample_forces.argtypes = [_dp, ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64, _dp, _i64p, _dp]
        L.orc_sample_forces.restype = None
        L.orc_mlp_loss_grad.argtypes = [_dp, _dp, _dp, ctypes.c_int64, _dp, _dp]
        L.orc_mlp_loss_grad.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def expm(A, tau):
    A, pA = _d(A)
    E = np.zeros(9)
    lib().orc_expm(pA, float(tau), E.ctypes.data_as(_dp))
    return E.reshape(3, 3)


def lattice(A, L0, T, t, centered=False):
    """L(t) = exp(A tau) L0 with its inverse, volume, heights and QR; tau = t mod T
    in [0, T), or in [-T/2, T/2) when centered (remap half way through a period)."""
    A, pA = _d(A)
    L0, pL = _d(L0)
    out = np.zeros(40)
    lib().orc_lattice(pA, pL, float(T), float(t), 1 if centered else 0, out.ctypes.data_as(_dp))
    return {"L": out[0:9].reshape(3, 3).copy(), "Linv": out[9:18].reshape(3, 3).copy(),
            "V": float(out[18]), "h": out[19:22].copy(), "Q": out[22:31].reshape(3, 3).copy(),
            "R": out[31:40].reshape(3, 3).copy()}


def kr_residual(A, L0, M, T):
    A, pA = _d(A)
    L0, pL = _d(L0)
    M, pM = _i64(M)
    return float(lib().orc_kr_residual(pA, pL, pM, float(T)))


def heights(L):
    L, pL = _d(L)
    h = np.zeros(3)
    lib().orc_heights(pL, h.ctypes.data_as(_dp))
    return h


def qr(L):
    L, pL = _d(L)
    Q = np.zeros(9)
    R = np.zeros(9)
    lib().orc_qr(pL, Q.ctypes.data_as(_dp), R.ctypes.data_as(_dp))
    return Q.reshape(3, 3), R.reshape(3, 3)


def wrap(L, Linv, q):
    L, pL = _d(L)
    Li, pLi = _d(Linv)
    q, pq = _d(q)
    n = q.shape[0]
    s = np.zeros((n, 3))
    qp = np.zeros((n, 3))
    lib().orc_wrap(pL, pLi, n, pq, s.ctypes.data_as(_dp), qp.ctypes.data_as(_dp))
    return s, qp


def ds_counts(L, rc, kfac=1):
    L, pL = _d(L)
    c = np.zeros(3, dtype=np.int64)
    lib().orc_ds_counts(pL, float(rc), int(kfac), c.ctypes.data_as(_i64p))
    return c


def do_counts(R, rc, kfac=1):
    R, pR = _d(R)
    c = np.zeros(3, dtype=np.int64)
    lib().orc_do_counts(pR, float(rc), int(kfac), c.ctypes.data_as(_i64p))
    return c


def do_stencil(R, rc, kfac=1):
    """Rows (iy, iz, jyu, jzu, dxlo, dxhi) of the tight dynamic offset stencil."""
    R, pR = _d(R)
    l = np.zeros(3, dtype=np.int64)
    total = lib().orc_do_stencil(pR, float(rc), int(kfac), l.ctypes.data_as(_i64p), None, 0)
    if total < 0:
        raise ValueError("box too small for the cut-off")
    rows = np.zeros((total, 6), dtype=np.int64)
    lib().orc_do_stencil(pR, float(rc), int(kfac), l.ctypes.data_as(_i64p),
                         rows.ctypes.data_as(_i64p), total)
    return l, rows


def do_fixed_count(l, iy, iz):
    l, pl = _i64(l)
    return int(lib().orc_do_fixed_count(pl, int(iy), int(iz)))


def do_total_stencil_cells(R, rc, kfac=1):
    R, pR = _d(R)
    return int(lib().orc_do_total_stencil_cells(pR, float(rc), int(kfac)))


def sample_forces(L, s, qp, idx, rc, eps=1.0, sigma=1.0, shift=1):
    """Brute-force forces (and per-particle neighbour counts, half energies) on sampled particles."""
    L, pL = _d(L)
    s, ps = _d(s)
    qp, pq = _d(qp)
    idx, pi = _i64(idx)
    F = np.zeros((len(idx), 3))
    cnt = np.zeros(len(idx), dtype=np.int64)
    uh = np.zeros(len(idx))
    lib().orc_sample_forces(pL, s.shape[0], ps, pq, float(rc), float(eps), float(sigma), int(shift), pi,
                            len(idx), F.ctypes.data_as(_dp), cnt.ctypes.data_as(_i64p), uh.ctypes.data_as(_dp))
    return F, cnt, uh


MLP_PARAMS = 64 * 12 + 64 + 64 * 64 + 64 + 4 * 64 + 4


def mlp_loss_grad(params, X, T, want_grad=True):
    """The selector network in FP64: (loss, gradient or None, outputs)."""
    p, pp = _d(params)
    X, px = _d(X)
    T, pt = _d(T)
    rows = X.shape[0]
    g = np.zeros(MLP_PARAMS) if want_grad else None
    Y = np.zeros((rows, 4))
    loss = lib().orc_mlp_loss_grad(pp, px, pt, rows, g.ctypes.data_as(_dp) if want_grad else None,
                                   Y.ctypes.data_as(_dp))
    return float(loss), g, Y


class Result:
    """Pairs (unordered, canonical orientation), forces, energy, virial, counters."""

    def __init__(self, pairs, F, U, W, npairs, ncand):
        self.pairs = pairs
        self.F = F
        self.U = U
        self.W = W
        self.npairs = npairs
        self.ncand = ncand


def _run(fn, L, s, qp, rc, eps, sigma, shift, want_pairs, kfac=None):
    L, pL = _d(L)
    s, ps = _d(s)
    qp, pq = _d(qp)
    n = s.shape[0]
    F = np.zeros((n, 3))
    UW = np.zeros(10)
    stats = np.zeros(2, dtype=np.int64)
    args_head = [pL, n, ps, pq, float(rc)]
    if kfac is not None:
        args_head.append(int(kfac))
    tail = [float(eps), float(sigma), int(shift)]
    cap = 0
    pairs = None
    if want_pairs:
        cnt = fn(*args_head, *tail, None, 0, None, None, stats.ctypes.data_as(_i64p))
        if cnt < 0:
            raise ValueError("box too small for the cut-off")
        cap = int(cnt)
        pairs = np.zeros((max(cap, 1), 5), dtype=np.int32)
    ptr = pairs.ctypes.data_as(_i32p) if pairs is not None else None
    cnt = fn(*args_head, *tail, ptr, cap, F.ctypes.data_as(_dp), UW.ctypes.data_as(_dp),
             stats.ctypes.data_as(_i64p))
    if cnt < 0:
        raise ValueError("box too small for the cut-off")
    if pairs is not None:
        pairs = pairs[:cnt]
    return Result(pairs, F, float(UW[0]), UW[1:].reshape(3, 3).copy(), int(stats[0]), int(stats[1]))


def brute(L, s, qp, rc, eps=1.0, sigma=1.0, shift=1, want_pairs=True):
    return _run(lib().orc_brute, L, s, qp, rc, eps, sigma, shift, want_pairs)


def cells_ds(L, s, qp, rc, kfac=1, eps=1.0, sigma=1.0, shift=1, want_pairs=True):
    return _run(lib().orc_cells_ds, L, s, qp, rc, eps, sigma, shift, want_pairs, kfac=kfac)


def cells_do(L, s, qp, rc, kfac=1, eps=1.0, sigma=1.0, shift=1, want_pairs=True):
    return _run(lib().orc_cells_do, L, s, qp, rc, eps, sigma, shift, want_pairs, kfac=kfac)


def evaluate(w, method="ds", kfac=1, want_pairs=False):
    """Full oracle evaluation of a workload: lattice, wrap, then the chosen sum."""
    lat = lattice(w.A, w.L0, w.T, w.t, centered=bool(getattr(w, "remap", 0)))
    s, qp = wrap(lat["L"], lat["Linv"], w.q)
    if method == "brute":
        res = brute(lat["L"], s, qp, w.rc, w.eps, w.sigma, w.shift, want_pairs)
    elif method == "ds":
        res = cells_ds(lat["L"], s, qp, w.rc, kfac, w.eps, w.sigma, w.shift, want_pairs)
    elif method == "do":
        res = cells_do(lat["L"], s, qp, w.rc, kfac, w.eps, w.sigma, w.shift, want_pairs)
    else:
        raise ValueError(method)
    res.lattice = lat
    res.s = s
    res.qp = qp
    return res


def canonical_pair_keys(pairs):
    """Pairs (i, j, n1, n2, n3) as a sorted int64 key array for set comparison."""
    p = np.asarray(pairs, dtype=np.int64)
    if p.size == 0:
        return np.zeros(0, dtype=np.int64)
    key = ((((p[:, 0] << 22) + p[:, 1]) * 16 + (p[:, 2] + 8)) * 16 + (p[:, 3] + 8)) * 16 + (p[:, 4] + 8)
    return np.sort(key)
