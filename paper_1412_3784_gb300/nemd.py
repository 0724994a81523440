"""Thin ctypes binding of the C ABI in include/nemd.h (libnemd.so).

Argument marshalling only: every step of the force evaluation runs in the
library's CUDA kernels.  Importing this module loads libnemd.so and raises
ImportError if it is missing -- there is no CPU fallback.

Functions keep the C names (nemd_create, nemd_set_flow, ...).  `Context` is a
small convenience wrapper that accepts torch tensors or numpy arrays and uses
torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnemd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1412_3784_gb300.build.build() "
                      "(the CUDA library is required; there is no fallback)")

_lib = ctypes.CDLL(LIB_PATH)

NEMD_OK = 0
ERRORS = {1: "ARG", 2: "NOT_SL3Z", 3: "NOT_KR", 4: "TRACE", 5: "BOX_TOO_SMALL", 6: "ORDER",
          7: "CUDA", 8: "NONFINITE", 9: "TIMEOUT", 10: "CAPACITY", 11: "NOMEM", 12: "UNSUPPORTED"}
NEMD_DS, NEMD_DO, NEMD_AUTO_HEURISTIC, NEMD_AUTO_LEARNED = 0, 1, 2, 3
NEMD_LJ, NEMD_WCA = 0, 1
NEMD_OPT_PRECISE, NEMD_OPT_RECORD_PAIRS, NEMD_OPT_KERNEL, NEMD_OPT_CELL_FACTOR, NEMD_OPT_BLOCK = 1, 2, 3, 4, 5
NEMD_OPT_TIMING = 6
NEMD_OPT_GROUP = 7
NEMD_OPT_AUTOTUNED = 8
NEMD_OPT_REMAP = 9
NEMD_OPT_ASYNC_HOST = 10
NEMD_OPT_INT_GRAPH = 11

EXPORTED = ["nemd_create", "nemd_destroy", "nemd_set_flow", "nemd_set_potential", "nemd_set_state",
            "nemd_build_cells", "nemd_compute_forces", "nemd_integrate", "nemd_sync", "nemd_last_error",
            "nemd_set_option", "nemd_get_lattice", "nemd_get_stats", "nemd_get_pairs",
            "nemd_get_kernel_time", "nemd_measure_peaks", "nemd_forces_noalloc", "nemd_autotune",
            "nemd_tune_save", "nemd_tune_load", "nemd_features", "nemd_time_options", "nemd_model_train",
            "nemd_model_predict", "nemd_model_grad", "nemd_model_set_params", "nemd_model_get_params",
            "nemd_model_save", "nemd_model_load", "nemd_batch_create", "nemd_batch_destroy",
            "nemd_batch_last_error", "nemd_batch_add", "nemd_batch_finalize", "nemd_batch_offsets",
            "nemd_batch_set_state", "nemd_batch_compute", "nemd_batch_sync", "nemd_batch_set_option",
            "nemd_batch_get_stats", "nemd_batch_autotune", "nemd_set_verlet", "nemd_get_verlet_stats"]
NEMD_BATCH_OPT_CELL_FACTOR, NEMD_BATCH_OPT_TILE, NEMD_BATCH_OPT_GRAPH, NEMD_BATCH_OPT_KERNEL = 1, 2, 3, 4
NEMD_MLP_INPUTS, NEMD_MLP_OUTPUTS, NEMD_MLP_PARAMS, NEMD_MLP_NORM = 12, 4, 5252, 26
NEMD_NOALLOC_MAX_N = 16384
NEMD_NOALLOC_MAX_CELLS = 16384


class nemd_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pairs", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("ncells", ctypes.c_int64), ("counts", ctypes.c_int32 * 3), ("variant", ctypes.c_int32),
                ("cell_factor", ctypes.c_int32), ("max_rows", ctypes.c_int32),
                ("stencil_cells", ctypes.c_int64), ("rechecks", ctypes.c_int64),
                ("tau", ctypes.c_double), ("band", ctypes.c_double), ("launches", ctypes.c_int64)]


class nemd_tune_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("group", ctypes.c_int32), ("cell_factor", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class nemd_tune_entry(ctypes.Structure):
    _fields_ = [("cfg", nemd_tune_config), ("ms", ctypes.c_double)]


class nemd_system(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 9), ("L0", ctypes.c_double * 9), ("M", ctypes.c_int64 * 9),
                ("T", ctypes.c_double), ("eps", ctypes.c_double), ("sigma", ctypes.c_double),
                ("rc", ctypes.c_double), ("n", ctypes.c_int64), ("kind", ctypes.c_int32),
                ("shift", ctypes.c_int32), ("variant", ctypes.c_int32), ("remap", ctypes.c_int32)]


class nemd_batch_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("candidates", ctypes.c_int64), ("band", ctypes.c_int64),
                ("counts", ctypes.c_int32 * 3), ("variant", ctypes.c_int32), ("cell_factor", ctypes.c_int32),
                ("status", ctypes.c_int32)]


_vp = ctypes.c_void_p
_sig = {
    "nemd_create": ([ctypes.POINTER(_vp), ctypes.c_int, _vp], ctypes.c_int),
    "nemd_destroy": ([_vp], ctypes.c_int),
    "nemd_set_flow": ([_vp, _vp, _vp, _vp, ctypes.c_double], ctypes.c_int),
    "nemd_set_potential": ([_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int], ctypes.c_int),
    "nemd_set_state": ([_vp, _vp, ctypes.c_int64, ctypes.c_double], ctypes.c_int),
    "nemd_build_cells": ([_vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
    "nemd_compute_forces": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "nemd_integrate": ([_vp, _vp, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                        ctypes.c_int, ctypes.c_double, ctypes.c_int], ctypes.c_int),
    "nemd_sync": ([_vp], ctypes.c_int),
    "nemd_set_verlet": ([_vp, ctypes.c_double], ctypes.c_int),
    "nemd_get_verlet_stats": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "nemd_last_error": ([_vp], ctypes.c_char_p),
    "nemd_set_option": ([_vp, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "nemd_get_lattice": ([_vp, _vp], ctypes.c_int),
    "nemd_get_stats": ([_vp, ctypes.POINTER(nemd_stats)], ctypes.c_int),
    "nemd_get_pairs": ([_vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "nemd_get_kernel_time": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
                             ctypes.c_int),
    "nemd_measure_peaks": ([ctypes.c_int, _vp], ctypes.c_int),
    "nemd_autotune": ([_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(nemd_tune_config),
                       ctypes.POINTER(nemd_tune_entry), ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "nemd_tune_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "nemd_tune_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "nemd_features": ([_vp, ctypes.c_double, _vp], ctypes.c_int),
    "nemd_time_options": ([_vp, ctypes.c_double, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "nemd_model_train": ([_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                          _vp], ctypes.c_int),
    "nemd_model_predict": ([_vp, _vp, ctypes.c_int64, _vp], ctypes.c_int),
    "nemd_model_grad": ([_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "nemd_model_set_params": ([_vp, _vp, _vp], ctypes.c_int),
    "nemd_model_get_params": ([_vp, _vp, _vp], ctypes.c_int),
    "nemd_model_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "nemd_model_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "nemd_batch_create": ([ctypes.POINTER(_vp), ctypes.c_int, _vp], ctypes.c_int),
    "nemd_batch_destroy": ([_vp], ctypes.c_int),
    "nemd_batch_last_error": ([_vp], ctypes.c_char_p),
    "nemd_batch_add": ([_vp, ctypes.POINTER(nemd_system), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "nemd_batch_finalize": ([_vp], ctypes.c_int),
    "nemd_batch_offsets": ([_vp, _vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "nemd_batch_set_state": ([_vp, _vp, _vp], ctypes.c_int),
    "nemd_batch_compute": ([_vp, _vp, _vp], ctypes.c_int),
    "nemd_batch_sync": ([_vp, _vp], ctypes.c_int),
    "nemd_batch_set_option": ([_vp, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "nemd_batch_get_stats": ([_vp, ctypes.POINTER(nemd_batch_stats), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "nemd_batch_autotune": ([_vp, ctypes.c_int, ctypes.POINTER(nemd_tune_entry), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "nemd_forces_noalloc": ([_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int64, ctypes.c_int,
                             ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             _vp, _vp, _vp, _vp], ctypes.c_int),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f


class NemdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nemd error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def _ptr(x):
    """Raw address of a torch tensor, numpy array, or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(type(x))


def _current_stream(device):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


def measure_peaks(device=0):
    out = np.zeros(6)
    rc = nemd_measure_peaks(int(device), out.ctypes.data)
    if rc:
        raise NemdError(rc, "measure_peaks")
    return {"fp32_fma_ops": out[0], "fp32x2_fma_ops": out[1], "fp64_fma_ops": out[2],
            "copy_bytes_per_s": out[3], "sms": int(out[4]), "sm_clock_khz": out[5]}


class Context:
    """One nemd_ctx on a CUDA device and stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None):
        if stream is None:
            stream = _current_stream(device)
        h = _vp()
        rc = nemd_create(ctypes.byref(h), int(device), _vp(stream))
        if rc:
            raise NemdError(rc, "nemd_create")
        self.h = h
        self._keep = {}

    def close(self):
        if self.h:
            nemd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise NemdError(rc, nemd_last_error(self.h).decode())
        return rc

    def set_flow(self, A, L0, M, T):
        A = np.ascontiguousarray(A, dtype=np.float64)
        L0 = np.ascontiguousarray(L0, dtype=np.float64)
        M = np.ascontiguousarray(M, dtype=np.int64)
        return self._check(nemd_set_flow(self.h, A.ctypes.data, L0.ctypes.data, M.ctypes.data, float(T)))

    def set_potential(self, kind=NEMD_LJ, eps=1.0, sigma=1.0, shift=1):
        return self._check(nemd_set_potential(self.h, int(kind), float(eps), float(sigma), int(shift)))

    def set_state(self, q, t):
        self._keep["q"] = q   # keep the buffer alive while the device may read it
        n = int(q.shape[0])
        return self._check(nemd_set_state(self.h, _ptr(q), n, float(t)))

    def build_cells(self, variant, rc):
        return self._check(nemd_build_cells(self.h, int(variant), float(rc)))

    def compute_forces(self, F=None, U=None, W=None):
        return self._check(nemd_compute_forces(self.h, _ptr(F), _ptr(U), _ptr(W)))

    def integrate(self, q, p, t0, dt, nsteps, variant, rc, thermostat=1):
        """Advance device float64 (N, 3) positions q and peculiar momenta p in place
        by nsteps steps of dt from time t0 (see nemd_integrate)."""
        self._keep["q"] = q
        self._keep["p"] = p
        return self._check(nemd_integrate(self.h, _ptr(q), _ptr(p), int(q.shape[0]), float(t0), float(dt),
                                          int(nsteps), int(variant), float(rc), int(thermostat)))

    def sync(self):
        return self._check(nemd_sync(self.h))

    def set_verlet(self, skin):
        """Verlet list with this skin for integrate (0: off; see nemd_set_verlet)."""
        return self._check(nemd_set_verlet(self.h, float(skin)))

    def verlet_stats(self):
        """(builds, evaluations, entries per particle, last displacement) since the last set_verlet."""
        b, s, w, d = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0.0)
        self._check(nemd_get_verlet_stats(self.h, ctypes.byref(b), ctypes.byref(s), ctypes.byref(w),
                                          ctypes.byref(d)))
        return int(b.value), int(s.value), int(w.value), float(d.value)

    def set_option(self, key, value):
        return self._check(nemd_set_option(self.h, int(key), int(value)))

    def lattice(self):
        out = np.zeros(48)
        self._check(nemd_get_lattice(self.h, out.ctypes.data))
        return {"L": out[0:9].reshape(3, 3).copy(), "Linv": out[9:18].reshape(3, 3).copy(),
                "V": float(out[18]), "h": out[19:22].copy(), "Q": out[22:31].reshape(3, 3).copy(),
                "R": out[31:40].reshape(3, 3).copy(), "tau": float(out[40]), "band": float(out[41]),
                "counts": out[42:45].astype(np.int64), "ncells": int(out[45]),
                "variant": int(out[46]), "maxrows": int(out[47])}

    def stats(self):
        s = nemd_stats()
        self._check(nemd_get_stats(self.h, ctypes.byref(s)))
        return {"n": s.n, "pairs": s.pairs, "candidates": s.candidates, "ncells": s.ncells,
                "counts": list(s.counts), "variant": s.variant, "cell_factor": s.cell_factor,
                "max_rows": s.max_rows, "stencil_cells": s.stencil_cells, "rechecks": s.rechecks,
                "tau": s.tau, "band": s.band, "launches": s.launches}

    def autotune(self, variant, rc, reps=3):
        """Time every candidate configuration; returns (best config dict, list of (config, ms))."""
        best = nemd_tune_config()
        times = (nemd_tune_entry * 32)()
        nt = ctypes.c_int(0)
        self._check(nemd_autotune(self.h, int(variant), float(rc), int(reps), ctypes.byref(best), times, 32,
                                  ctypes.byref(nt)))
        cfg = lambda c: {"kernel": c.kernel, "group": c.group, "cell_factor": c.cell_factor}
        return cfg(best), [(cfg(times[k].cfg), times[k].ms) for k in range(nt.value)]

    def tune_save(self, path):
        return self._check(nemd_tune_save(self.h, str(path).encode()))

    def tune_load(self, path):
        return self._check(nemd_tune_load(self.h, str(path).encode()))

    # ---- learned selector ----
    def features(self, rc):
        out = np.zeros(NEMD_MLP_INPUTS, dtype=np.float32)
        self._check(nemd_features(self.h, float(rc), out.ctypes.data))
        return out

    def time_options(self, rc, reps=2):
        f = np.zeros(NEMD_MLP_INPUTS, dtype=np.float32)
        ms = np.zeros(NEMD_MLP_OUTPUTS, dtype=np.float32)
        self._check(nemd_time_options(self.h, float(rc), int(reps), f.ctypes.data, ms.ctypes.data))
        return f, ms

    def model_train(self, X, T_ms, steps=2000, batch=128, lr=3e-3, seed=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T_ms, dtype=np.float32)
        hist = np.zeros(int(steps), dtype=np.float32)
        self._check(nemd_model_train(self.h, X.ctypes.data, T.ctypes.data, X.shape[0], int(steps), int(batch),
                                     float(lr), int(seed), hist.ctypes.data))
        return hist

    def model_predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], NEMD_MLP_OUTPUTS), dtype=np.float32)
        self._check(nemd_model_predict(self.h, X.ctypes.data, X.shape[0], Y.ctypes.data))
        return Y

    def model_grad(self, Xn, Tn):
        Xn = np.ascontiguousarray(Xn, dtype=np.float32)
        Tn = np.ascontiguousarray(Tn, dtype=np.float32)
        g = np.zeros(NEMD_MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        self._check(nemd_model_grad(self.h, Xn.ctypes.data, Tn.ctypes.data, Xn.shape[0], g.ctypes.data,
                                    ctypes.byref(loss)))
        return g, loss.value

    def model_set_params(self, params, norm):
        p = np.ascontiguousarray(params, dtype=np.float32)
        nrm = np.ascontiguousarray(norm, dtype=np.float32)
        return self._check(nemd_model_set_params(self.h, p.ctypes.data, nrm.ctypes.data))

    def model_get_params(self):
        p = np.zeros(NEMD_MLP_PARAMS, dtype=np.float32)
        nrm = np.zeros(NEMD_MLP_NORM, dtype=np.float32)
        self._check(nemd_model_get_params(self.h, p.ctypes.data, nrm.ctypes.data))
        return p, nrm

    def model_save(self, path):
        return self._check(nemd_model_save(self.h, str(path).encode()))

    def model_load(self, path):
        return self._check(nemd_model_load(self.h, str(path).encode()))

    def kernel_time(self):
        """(total ms, launches) of the force kernel since the last call (timing option on)."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._check(nemd_get_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, int(n.value)

    def pairs(self, cap=None):
        cnt = ctypes.c_int64(0)
        rc = nemd_get_pairs(self.h, None, 0, ctypes.byref(cnt))
        if rc not in (0, 10):
            self._check(rc)
        n = int(cnt.value) if cap is None else int(cap)
        out = np.zeros((max(n, 1), 5), dtype=np.int32)
        self._check(nemd_get_pairs(self.h, out.ctypes.data, n, ctypes.byref(cnt)))
        return out[: int(cnt.value)]


class Batch:
    """One nemd_batch: many independent systems evaluated by one launch per stage
    (a captured CUDA graph).  `systems` is a list of dicts with the keys of
    nemd_system: A, L0, M, T, rc, n, and optionally kind, eps, sigma, shift,
    variant."""

    def __init__(self, systems, device=0, stream=None):
        if stream is None:
            stream = _current_stream(device)
        h = _vp()
        rc = nemd_batch_create(ctypes.byref(h), int(device), _vp(stream))
        if rc:
            raise NemdError(rc, "nemd_batch_create")
        self.h = h
        self._keep = {}
        for s in systems:
            y = nemd_system()
            y.A[:] = [float(x) for x in np.asarray(s["A"], dtype=np.float64).ravel()]
            y.L0[:] = [float(x) for x in np.asarray(s["L0"], dtype=np.float64).ravel()]
            y.M[:] = [int(x) for x in np.asarray(s["M"], dtype=np.int64).ravel()]
            y.T = float(s["T"])
            y.eps = float(s.get("eps", 1.0))
            y.sigma = float(s.get("sigma", 1.0))
            y.rc = float(s["rc"])
            y.n = int(s["n"])
            y.kind = int(s.get("kind", NEMD_LJ))
            y.shift = int(s.get("shift", 1))
            y.variant = int(s.get("variant", NEMD_AUTO_HEURISTIC))
            y.remap = int(s.get("remap", 0))
            self._check(nemd_batch_add(self.h, ctypes.byref(y), None))
        self._check(nemd_batch_finalize(self.h))
        ns = ctypes.c_int64()
        nemd_batch_offsets(self.h, None, ctypes.byref(ns))
        self.nsys = ns.value
        self.offsets = np.zeros(self.nsys + 1, dtype=np.int64)
        nemd_batch_offsets(self.h, self.offsets.ctypes.data, ctypes.byref(ns))
        self.ntot = int(self.offsets[-1])

    def close(self):
        if self.h:
            nemd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise NemdError(rc, nemd_batch_last_error(self.h).decode())
        return rc

    def set_state(self, q, t):
        t = np.ascontiguousarray(t, dtype=np.float64)
        self._keep["q"] = q
        self._keep["t"] = t
        return self._check(nemd_batch_set_state(self.h, _ptr(q), t.ctypes.data))

    def compute(self, F=None, UW=None):
        return self._check(nemd_batch_compute(self.h, _ptr(F), _ptr(UW)))

    def sync(self, status=False):
        st = np.zeros(self.nsys, dtype=np.int32)
        rc = nemd_batch_sync(self.h, st.ctypes.data)
        if status:
            return st
        self._check(rc)
        return st

    def set_option(self, key, value):
        return self._check(nemd_batch_set_option(self.h, int(key), int(value)))

    def stats(self):
        arr = (nemd_batch_stats * self.nsys)()
        nl = ctypes.c_int64()
        self._check(nemd_batch_get_stats(self.h, arr, ctypes.byref(nl)))
        out = [{"pairs": a.pairs, "candidates": a.candidates, "band": a.band, "counts": tuple(a.counts),
                "variant": a.variant, "cell_factor": a.cell_factor, "status": a.status} for a in arr]
        return out, nl.value

    def autotune(self, reps=3):
        times = (nemd_tune_entry * 8)()
        nt = ctypes.c_int()
        self._check(nemd_batch_autotune(self.h, int(reps), times, 8, ctypes.byref(nt)))
        return [({"tile": times[k].cfg.group, "cell_factor": times[k].cfg.cell_factor}, times[k].ms)
                for k in range(nt.value)]
