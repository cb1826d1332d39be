"""FP64 CPU oracle for the RIME predict + weighted chi^2 (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It loads ``librime_oracle.so`` (built from
``rime_oracle.c`` by ``oracle.build``), which shares no code with the CUDA
library.  Every function here only marshals numpy arrays into the C oracle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.environ.get("RIME_ORACLE_LIB") or os.path.join(_HERE, "librime_oracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [
        ("na", C.c_int), ("ntime", C.c_int), ("nchan", C.c_int), ("nsrc", C.c_int),
        ("stokes_time_varying", C.c_int),
        ("ref_freq_hz", C.c_double), ("beam_c", C.c_double), ("beam_model", C.c_int),
        ("uvw", _dp), ("freq_hz", _dp), ("lm", _dp), ("stokes", _dp),
        ("alpha", _dp), ("shape", _dp), ("kind", _ip), ("pointing", _dp), ("gains", _dp),
        ("data", _dp), ("weight", _dp),
    ]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            from . import build
            build.build()
        L = C.CDLL(_LIB_PATH)
        L.rime_oracle_vis.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_int, C.c_int, _dp]
        L.rime_oracle_vis_list.argtypes = [C.POINTER(_Problem), C.c_long, _ip, _ip, _ip, _ip, _dp]
        L.rime_oracle_predict.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, _dp]
        L.rime_oracle_chi2.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int]
        L.rime_oracle_chi2.restype = C.c_double
        L.rime_oracle_chi2_grad.argtypes = [C.POINTER(_Problem), _dp, _dp]
        L.rime_oracle_chi2_grad.restype = C.c_double
        L.rime_oracle_ln_norm.argtypes = [C.POINTER(_Problem)]
        L.rime_oracle_ln_norm.restype = C.c_double
        L.rime_oracle_threads.restype = C.c_int
        L.rime_oracle_reduced_phase.argtypes = [C.c_long, _dp, _dp, _dp]
        _lib = L
    return _lib


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


def _cplx_as_f64(x):
    if x is None:
        return None
    x = np.ascontiguousarray(x, dtype=np.complex128)
    return x.view(np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


class Problem:
    """Holds contiguous float64 copies of one problem's arrays.

    inp: dict with na, ntime, nchan, ref_freq_hz, beam_c, beam_model
         (optional: 0 cos^3, 1 Jinc), uvw, freq,
         pointing, sources{lm, stokes, alpha, shape}, gains, weight and
         optionally data (complex, [ntime][nbl][nchan][4]).
    """

    def __init__(self, inp: dict, sources: dict | None = None, data=None):
        src = inp["sources"] if sources is None else sources
        self._keep = {
            "uvw": _f64(inp["uvw"]), "freq": _f64(inp["freq"]),
            "lm": _f64(src["lm"]), "stokes": _f64(src["stokes"]),
            "alpha": _f64(src["alpha"]),
            "shape": _f64(src.get("shape")),
            "kind": None if src.get("kind") is None else np.ascontiguousarray(src["kind"], dtype=np.int32),
            "pointing": _f64(inp.get("pointing")),
            "gains": _cplx_as_f64(inp.get("gains")),
            "data": _cplx_as_f64(inp.get("data") if data is None else data),
            "weight": _f64(inp.get("weight")),
        }
        k = self._keep
        nsrc = k["alpha"].shape[0]
        tv = 1 if k["stokes"].ndim == 3 else 0
        self.na, self.ntime, self.nchan, self.nsrc = inp["na"], inp["ntime"], inp["nchan"], nsrc
        self.nbl = self.na * (self.na - 1) // 2
        self.s = _Problem(
            self.na, self.ntime, self.nchan, nsrc, tv,
            float(inp["ref_freq_hz"]), float(inp["beam_c"]), int(inp.get("beam_model", 0)),
            _ptr(k["uvw"]), _ptr(k["freq"]), _ptr(k["lm"]), _ptr(k["stokes"]),
            _ptr(k["alpha"]), _ptr(k["shape"]),
            k["kind"].ctypes.data_as(_ip) if k["kind"] is not None else None, _ptr(k["pointing"]),
            _ptr(k["gains"]), _ptr(k["data"]), _ptr(k["weight"]))

    # ---- calls -----------------------------------------------------------
    def vis(self, t, p, q, k) -> np.ndarray:
        out = np.zeros(8)
        lib().rime_oracle_vis(C.byref(self.s), t, p, q, k, _ptr(out))
        return out.view(np.complex128)

    def vis_list(self, t, p, q, k) -> np.ndarray:
        t, p, q, k = (np.ascontiguousarray(a, dtype=np.int32) for a in (t, p, q, k))
        n = t.shape[0]
        out = np.zeros((n, 8))
        lib().rime_oracle_vis_list(C.byref(self.s), n, t.ctypes.data_as(_ip),
                                   p.ctypes.data_as(_ip), q.ctypes.data_as(_ip),
                                   k.ctypes.data_as(_ip), _ptr(out))
        return out.view(np.complex128).reshape(n, 4)

    def predict(self, t0=0, t1=None) -> np.ndarray:
        t1 = self.ntime if t1 is None else t1
        out = np.zeros((t1 - t0, self.nbl, self.nchan, 8))
        lib().rime_oracle_predict(C.byref(self.s), t0, t1, _ptr(out))
        return out.view(np.complex128).reshape(t1 - t0, self.nbl, self.nchan, 4)

    def chi2(self, t0=0, t1=None) -> float:
        if self._keep["data"] is None:
            raise ValueError("chi2 needs observed data")
        t1 = self.ntime if t1 is None else t1
        return lib().rime_oracle_chi2(C.byref(self.s), t0, t1)

    def chi2_grad(self, want_gains=True):
        gs = np.zeros((self.nsrc, 10))
        gg = np.zeros((self.ntime, self.na, self.nchan, 4, 2)) if want_gains else None
        chi = lib().rime_oracle_chi2_grad(C.byref(self.s), _ptr(gs), _ptr(gg))
        if gg is not None:
            gg = gg.view(np.complex128).reshape(self.ntime, self.na, self.nchan, 4)
        return chi, gs, gg

    def ln_norm(self) -> float:
        return lib().rime_oracle_ln_norm(C.byref(self.s))


def threads() -> int:
    return lib().rime_oracle_threads()


def reduced_phase(nu, tau) -> np.ndarray:
    """nu tau - round(nu tau) in turns (eq. 3's phase modulo whole turns), FP64."""
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    out = np.zeros(nu.shape)
    lib().rime_oracle_reduced_phase(int(nu.size), _ptr(nu), _ptr(tau), _ptr(out))
    return out
