"""CPU oracle for the L.A.Cosmic detect-and-clean iteration (van Dokkum 2001).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The CUDA
product path never imports this package, and this package imports nothing
from the product package.

The arithmetic lives in ``lacos_oracle.cpp`` (plain single-threaded C++,
templated on float and double, built with ``-O2 -ffp-contract=off`` and no
fast-math).  This module only compiles it and marshals numpy arrays through
ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lacos_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liblacos_oracle.so")
_lock = threading.Lock()
_lib = None

F32, U16 = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # LACOS_ORACLE_LIB: another build of this source (the planted-slip
            # tests load mutated copies through it).
            path = os.environ.get("LACOS_ORACLE_LIB")
            if not path:
                build()
                path = _LIB
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i, f, ll = ctypes.c_int, ctypes.c_float, ctypes.c_longlong
            for suf in ("f32", "f64"):
                fn = getattr(lib, f"oracle_run_{suf}")
                fn.argtypes = [P, i, i, i, f, f, f, f, f, f, i, i, i, i, P, P, P, P, P, P]
                fn.restype = i
                fn = getattr(lib, f"oracle_estimate_gain_{suf}")
                fn.argtypes = [P, P, P, i, i, f, P, P, P]
                fn.restype = i
                fn = getattr(lib, f"oracle_iterate_{suf}")
                fn.argtypes = [P, P, i, i, f, f, f, f, f, i, P, P] + [P] * 12
                fn.restype = ll
                for name in ("lplus", "lplus_literal"):
                    fn = getattr(lib, f"oracle_{name}_{suf}")
                    fn.argtypes = [P, i, i, P]
                    fn.restype = None
                for name in ("median", "median_sep"):
                    fn = getattr(lib, f"oracle_{name}_{suf}")
                    fn.argtypes = [P, i, i, i, P]
                    fn.restype = None
                fn = getattr(lib, f"oracle_maskmed_{suf}")
                fn.argtypes = [P, P, i, i, i, i, P]
                fn.restype = i
            lib.oracle_dilate3.argtypes = [P, i, i, P]
            lib.oracle_dilate3.restype = None
            lib.oracle_dilate_square.argtypes = [P, i, i, i, P]
            lib.oracle_dilate_square.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dt(precision: str):
    return (np.float32, "f32") if precision == "f32" else (np.float64, "f64")


def run(frame: np.ndarray, gain: float, readnoise: float, satlevel: float = 65535.0,
        sigclip: float = 4.5, sigfrac: float = 0.3, objlim: float = 5.0, niter: int = 4,
        fnorm: bool = True, precision: str = "f32", satgrow: int = 0, sepmed: bool = False,
        return_gain: bool = False):
    """Full detect-and-clean loop.  Returns (mask u8, cleaned, iters_run, n_flagged),
    and with return_gain also the gain of the last iteration run and whether every
    iteration's gain estimate was defined.
    gain: 0 estimates it at every iteration (reading C15, uint16 frames only).
    satgrow: radius of the protected square around saturated pixels (reading C16).
    sepmed: both 5x5 detection medians taken separably (comparison mode, reading C17)."""
    lib = _load()
    frame = np.ascontiguousarray(frame)
    if frame.dtype == np.uint16:
        dtype = U16
    elif frame.dtype == np.float32:
        dtype = F32
    else:
        raise TypeError("frame must be float32 or uint16")
    ny, nx = frame.shape
    T, suf = _dt(precision)
    mask = np.zeros((ny, nx), np.uint8)
    clean = np.zeros((ny, nx), T)
    it = ctypes.c_int(0)
    nf = ctypes.c_longlong(0)
    g_last = ctypes.c_double(0.0)
    g_ok = ctypes.c_int(0)
    rc = getattr(lib, f"oracle_run_{suf}")(
        _ptr(frame), dtype, ny, nx, gain, readnoise, satlevel, sigclip, sigfrac, objlim,
        int(niter), int(bool(fnorm)), int(satgrow), int(bool(sepmed)), _ptr(mask), _ptr(clean), ctypes.byref(it),
        ctypes.byref(nf), ctypes.byref(g_last), ctypes.byref(g_ok))
    if rc != 0:
        raise ValueError(f"oracle_run_{suf} failed with code {rc}")
    if return_gain:
        return mask, clean, it.value, nf.value, g_last.value, bool(g_ok.value)
    return mask, clean, it.value, nf.value


def estimate_gain(I: np.ndarray, M: np.ndarray, sat: np.ndarray, readnoise: float,
                  precision: str = "f32"):
    """Reading C15 on one image: the gain estimated from the adjacent pixel pairs of I
    that M and sat leave.  Returns (gain or None when undefined, clipping rounds,
    (n, sum d, sum d^2, sum(a+b)) of the final pair set)."""
    lib = _load()
    T, suf = _dt(precision)
    I = np.ascontiguousarray(I, T)
    M = np.ascontiguousarray(M, np.uint8)
    sat = np.ascontiguousarray(sat, np.uint8)
    ny, nx = I.shape
    g = ctypes.c_double(0.0)
    rounds = ctypes.c_int(0)
    stats = np.zeros(4, np.int64)
    rc = getattr(lib, f"oracle_estimate_gain_{suf}")(_ptr(I), _ptr(M), _ptr(sat), ny, nx, readnoise,
                                                      ctypes.byref(g), ctypes.byref(rounds), _ptr(stats))
    if rc < 0:
        raise ValueError("gain estimation needs integer pixel values")
    return (g.value if rc == 1 else None), rounds.value, tuple(int(v) for v in stats)


def ingest(frame: np.ndarray, satlevel: float, precision: str = "f32"):
    """Working image X0 (with -0 -> +0) and the saturation map, as the oracle forms them."""
    T, _ = _dt(precision)
    x0 = frame.astype(T)
    x0[x0 == 0] = 0
    sat = ((satlevel > 0) & (x0 >= T(satlevel))).astype(np.uint8)
    return x0, sat


def iterate(x0: np.ndarray, sat: np.ndarray, I: np.ndarray, M: np.ndarray, gain: float,
            readnoise: float, sigclip: float, sigfrac: float, objlim: float,
            fnorm: bool = True, precision: str = "f32"):
    """One iteration; returns (new_count, I_new, M_new, dict of intermediates)."""
    lib = _load()
    T, suf = _dt(precision)
    ny, nx = x0.shape
    x0 = np.ascontiguousarray(x0, T)
    sat = np.ascontiguousarray(sat, np.uint8)
    I = np.array(I, T, copy=True, order="C")
    M = np.array(M, np.uint8, copy=True, order="C")
    names_f = ["L", "m5", "N", "S", "mS", "Sp", "m3", "m7", "F"]
    names_b = ["cand", "g1", "g2"]
    d = {k: np.zeros((ny, nx), T) for k in names_f}
    d.update({k: np.zeros((ny, nx), np.uint8) for k in names_b})
    fresh = getattr(lib, f"oracle_iterate_{suf}")(
        _ptr(x0), _ptr(sat), ny, nx, gain, readnoise, sigclip, sigfrac, objlim,
        int(bool(fnorm)), _ptr(I), _ptr(M), *[_ptr(d[k]) for k in names_f + names_b])
    return int(fresh), I, M, d


def lplus(I: np.ndarray, literal: bool = False, precision: str = "f32"):
    lib = _load()
    T, suf = _dt(precision)
    I = np.ascontiguousarray(I, T)
    out = np.zeros_like(I)
    name = "lplus_literal" if literal else "lplus"
    getattr(lib, f"oracle_{name}_{suf}")(_ptr(I), I.shape[0], I.shape[1], _ptr(out))
    return out


def median(A: np.ndarray, K: int, precision: str = "f32"):
    lib = _load()
    T, suf = _dt(precision)
    A = np.ascontiguousarray(A, T)
    out = np.zeros_like(A)
    getattr(lib, f"oracle_median_{suf}")(_ptr(A), A.shape[0], A.shape[1], int(K), _ptr(out))
    return out


def median_sep(A: np.ndarray, K: int, precision: str = "f32"):
    """Separable K x K median (median of the row medians), clamp-to-edge (C17)."""
    lib = _load()
    T, suf = _dt(precision)
    A = np.ascontiguousarray(A, T)
    out = np.zeros_like(A)
    getattr(lib, f"oracle_median_sep_{suf}")(_ptr(A), A.shape[0], A.shape[1], int(K), _ptr(out))
    return out


def dilate3(B: np.ndarray):
    lib = _load()
    B = np.ascontiguousarray(B, np.uint8)
    out = np.zeros_like(B)
    lib.oracle_dilate3(_ptr(B), B.shape[0], B.shape[1], _ptr(out))
    return out


def dilate_square(B: np.ndarray, r: int):
    """The saturated set grown by the square of radius r, inside the frame (C16)."""
    lib = _load()
    B = np.ascontiguousarray(B, np.uint8)
    out = np.zeros_like(B)
    lib.oracle_dilate_square(_ptr(B), B.shape[0], B.shape[1], int(r), _ptr(out))
    return out


def maskmed(x0: np.ndarray, M: np.ndarray, i: int, j: int, precision: str = "f32"):
    lib = _load()
    T, suf = _dt(precision)
    x0 = np.ascontiguousarray(x0, T)
    M = np.ascontiguousarray(M, np.uint8)
    out = np.zeros(1, T)
    rc = getattr(lib, f"oracle_maskmed_{suf}")(_ptr(x0), _ptr(M), x0.shape[0], x0.shape[1],
                                               int(i), int(j), _ptr(out))
    return None if rc else out[0]
