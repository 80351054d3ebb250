"""CPU throughput baselines -- MEASUREMENT INFRASTRUCTURE.

FP32 O(mM) (Eq. 7) and O(M^2) (Eq. 2) synchronous sum-product iterations on
the host cores, OpenMP over grid rows: the CPU comparison of Sec. 6, made on
the machine that holds the GPU.  Only `bench.py` and `tests/` use this
package.  It is neither the oracle nor a fallback of the CUDA library, and it
shares no code with either.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_cpu.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbpcpu.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """gcc -O3 with OpenMP (without it if the compiler lacks OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp]
        try:
            subprocess.check_call(base[:5] + ["-fopenmp"] + base[5:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I, P, F = ctypes.c_int, ctypes.c_void_p, ctypes.c_float
            lib.cpu_threads.argtypes = []
            lib.cpu_threads.restype = I
            lib.cpu_band_iteration.argtypes = [I, I, I, P, P, P, P, I, F, I, I, I]
            lib.cpu_band_iteration.restype = I
            lib.cpu_dense_iteration.argtypes = [I, I, I, P, P, P, P, I, I, I]
            lib.cpu_dense_iteration.restype = I
            _lib = lib
    return _lib


def threads() -> int:
    """Threads an OpenMP region uses by default (1 without OpenMP)."""
    return int(_load().cpu_threads())


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def band_iteration(g, planes_in, planes_out, table, T, fbar, rows=None, n_threads=0):
    """One FP32 O(mM) iteration: nodes of rows [lo, hi) write their outgoing
    messages into planes_out (float32 [4][H][W][M], modified in place)."""
    H, W, M = g.shape
    g = _f32(g)
    pin = _f32(planes_in, (4, H, W, M))
    if planes_out.dtype != np.float32 or not planes_out.flags.c_contiguous or planes_out.shape != (4, H, W, M):
        raise ValueError("planes_out must be a C-contiguous float32 [4][H][W][M] array")
    tab = _f32(table, (2 * T + 1,))
    lo, hi = (0, H) if rows is None else rows
    if _load().cpu_band_iteration(W, H, M, _p(g), _p(pin), _p(planes_out), _p(tab), T, float(fbar),
                                  lo, hi, n_threads):
        raise ValueError("cpu_band_iteration: bad arguments")


def dense_iteration(g, planes_in, planes_out, F, rows=None, n_threads=0):
    """One FP32 O(M^2) iteration with the full table F[x_i][x_j]."""
    H, W, M = g.shape
    g = _f32(g)
    pin = _f32(planes_in, (4, H, W, M))
    if planes_out.dtype != np.float32 or not planes_out.flags.c_contiguous or planes_out.shape != (4, H, W, M):
        raise ValueError("planes_out must be a C-contiguous float32 [4][H][W][M] array")
    F = _f32(F, (M, M))
    lo, hi = (0, H) if rows is None else rows
    if _load().cpu_dense_iteration(W, H, M, _p(g), _p(pin), _p(planes_out), _p(F), lo, hi, n_threads):
        raise ValueError("cpu_dense_iteration: bad arguments")


def messages_sent(W, H, rows):
    """Directed messages the nodes of rows [lo, hi) send (one update per label each)."""
    lo, hi = rows
    n = 0
    for r in range(lo, hi):
        n += 2 * (W - 1)                       # left and right
        n += W * ((r > 0) + (r < H - 1))       # up and down
    return n
