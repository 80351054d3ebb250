"""Oracle for belief propagation on pairwise MRFs -- TEST INFRASTRUCTURE.

A plain, slow, obviously correct FP64 / exact-integer implementation of
standard (dense, O(M^2)) loopy BP written from the paper's problem statement:
the message update Eq. 2 with explicit normalisation, its max-product form
Eq. 9 in energies (min-sum), and the beliefs Eq. 3.  It never uses the
constant-plus-band split of the pairwise potential (Eq. 7 / Eq. 11): the fast
method has to reproduce these results exactly.

Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It shares no code with the CUDA path.

Submodules:
  grid      4-connected grid edge lists and the message-plane layout
  stereo    the stereo model's potentials written from their definitions
  gradient  FP64 reference gradient of the log-domain loss (torch autograd
            on the dense update) and central finite differences
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, IEEE arithmetic, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I, P = ctypes.c_int, ctypes.c_void_p
            for name in ("oracle_sum_product", "oracle_min_sum"):
                fn = getattr(lib, name)
                fn.argtypes = [I, I, I, P, P, P, P, P, I, I, P]
                fn.restype = I
            for name in ("oracle_sum_beliefs", "oracle_min_beliefs"):
                fn = getattr(lib, name)
                fn.argtypes = [I, I, I, P, P, P, P]
                fn.restype = I
            lib.oracle_sum_edge_update.argtypes = [I, P, I, P, P, P]
            lib.oracle_sum_edge_update.restype = I
            lib.oracle_min_edge_update.argtypes = [I, P, I, P, P, P]
            lib.oracle_min_edge_update.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _graph(src, dst):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape or src.ndim != 1:
        raise ValueError("src and dst must be 1-D arrays of equal length")
    return src, dst


SCHEDULES = {"sync": 0, "redblack": 1, "two_colour": 1}


def sum_product(src, dst, g, F, n_iters, msg0=None, color=None, schedule="sync"):
    """Loopy sum-product BP (Eq. 2, normalised) on a directed edge list.

    g: [n_nodes][M] unary; F: [M][M] with F[x_i, x_j] = f(x_i, x_j);
    msg0: [n_edges][M] initial messages (default uniform 1/M).
    Returns the messages after n_iters iterations, [n_edges][M] float64."""
    src, dst = _graph(src, dst)
    g = np.ascontiguousarray(g, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    n, M = g.shape
    if F.shape != (M, M):
        raise ValueError("F must be M x M")
    E = src.size
    msg = (np.full((E, M), 1.0 / M) if msg0 is None else np.array(msg0, dtype=np.float64, copy=True))
    msg = np.ascontiguousarray(msg)
    col = None if color is None else np.ascontiguousarray(color, dtype=np.int32)
    rc = _load().oracle_sum_product(n, M, E, _ptr(src), _ptr(dst), _ptr(g), _ptr(F),
                                    None if col is None else _ptr(col), SCHEDULES[schedule],
                                    int(n_iters), _ptr(msg))
    if rc:
        raise ValueError("oracle_sum_product rejected its arguments or met a zero message")
    return msg


def min_sum(src, dst, Eu, V, n_iters, msg0=None, color=None, schedule="sync"):
    """Loopy min-sum BP (Eq. 9 in energies, min shifted to 0), exact int64."""
    src, dst = _graph(src, dst)
    Eu = np.ascontiguousarray(Eu, dtype=np.int64)
    V = np.ascontiguousarray(V, dtype=np.int64)
    n, M = Eu.shape
    if V.shape != (M, M):
        raise ValueError("V must be M x M")
    E = src.size
    msg = (np.zeros((E, M), dtype=np.int64) if msg0 is None else np.array(msg0, dtype=np.int64, copy=True))
    msg = np.ascontiguousarray(msg)
    col = None if color is None else np.ascontiguousarray(color, dtype=np.int32)
    rc = _load().oracle_min_sum(n, M, E, _ptr(src), _ptr(dst), _ptr(Eu), _ptr(V),
                                None if col is None else _ptr(col), SCHEDULES[schedule],
                                int(n_iters), _ptr(msg))
    if rc:
        raise ValueError("oracle_min_sum rejected its arguments")
    return msg


def sum_beliefs(dst, g, msg):
    """Normalised beliefs, Eq. 3; [n_nodes][M] float64."""
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    g = np.ascontiguousarray(g, dtype=np.float64)
    msg = np.ascontiguousarray(msg, dtype=np.float64)
    n, M = g.shape
    out = np.empty_like(g)
    if _load().oracle_sum_beliefs(n, M, dst.size, _ptr(dst), _ptr(g), _ptr(msg), _ptr(out)):
        raise ValueError("oracle_sum_beliefs failed")
    return out


def min_beliefs(dst, Eu, msg):
    """Min-sum beliefs E_i + sum of incoming messages; [n_nodes][M] int64."""
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    Eu = np.ascontiguousarray(Eu, dtype=np.int64)
    msg = np.ascontiguousarray(msg, dtype=np.int64)
    n, M = Eu.shape
    out = np.empty_like(Eu)
    if _load().oracle_min_beliefs(n, M, dst.size, _ptr(dst), _ptr(Eu), _ptr(msg), _ptr(out)):
        raise ValueError("oracle_min_beliefs failed")
    return out


def sum_edge_update(g_i, incoming, F):
    """One normalised Eq. 2 update from the unary of node i and the messages
    m_ki, k in N(i) minus j.  Returns [M] float64."""
    g_i = np.ascontiguousarray(g_i, dtype=np.float64)
    M = g_i.size
    inc = [np.ascontiguousarray(m, dtype=np.float64) for m in incoming]
    arr = (ctypes.c_void_p * max(1, len(inc)))(*[m.ctypes.data for m in inc])
    out = np.empty(M)
    F = np.ascontiguousarray(F, dtype=np.float64)
    if _load().oracle_sum_edge_update(M, _ptr(g_i), len(inc), ctypes.cast(arr, ctypes.c_void_p),
                                      _ptr(F), _ptr(out)):
        raise ValueError("zero message")
    return out


def min_edge_update(E_i, incoming, V):
    """One Eq. 9 (min-sum) update; [M] int64."""
    E_i = np.ascontiguousarray(E_i, dtype=np.int64)
    M = E_i.size
    inc = [np.ascontiguousarray(m, dtype=np.int64) for m in incoming]
    arr = (ctypes.c_void_p * max(1, len(inc)))(*[m.ctypes.data for m in inc])
    out = np.empty(M, dtype=np.int64)
    V = np.ascontiguousarray(V, dtype=np.int64)
    _load().oracle_min_edge_update(M, _ptr(E_i), len(inc), ctypes.cast(arr, ctypes.c_void_p),
                                   _ptr(V), _ptr(out))
    return out


def map_labels(belief, maximise: bool):
    """MAP label per node with the lowest-label tie-break."""
    b = np.asarray(belief)
    return (np.argmax(b, axis=-1) if maximise else np.argmin(b, axis=-1)).astype(np.int32)
