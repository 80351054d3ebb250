"""Python binding of the bpgrid C ABI (include/bp.h): argument marshalling only.

Every function below has the name of the C entry point it calls and passes
torch tensors as raw device pointers.  All arithmetic runs in the CUDA
library; there is no CPU path.  If the library has not been built the import
of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbpgrid.so")

BP_OK, BP_ERR_ARG, BP_ERR_STATE, BP_ERR_CUDA, BP_ERR_OOM, BP_ERR_POTENTIAL, BP_ERR_TIMEOUT, \
    BP_ERR_UNSUPPORTED = range(8)
BP_SUM, BP_MAX, BP_LOG, BP_RECORD = 0, 1, 2, 4
BP_SYNC, BP_REDBLACK = 0, 1
BP_F32, BP_I32 = 0, 1
BP_DENSE_CUDA_CORE, BP_DENSE_BF16_TC, BP_DENSE_BF16_TC_FUSED = 0, 1, 2
BP_SPARSE_AUTO, BP_SPARSE_LISTS, BP_SPARSE_REGISTERS = 0, 1, 2
STATUS_NAMES = {0: "BP_OK", 1: "BP_ERR_ARG", 2: "BP_ERR_STATE", 3: "BP_ERR_CUDA", 4: "BP_ERR_OOM",
                5: "BP_ERR_POTENTIAL", 6: "BP_ERR_TIMEOUT", 7: "BP_ERR_UNSUPPORTED"}
SCHEDULES = {"sync": BP_SYNC, "redblack": BP_REDBLACK}


class BPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run paper_1010_0012_gb300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    I, P, D = ctypes.c_int, ctypes.c_void_p, ctypes.c_double
    sig = {
        "bp_create": ([I, I, I, I, P, ctypes.POINTER(P)], I),
        "bp_set_unary": ([P, P], I),
        "bp_set_unary_stereo": ([P, P, P, P, I], I),
        "bp_set_unary_log": ([P, P], I),
        "bp_set_potential": ([P, P, I, D], I),
        "bp_set_potential_sparse": ([P, P, P, P, D], I),
        "bp_reset_messages": ([P], I),
        "bp_iterate": ([P, I, I, I], I),
        "bp_iterate_dense": ([P, I, I], I),
        "bp_iterate_multiscale": ([P, I, P, I, I], I),
        "bp_beliefs": ([P, P, P], I),
        "bp_get_messages": ([P, P], I),
        "bp_set_messages": ([P, P], I),
        "bp_backward": ([P, P, P, P, P], I),
        "bp_backward_device": ([P, P, P, P, P], I),
        "bp_set_checkpoint_interval": ([P, I], I),
        "bp_set_persistent": ([P, I], I),
        "bp_set_sparse_kernel": ([P, I], I),
        "bp_get_sparse_kernel": ([P, P, P, P], I),
        "bp_sparse_schedule": ([I, P, P, I, P, P, P, P, P, P], I),
        "bp_set_grid": ([P, I], I),
        "bp_sync": ([P], I),
        "bp_last_error": ([P], ctypes.c_char_p),
        "bp_destroy": ([P], None),
        "bp_set_layout": ([P, I, I], I),
        "bp_get_layout": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "bp_autotune": ([P, I, I, ctypes.POINTER(ctypes.c_float)], I),
        "bp_launch_count": ([P], ctypes.c_longlong),
        "bp_iterate_dense_tc_noalloc": ([I, I, I, P, P, P, P, I, D, P], I),
        "bp_version": ([], I),
        "bp_batch_create": ([I, P, I, P, ctypes.POINTER(P)], I),
        "bp_batch_reset_messages": ([P], I),
        "bp_batch_iterate": ([P, I, I], I),
        "bp_batch_beliefs": ([P, I, P, P], I),
        "bp_batch_get_messages": ([P, I, P], I),
        "bp_batch_set_tiling": ([P, I, I], I),
        "bp_batch_get_tiling": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "bp_batch_class_count": ([P], I),
        "bp_batch_get_class_tiling": ([P, I, P, P, P, P], I),
        "bp_batch_set_class_tiling": ([P, I, I, I, I], I),
        "bp_batch_autotune": ([P, I, I, ctypes.POINTER(ctypes.c_float)], I),
        "bp_batch_set_wait_limit": ([P, D, I], I),
        "bp_batch_sync": ([P], I),
        "bp_batch_last_error": ([P], ctypes.c_char_p),
        "bp_batch_launch_count": ([P], ctypes.c_longlong),
        "bp_batch_destroy": ([P], None),
        "bp_fg_create": ([I, I, I, P, I, P, ctypes.POINTER(P)], I),
        "bp_fg_set_unary": ([P, P], I),
        "bp_fg_set_factor": ([P, I, P, P, D], I),
        "bp_fg_reset_messages": ([P], I),
        "bp_fg_iterate": ([P, I, I], I),
        "bp_fg_iterate_dense": ([P, I, I], I),
        "bp_fg_beliefs": ([P, P, P], I),
        "bp_fg_get_messages": ([P, P], I),
        "bp_fg_sync": ([P], I),
        "bp_fg_last_error": ([P], ctypes.c_char_p),
        "bp_fg_launch_count": ([P], ctypes.c_longlong),
        "bp_fg_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(h, st):
    if st != BP_OK:
        raise BPError(st, _lib.bp_last_error(h).decode())


def _dptr(t: torch.Tensor, dtype, numel=None):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---- one function per C entry point -------------------------------------------

def bp_version():
    return _lib.bp_version()


def bp_create(W, H, M, dtype=BP_F32, stream=None):
    h = ctypes.c_void_p()
    st = _lib.bp_create(W, H, M, dtype, _stream_ptr(stream), ctypes.byref(h))
    _check(None, st)
    return h


def bp_destroy(h):
    _lib.bp_destroy(h)


def bp_set_unary(h, unary: torch.Tensor, dtype):
    _check(h, _lib.bp_set_unary(h, _dptr(unary, torch.float32 if dtype == BP_F32 else torch.int32)))


def _image_ptr(t: torch.Tensor):
    """A [H][W] uint8 image on the device or in host memory (the library
    copies host images itself)."""
    if t.is_cuda:
        return _dptr(t, torch.uint8)
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise TypeError("expected a contiguous uint8 image")
    return ctypes.c_void_p(t.data_ptr())


def bp_set_unary_stereo(h, left: torch.Tensor, right: torch.Tensor, table, Tu: int, dtype):
    """left, right: [H][W] uint8 images, on the device or in (preferably
    pinned) host memory; table: Tu + 1 values indexed by the matching cost
    (float32 g or int32 E_u by the handle's dtype)."""
    import numpy as np
    arr = np.ascontiguousarray(table, dtype=np.float32 if dtype == BP_F32 else np.int32)
    if arr.size != Tu + 1:
        raise ValueError("table must hold Tu + 1 values")
    _check(h, _lib.bp_set_unary_stereo(h, _image_ptr(left), _image_ptr(right),
                                       arr.ctypes.data_as(ctypes.c_void_p), int(Tu)))


def bp_set_unary_log(h, logg: torch.Tensor):
    _check(h, _lib.bp_set_unary_log(h, _dptr(logg, torch.float32)))


def bp_set_potential(h, table, T: int, fbar: float, dtype):
    import numpy as np
    arr = np.ascontiguousarray(table, dtype=np.float32 if dtype == BP_F32 else np.int32)
    if arr.size != 2 * T + 1:
        raise ValueError("table must hold 2T + 1 values")
    _check(h, _lib.bp_set_potential(h, arr.ctypes.data_as(ctypes.c_void_p), int(T), float(fbar)))


def bp_set_potential_sparse(h, rowptr, cols, vals, fbar: float, dtype):
    """CSR over receiver labels: cols[rowptr[xj]:rowptr[xj+1]] are the
    compatible sender labels of xj, vals their f (or E)."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(cols, dtype=np.int32)
    vl = np.ascontiguousarray(vals, dtype=np.float32 if dtype == BP_F32 else np.int32)
    if cl.size != vl.size or rp[-1] != cl.size:
        raise ValueError("rowptr[-1] must equal len(cols) == len(vals)")
    _check(h, _lib.bp_set_potential_sparse(h, rp.ctypes.data_as(ctypes.c_void_p),
                                           cl.ctypes.data_as(ctypes.c_void_p) if cl.size else None,
                                           vl.ctypes.data_as(ctypes.c_void_p), float(fbar)))


def bp_reset_messages(h):
    _check(h, _lib.bp_reset_messages(h))


def bp_iterate(h, n_iters, mode=BP_SUM, schedule=BP_SYNC):
    _check(h, _lib.bp_iterate(h, int(n_iters), int(mode), int(schedule)))


def bp_iterate_multiscale(h, iters, mode=BP_SUM, schedule=BP_SYNC):
    """iters: iteration counts per level, coarsest first (last = this grid)."""
    import numpy as np
    it = np.ascontiguousarray(iters, dtype=np.int32)
    _check(h, _lib.bp_iterate_multiscale(h, int(it.size), it.ctypes.data_as(ctypes.c_void_p), int(mode),
                                         int(SCHEDULES.get(schedule, schedule))))


def bp_iterate_dense(h, n_iters, kind=BP_DENSE_CUDA_CORE):
    _check(h, _lib.bp_iterate_dense(h, int(n_iters), int(kind)))


def bp_beliefs(h, out: torch.Tensor, map_out: Optional[torch.Tensor] = None):
    mp = None if map_out is None else _dptr(map_out, torch.int32)
    _check(h, _lib.bp_beliefs(h, ctypes.c_void_p(out.data_ptr()), mp))


def bp_get_messages(h, planes: torch.Tensor):
    _check(h, _lib.bp_get_messages(h, ctypes.c_void_p(planes.data_ptr())))


def bp_set_messages(h, planes: torch.Tensor):
    if not planes.is_contiguous() or not planes.is_cuda:
        raise ValueError("expected a contiguous CUDA tensor")
    _check(h, _lib.bp_set_messages(h, ctypes.c_void_p(planes.data_ptr())))


def bp_backward(h, dlogb: torch.Tensor, dlogg: torch.Tensor, n_table: int):
    import numpy as np
    dtab = np.zeros(n_table, dtype=np.float64)
    dfbar = ctypes.c_double(0.0)
    _check(h, _lib.bp_backward(h, _dptr(dlogb, torch.float32), _dptr(dlogg, torch.float32),
                               dtab.ctypes.data_as(ctypes.c_void_p), ctypes.byref(dfbar)))
    return dtab, dfbar.value


def bp_backward_device(h, dlogb: torch.Tensor, dlogg: torch.Tensor, dtab: torch.Tensor, dfbar: torch.Tensor):
    """bp_backward with dL/df(d) and dL/dfbar written into float64 CUDA tensors
    on the handle's stream (no synchronisation)."""
    _check(h, _lib.bp_backward_device(h, _dptr(dlogb, torch.float32), _dptr(dlogg, torch.float32),
                                      _dptr(dtab, torch.float64), _dptr(dfbar, torch.float64, 1)))


def bp_set_checkpoint_interval(h, every):
    _check(h, _lib.bp_set_checkpoint_interval(h, int(every)))


def bp_set_grid(h, blocks):
    _check(h, _lib.bp_set_grid(h, int(blocks)))


def bp_set_persistent(h, mode):
    _check(h, _lib.bp_set_persistent(h, int(mode)))


def bp_set_sparse_kernel(h, kind):
    _check(h, _lib.bp_set_sparse_kernel(h, int(kind)))


def bp_sparse_schedule(M, rowptr, cols, gather_bytes=16):
    """The register kernel's schedule of a CSR pattern (host only) for 16-byte
    (FP32 / int32) or 8-byte (16-bit min-sum) gathers: dict with KM, LM,
    steps, wavefronts, lab [KM][32] and ent [KM][LM][32][2] (byte offset of
    the h slot or 0xFFFF, CSR position), or None without one."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(cols, dtype=np.int32)
    v = [ctypes.c_int() for _ in range(4)]
    vp = rp.ctypes.data_as(ctypes.c_void_p)
    cp = cl.ctypes.data_as(ctypes.c_void_p) if cl.size else None
    _check(None, _lib.bp_sparse_schedule(int(M), vp, cp, int(gather_bytes), *[ctypes.byref(x) for x in v], None, None))
    KM, LM, steps, wf = (x.value for x in v)
    if KM == 0:
        return None
    lab = np.empty((KM, 32), np.int32)
    ent = np.empty((KM, LM, 32, 2), np.int32)
    _check(None, _lib.bp_sparse_schedule(int(M), vp, cp, int(gather_bytes), *[ctypes.byref(x) for x in v],
                                         lab.ctypes.data_as(ctypes.c_void_p), ent.ctypes.data_as(ctypes.c_void_p)))
    return {"KM": KM, "LM": LM, "steps": steps, "wavefronts": wf, "lab": lab, "ent": ent}


def bp_get_sparse_kernel(h):
    """(kernel in use, steps per block, gather wavefronts per node)."""
    k, st, wf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(h, _lib.bp_get_sparse_kernel(h, ctypes.byref(k), ctypes.byref(st), ctypes.byref(wf)))
    return k.value, st.value, wf.value


def bp_sync(h):
    _check(h, _lib.bp_sync(h))


def bp_last_error(h=None):
    return _lib.bp_last_error(h).decode()


def bp_set_layout(h, L, C):
    _check(h, _lib.bp_set_layout(h, int(L), int(C)))


def bp_get_layout(h):
    L, C = ctypes.c_int(), ctypes.c_int()
    _check(h, _lib.bp_get_layout(h, ctypes.byref(L), ctypes.byref(C)))
    return L.value, C.value


def bp_autotune(h, mode, n_iters=3):
    ms = ctypes.c_float(0.0)
    _check(h, _lib.bp_autotune(h, int(mode), int(n_iters), ctypes.byref(ms)))
    return ms.value


def bp_launch_count(h):
    return _lib.bp_launch_count(h)


def bp_iterate_dense_tc_noalloc(W, H, M, unary: torch.Tensor, in_planes: torch.Tensor, out_planes: torch.Tensor,
                                table, T: int, fbar: float, stream=None):
    """One dense tensor-core iteration that allocates nothing (see include/bp.h)."""
    import numpy as np
    tab = np.ascontiguousarray(table, dtype=np.float32)
    if tab.size != 2 * T + 1:
        raise ValueError("table must hold 2T + 1 values")
    st = _lib.bp_iterate_dense_tc_noalloc(int(W), int(H), int(M), _dptr(unary, torch.float32, H * W * M),
                                          _dptr(in_planes, torch.float32, 4 * H * W * M),
                                          _dptr(out_planes, torch.float32, 4 * H * W * M),
                                          tab.ctypes.data_as(ctypes.c_void_p), int(T), float(fbar),
                                          _stream_ptr(stream))
    _check(None, st)


# ---- batches ---------------------------------------------------------------------

class bp_mrf_desc(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("M", ctypes.c_int), ("T", ctypes.c_int),
                ("dev_unary", ctypes.c_void_p), ("host_table", ctypes.c_void_p), ("fbar", ctypes.c_double)]


def _bcheck(b, st):
    if st != BP_OK:
        raise BPError(st, _lib.bp_batch_last_error(b).decode())


def bp_batch_create(mrfs, dtype, stream=None):
    """mrfs: list of (unary tensor [H][W][M], table, T, fbar)."""
    import numpy as np
    descs = (bp_mrf_desc * len(mrfs))()
    keep = []
    for i, (un, table, T, fbar) in enumerate(mrfs):
        Hh, W, M = un.shape
        tab = np.ascontiguousarray(table, dtype=np.float32 if dtype == BP_F32 else np.int32)
        if tab.size != 2 * T + 1:
            raise ValueError("table must hold 2T + 1 values")
        keep.append(tab)
        descs[i] = bp_mrf_desc(W, Hh, M, T, _dptr(un, torch.float32 if dtype == BP_F32 else torch.int32).value,
                               tab.ctypes.data, float(fbar))
    b = ctypes.c_void_p()
    st = _lib.bp_batch_create(len(mrfs), descs, dtype, _stream_ptr(stream), ctypes.byref(b))
    _bcheck(None, st)
    return b


def bp_batch_reset_messages(b):
    _bcheck(b, _lib.bp_batch_reset_messages(b))


def bp_batch_iterate(b, n_iters, mode):
    _bcheck(b, _lib.bp_batch_iterate(b, int(n_iters), int(mode)))


def bp_batch_beliefs(b, k, out: torch.Tensor, map_out: Optional[torch.Tensor] = None):
    mp = None if map_out is None else _dptr(map_out, torch.int32)
    _bcheck(b, _lib.bp_batch_beliefs(b, int(k), ctypes.c_void_p(out.data_ptr()), mp))


def bp_batch_get_messages(b, k, planes: torch.Tensor):
    _bcheck(b, _lib.bp_batch_get_messages(b, int(k), ctypes.c_void_p(planes.data_ptr())))


def bp_batch_set_tiling(b, family, tile_words):
    _bcheck(b, _lib.bp_batch_set_tiling(b, int(family), int(tile_words)))


def bp_batch_get_tiling(b):
    f, t = ctypes.c_int(), ctypes.c_int()
    _bcheck(b, _lib.bp_batch_get_tiling(b, ctypes.byref(f), ctypes.byref(t)))
    return f.value, t.value


def bp_batch_class_count(b):
    return _lib.bp_batch_class_count(b)


def bp_batch_get_class_tiling(b, k):
    """(Mp, T, family, tile_words) of class k."""
    v = [ctypes.c_int() for _ in range(4)]
    _bcheck(b, _lib.bp_batch_get_class_tiling(b, int(k), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def bp_batch_set_class_tiling(b, Mp, T, family, tile_words):
    _bcheck(b, _lib.bp_batch_set_class_tiling(b, int(Mp), int(T), int(family), int(tile_words)))


def bp_batch_autotune(b, mode, n_iters=3):
    ms = ctypes.c_float(0.0)
    _bcheck(b, _lib.bp_batch_autotune(b, int(mode), int(n_iters), ctypes.byref(ms)))
    return ms.value


def bp_batch_set_wait_limit(b, seconds, extra_arrivals=0):
    _bcheck(b, _lib.bp_batch_set_wait_limit(b, float(seconds), int(extra_arrivals)))


def bp_batch_sync(b):
    _bcheck(b, _lib.bp_batch_sync(b))


def bp_batch_last_error(b=None):
    return _lib.bp_batch_last_error(b).decode()


def bp_batch_launch_count(b):
    return _lib.bp_batch_launch_count(b)


def bp_batch_destroy(b):
    _lib.bp_batch_destroy(b)


# ---- factor graphs ------------------------------------------------------------------

def _fcheck(g, st):
    if st != BP_OK:
        raise BPError(st, _lib.bp_fg_last_error(g).decode())


def bp_fg_create(n_vars, M, factor_vars, dtype, stream=None):
    import numpy as np
    fv = np.ascontiguousarray(factor_vars, dtype=np.int32).reshape(-1, 3)
    g = ctypes.c_void_p()
    st = _lib.bp_fg_create(int(n_vars), int(M), int(fv.shape[0]), fv.ctypes.data_as(ctypes.c_void_p), int(dtype),
                           _stream_ptr(stream), ctypes.byref(g))
    _fcheck(None, st)
    return g


def bp_fg_set_unary(g, unary: torch.Tensor):
    _fcheck(g, _lib.bp_fg_set_unary(g, ctypes.c_void_p(unary.data_ptr())))


def bp_fg_set_factor(g, triplets, vals, fbar, dtype):
    import numpy as np
    t = np.ascontiguousarray(triplets, dtype=np.int32).reshape(-1, 3)
    v = np.ascontiguousarray(vals, dtype=np.float32 if dtype == BP_F32 else np.int32)
    if v.size != t.shape[0]:
        raise ValueError("one value per triplet")
    _fcheck(g, _lib.bp_fg_set_factor(g, int(t.shape[0]), t.ctypes.data_as(ctypes.c_void_p),
                                     v.ctypes.data_as(ctypes.c_void_p), float(fbar)))


def bp_fg_reset_messages(g):
    _fcheck(g, _lib.bp_fg_reset_messages(g))


def bp_fg_iterate(g, n_iters, mode):
    _fcheck(g, _lib.bp_fg_iterate(g, int(n_iters), int(mode)))


def bp_fg_iterate_dense(g, n_iters, mode):
    _fcheck(g, _lib.bp_fg_iterate_dense(g, int(n_iters), int(mode)))


def bp_fg_beliefs(g, out: torch.Tensor, map_out: Optional[torch.Tensor] = None):
    mp = None if map_out is None else _dptr(map_out, torch.int32)
    _fcheck(g, _lib.bp_fg_beliefs(g, ctypes.c_void_p(out.data_ptr()), mp))


def bp_fg_get_messages(g, out: torch.Tensor):
    _fcheck(g, _lib.bp_fg_get_messages(g, ctypes.c_void_p(out.data_ptr())))


def bp_fg_sync(g):
    _fcheck(g, _lib.bp_fg_sync(g))


def bp_fg_last_error(g=None):
    return _lib.bp_fg_last_error(g).decode()


def bp_fg_launch_count(g):
    return _lib.bp_fg_launch_count(g)


def bp_fg_destroy(g):
    _lib.bp_fg_destroy(g)


# ---- a thin owner of one handle -------------------------------------------------

class BPGrid:
    """One H x W grid with M labels; wraps a bp_handle (no arithmetic here)."""

    def __init__(self, W, H, M, dtype=BP_F32, stream=None):
        self.W, self.H, self.M, self.dtype = W, H, M, dtype
        self.T = None
        self.stream = stream          # the torch stream the handle orders its work on, or None
        self.h = bp_create(W, H, M, dtype, stream)

    def on_current_stream(self):
        """True when the handle's work is ordered on torch's current stream."""
        return self.stream is not None and self.stream == torch.cuda.current_stream()

    def close(self):
        if self.h is not None:
            bp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def tdtype(self):
        return torch.float32 if self.dtype == BP_F32 else torch.int32

    def set_unary(self, unary: torch.Tensor):
        if tuple(unary.shape) != (self.H, self.W, self.M):
            raise ValueError("unary must be [H][W][M]")
        bp_set_unary(self.h, unary, self.dtype)

    def set_unary_stereo(self, left: torch.Tensor, right: torch.Tensor, table, Tu: int):
        if tuple(left.shape) != (self.H, self.W) or tuple(right.shape) != (self.H, self.W):
            raise ValueError("images must be [H][W]")
        bp_set_unary_stereo(self.h, left, right, table, Tu, self.dtype)

    def set_potential(self, table, T, fbar):
        bp_set_potential(self.h, table, T, fbar, self.dtype)
        self.T = T

    def reset(self):
        bp_reset_messages(self.h)

    def iterate(self, n, mode=None, schedule="sync"):
        if mode is None:
            mode = BP_SUM if self.dtype == BP_F32 else BP_MAX
        bp_iterate(self.h, n, mode, SCHEDULES.get(schedule, schedule))

    def iterate_dense(self, n, kind=BP_DENSE_CUDA_CORE):
        bp_iterate_dense(self.h, n, kind)

    def beliefs(self, with_map=True):
        out = torch.empty((self.H, self.W, self.M), dtype=self.tdtype, device="cuda")
        mp = torch.empty((self.H, self.W), dtype=torch.int32, device="cuda") if with_map else None
        bp_beliefs(self.h, out, mp)
        return (out, mp) if with_map else out

    def get_messages(self):
        out = torch.empty((4, self.H, self.W, self.M), dtype=self.tdtype, device="cuda")
        bp_get_messages(self.h, out)
        return out

    def set_messages(self, planes: torch.Tensor):
        if tuple(planes.shape) != (4, self.H, self.W, self.M) or planes.dtype != self.tdtype:
            raise ValueError("planes must be [4][H][W][M] of the handle's dtype")
        bp_set_messages(self.h, planes)

    def sync(self):
        bp_sync(self.h)

    @property
    def launches(self):
        return bp_launch_count(self.h)
