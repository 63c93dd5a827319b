"""Thin ctypes binding of libtga (the C-ABI declared in include/tga.h).

Functions keep the C names (``tga_create``, ``tga_build_attrs``,
``tga_eval_best_move``, ``tga_apply_move``, ``tga_descend``,
``tga_descend_batch``, ...) and only marshal arguments: every step of the
local search runs in the CUDA kernels of libtga.so.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if libtga.so is missing or no
GPU is present, calls raise.

``LocalSearch`` is a convenience wrapper that owns the device copies of one
instance + solution (torch tensors) and one context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TGA_INDEX_CHECKS=1 loads the index-checked build of the same sources
LIB_PATH = os.path.join(_HERE, "libtga_check.so" if os.environ.get("TGA_INDEX_CHECKS") == "1" else "libtga.so")

TGA_OK, TGA_ERR_INVALID, TGA_ERR_RANGE, TGA_ERR_NOMEM, TGA_ERR_CUDA = 0, 1, 2, 3, 4
TGA_ERR_TIMEOUT, TGA_ERR_STATE, TGA_ERR_CHECK, TGA_ERR_BOUNDS = 5, 6, 7, 8
DESCENT_AUTO, DESCENT_PERSISTENT, DESCENT_GRAPH, DESCENT_HOST = 0, 1, 2, 3
DESCENT_NAMES = {0: "auto", 1: "persistent", 2: "graph", 3: "host"}
NO_MOVE_KEY = (1 << 64) - 1


class TGAError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = _lib().tga_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: libtga error {code} ({msg})")


class tga_instance(ctypes.Structure):
    _fields_ = [("n_customers", ctypes.c_int32), ("n_routes", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("has_tw", ctypes.c_int32),
                ("w_load", ctypes.c_int32), ("w_tw", ctypes.c_int32),
                ("dist", ctypes.c_void_p), ("demand", ctypes.c_void_p),
                ("service", ctypes.c_void_p), ("tw_early", ctypes.c_void_p),
                ("tw_late", ctypes.c_void_p), ("pickup", ctypes.c_void_p)]


class tga_solution(ctypes.Structure):
    _fields_ = [("tour", ctypes.c_void_p), ("route_start", ctypes.c_void_p)]


class tga_move(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_int32), ("move_index", ctypes.c_uint32),
                ("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32),
                ("valid", ctypes.c_int32)]


class tga_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("initial_cost", ctypes.c_int64), ("final_cost", ctypes.c_int64),
                ("status", ctypes.c_int32), ("local_optimum", ctypes.c_int32),
                ("evaluations", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) of every exported entry point in include/tga.h
_P = ctypes.c_void_p
EXPORTS = [
    ("tga_create", ctypes.c_int, [ctypes.POINTER(tga_instance), ctypes.POINTER(tga_solution),
                                  ctypes.c_uint32, _P, ctypes.POINTER(_P)]),
    ("tga_build_attrs", ctypes.c_int, [_P]),
    ("tga_eval_best_move", ctypes.c_int, [_P, _P]),
    ("tga_apply_move", ctypes.c_int, [_P, _P]),
    ("tga_descend", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(tga_stats)]),
    ("tga_descend_batch", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64,
                                         ctypes.POINTER(tga_stats)]),
    ("tga_batch_autotune", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]),
    ("tga_descend_async", ctypes.c_int, [_P, ctypes.c_int64]),
    ("tga_query", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    ("tga_workspace_bytes", ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    ("tga_sync", ctypes.c_int, [_P]),
    ("tga_get_stats", ctypes.c_int, [_P, ctypes.POINTER(tga_stats)]),
    ("tga_set_move_log", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("tga_set_granular", ctypes.c_int, [_P, _P, ctypes.c_int32]),
    ("tga_get_op_candidates", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    ("tga_set_tile", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("tga_get_tile", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("tga_eval_best_move_noalloc", ctypes.c_int, [ctypes.POINTER(tga_instance), ctypes.POINTER(tga_solution),
                                                  ctypes.c_uint32, _P, _P]),
    ("tga_profile_inter", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    ("tga_profile_xswap", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    ("tga_measure_int_peak", ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_float)]),
    ("tga_set_descent_mode", ctypes.c_int, [_P, ctypes.c_int32]),
    ("tga_get_descent_mode", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("tga_get_persistent_shape", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(ctypes.c_int32)]),
    ("tga_set_tile_shape", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("tga_get_tile_shape", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    ("tga_debug_read", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t)]),
    ("tga_set_wait_limit", ctypes.c_int, [_P, ctypes.c_int64]),
    ("tga_get_bounds_report", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    ("tga_set_persistent_shape", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("tga_set_tile_strip", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("tga_destroy", ctypes.c_int, [_P]),
    ("tga_strerror", ctypes.c_char_p, [ctypes.c_int]),
]

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtga.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in EXPORTS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(rc, where):
    if rc != TGA_OK:
        raise TGAError(rc, where)


# ---------------------------------------------------------------------------
# C-ABI wrappers (same names)

def tga_create(inst: tga_instance, sol: tga_solution, op_mask: int, stream: int = 0) -> int:
    out = _P()
    _check(_lib().tga_create(ctypes.byref(inst), ctypes.byref(sol), op_mask, _P(stream or None),
                             ctypes.byref(out)), "tga_create")
    return out.value


def tga_build_attrs(ctx: int):
    _check(_lib().tga_build_attrs(_P(ctx)), "tga_build_attrs")


def tga_eval_best_move(ctx: int, out_dev_ptr: int):
    _check(_lib().tga_eval_best_move(_P(ctx), _P(out_dev_ptr)), "tga_eval_best_move")


def tga_apply_move(ctx: int, move_dev_ptr: int):
    _check(_lib().tga_apply_move(_P(ctx), _P(move_dev_ptr)), "tga_apply_move")


def tga_descend(ctx: int, max_steps: int = (1 << 62)) -> dict:
    st = tga_stats()
    _check(_lib().tga_descend(_P(ctx), max_steps, ctypes.byref(st)), "tga_descend")
    return st.as_dict()


def tga_descend_batch(ctxs, max_steps: int = (1 << 62)):
    arr = (_P * len(ctxs))(*[_P(c) for c in ctxs])
    stats = (tga_stats * len(ctxs))()
    _check(_lib().tga_descend_batch(arr, len(ctxs), max_steps, stats), "tga_descend_batch")
    return [s.as_dict() for s in stats]


def tga_batch_autotune(ctxs):
    arr = (_P * len(ctxs))(*[_P(c) for c in ctxs])
    rows = (ctypes.c_int32 * len(ctxs))()
    _check(_lib().tga_batch_autotune(arr, len(ctxs), rows), "tga_batch_autotune")
    return list(rows)


def tga_descend_async(ctx: int, max_steps: int = (1 << 62)):
    _check(_lib().tga_descend_async(_P(ctx), max_steps), "tga_descend_async")


def tga_query(ctx: int) -> bool:
    done = ctypes.c_int32()
    _check(_lib().tga_query(_P(ctx), ctypes.byref(done)), "tga_query")
    return bool(done.value)


def tga_workspace_bytes(n: int, m: int) -> int:
    return int(_lib().tga_workspace_bytes(n, m))


def tga_sync(ctx: int):
    _check(_lib().tga_sync(_P(ctx)), "tga_sync")


def tga_get_stats(ctx: int) -> dict:
    st = tga_stats()
    _check(_lib().tga_get_stats(_P(ctx), ctypes.byref(st)), "tga_get_stats")
    return st.as_dict()


def tga_get_op_candidates(ctx: int):
    """Candidates evaluated per operator rank (8 ints: relocate, swap, 2-opt,
    2-opt*, or-opt 2, or-opt 3, customer/run-of-two swap, run/run swap) over
    all evaluations."""
    out = (ctypes.c_int64 * 8)()
    _check(_lib().tga_get_op_candidates(_P(ctx), out), "tga_get_op_candidates")
    return [int(v) for v in out]


def tga_set_granular(ctx: int, nbr_dev_ptr: int, theta: int):
    _check(_lib().tga_set_granular(_P(ctx), _P(nbr_dev_ptr or None), theta), "tga_set_granular")


def tga_set_move_log(ctx: int, log_dev_ptr: int, capacity: int):
    _check(_lib().tga_set_move_log(_P(ctx), _P(log_dev_ptr or None), capacity), "tga_set_move_log")


def tga_set_tile(ctx: int, rows: int = 0, warps: int = 0):
    _check(_lib().tga_set_tile(_P(ctx), rows, warps), "tga_set_tile")


def tga_get_tile(ctx: int):
    r, w = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().tga_get_tile(_P(ctx), ctypes.byref(r), ctypes.byref(w)), "tga_get_tile")
    return r.value, w.value


def tga_eval_best_move_noalloc(inst: tga_instance, sol: tga_solution, op_mask: int, stream: int,
                               out_dev_ptr: int):
    """Allocation-free best-move evaluation (scratch in a fixed device array
    inside the library; n + m + 1 <= 1280).  Synchronous."""
    _check(_lib().tga_eval_best_move_noalloc(ctypes.byref(inst), ctypes.byref(sol), op_mask,
                                             _P(stream or None), _P(out_dev_ptr)),
           "tga_eval_best_move_noalloc")


def tga_profile_inter(ctx: int, reps: int = 10) -> float:
    """Mean milliseconds per launch of the inter-route evaluation kernel."""
    ms = ctypes.c_float()
    _check(_lib().tga_profile_inter(_P(ctx), reps, ctypes.byref(ms)), "tga_profile_inter")
    return ms.value


def tga_profile_xswap(ctx: int, reps: int = 10) -> float:
    """Mean milliseconds per launch of the swaps-of-runs kernel (ranks 6, 7)."""
    ms = ctypes.c_float()
    _check(_lib().tga_profile_xswap(_P(ctx), reps, ctypes.byref(ms)), "tga_profile_xswap")
    return ms.value


def tga_measure_int_peak(kind: int, stream: int = 0, iters: int = 4000):
    """(integer operations per second, milliseconds) of the dependency-free
    stream `kind` (0: add + max, 1: three-input adds) on the current device."""
    ops = ctypes.c_double()
    ms = ctypes.c_float()
    _check(_lib().tga_measure_int_peak(kind, _P(stream or None), iters, ctypes.byref(ops), ctypes.byref(ms)),
           "tga_measure_int_peak")
    return float(ops.value), float(ms.value)


def tga_set_descent_mode(ctx: int, mode: int):
    _check(_lib().tga_set_descent_mode(_P(ctx), mode), "tga_set_descent_mode")


def tga_get_descent_mode(ctx: int):
    """(path of the last descent as a DESCENT_* value, persistent grid size or 0)."""
    m, g = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().tga_get_descent_mode(_P(ctx), ctypes.byref(m), ctypes.byref(g)), "tga_get_descent_mode")
    return m.value, g.value


def tga_get_persistent_shape(ctx: int):
    r, w, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().tga_get_persistent_shape(_P(ctx), ctypes.byref(r), ctypes.byref(w), ctypes.byref(s)),
           "tga_get_persistent_shape")
    return r.value, w.value, s.value


def tga_set_tile_shape(ctx: int, rows: int, col_warps: int, row_split: int):
    _check(_lib().tga_set_tile_shape(_P(ctx), rows, col_warps, row_split), "tga_set_tile_shape")


def tga_get_tile_shape(ctx: int):
    r, w, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().tga_get_tile_shape(_P(ctx), ctypes.byref(r), ctypes.byref(w), ctypes.byref(s)),
           "tga_get_tile_shape")
    return r.value, w.value, s.value


def tga_debug_read(ctx: int, what: int) -> np.ndarray:
    """Copy an internal array (see include/tga.h) as raw int32 values."""
    size = ctypes.c_size_t()
    _check(_lib().tga_debug_read(_P(ctx), what, None, 0, ctypes.byref(size)), "tga_debug_read")
    buf = np.zeros(max(1, size.value // 4), dtype=np.int32)
    _check(_lib().tga_debug_read(_P(ctx), what, buf.ctypes.data, size.value, None), "tga_debug_read")
    return buf


def tga_set_tile_strip(ctx: int, rows: int, col_warps: int):
    _check(_lib().tga_set_tile_strip(_P(ctx), rows, col_warps), "tga_set_tile_strip")


def tga_set_wait_limit(ctx: int, limit_ns: int):
    _check(_lib().tga_set_wait_limit(_P(ctx), int(limit_ns)), "tga_set_wait_limit")


def tga_set_persistent_shape(ctx: int, rows: int, col_warps: int, row_split: int):
    _check(_lib().tga_set_persistent_shape(ctx, rows, col_warps, row_split), "tga_set_persistent_shape")


def tga_get_bounds_report(ctx: int) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(_lib().tga_get_bounds_report(ctx, out), "tga_get_bounds_report")
    return {"checked": bool(out[0]), "site": int(out[1]), "index": int(out[2]), "limit": int(out[3])}


def tga_destroy(ctx: int):
    _check(_lib().tga_destroy(_P(ctx)), "tga_destroy")


def tga_strerror(code: int) -> str:
    return _lib().tga_strerror(code).decode()


# ---------------------------------------------------------------------------
# convenience owner of device memory (torch) + one context

class LocalSearch:
    """Device-resident instance + solution + libtga context.

    ``inst`` / ``sol`` are ``instances.Instance`` / ``instances.Solution``
    (host numpy).  Arrays are copied to ``device`` with torch on ``stream``
    (a torch.cuda.Stream or None for the current stream)."""

    def __init__(self, inst, sol, op_mask: int, device="cuda:0", stream=None, log_capacity: int = 0,
                 pinned: bool = False, granular=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n = int(inst.n)
        self.m = int(np.asarray(sol.route_start).shape[0] - 1)
        self.W = self.n + 1 + self.m
        self.op_mask = int(op_mask)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32))
        with torch.cuda.stream(self.stream):
            host = [t(inst.dist).reshape(-1), t(inst.demand), t(inst.service), t(inst.tw_early),
                    t(inst.tw_late), t(sol.tour), t(sol.route_start)]
            pk = getattr(inst, "pickup", None)
            if pk is not None:                   # VRPSPDTW: pickup quantities
                host.append(t(pk))
            if pinned:
                host = [h.pin_memory() for h in host]
            dev = [h.to(self.device, non_blocking=pinned) for h in host]
            (self.dist, self.demand, self.service, self.early, self.late,
             self.tour, self.route_start) = dev[:7]
            self.pickup = dev[7] if pk is not None else None
            self.move = torch.zeros(6, dtype=torch.int32, device=self.device)   # one tga_move
            self.log = (torch.full((log_capacity,), -1, dtype=torch.int64, device=self.device)
                        if log_capacity else None)
        self.c_inst = tga_instance(self.n, self.m, int(inst.capacity), int(bool(inst.has_tw)),
                                   int(inst.w_load), int(inst.w_tw), self.dist.data_ptr(),
                                   self.demand.data_ptr(),
                                   self.service.data_ptr() if inst.has_tw else None,
                                   self.early.data_ptr() if inst.has_tw else None,
                                   self.late.data_ptr() if inst.has_tw else None,
                                   self.pickup.data_ptr() if self.pickup is not None else None)
        self.c_sol = tga_solution(self.tour.data_ptr(), self.route_start.data_ptr())
        self.ctx = tga_create(self.c_inst, self.c_sol, self.op_mask, self.stream.cuda_stream)
        if self.log is not None:
            tga_set_move_log(self.ctx, self.log.data_ptr(), log_capacity)
        self.nbr = None
        if granular is not None:         # edge-based extraction: mask rows (n+1, theta)
            nbr = np.ascontiguousarray(granular, dtype=np.int32)
            with torch.cuda.stream(self.stream):
                self.nbr = torch.from_numpy(nbr.reshape(-1)).to(self.device)
            tga_set_granular(self.ctx, self.nbr.data_ptr(), int(nbr.shape[1]))

    # -- reuse the device buffers for another solution / instance of the same size
    def reload(self, inst=None, sol=None):
        """Copy new host arrays into the existing device tensors (same shapes)
        and rebuild the attributes.  Host arrays are staged in pinned memory so
        the copies are asynchronous on the context's stream."""
        torch = self.torch
        pairs = []
        if inst is not None:
            pairs += [(self.dist, inst.dist), (self.demand, inst.demand), (self.service, inst.service),
                      (self.early, inst.tw_early), (self.late, inst.tw_late)]
            if (getattr(inst, "pickup", None) is None) != (self.pickup is None):
                raise ValueError("reload cannot add or drop pickups")
            if self.pickup is not None:
                pairs.append((self.pickup, inst.pickup))
        if sol is not None:
            pairs += [(self.tour, sol.tour), (self.route_start, sol.route_start)]
        if not hasattr(self, "_pinned"):
            self._pinned = {}
        nbytes = 0
        with torch.cuda.stream(self.stream):
            for dev, host in pairs:
                key = dev.data_ptr()
                buf = self._pinned.get(key)
                if buf is None:
                    buf = torch.empty(dev.numel(), dtype=torch.int32).pin_memory()
                    self._pinned[key] = buf
                buf.numpy()[:] = np.ascontiguousarray(host, dtype=np.int32).reshape(-1)
                dev.view(-1).copy_(buf, non_blocking=True)
                nbytes += dev.numel() * 4
        tga_build_attrs(self.ctx)
        return nbytes

    # -- calls
    def build(self):
        tga_build_attrs(self.ctx)
        return self

    def eval_best_move(self) -> dict:
        tga_eval_best_move(self.ctx, self.move.data_ptr())
        self.stream.synchronize()
        v = self.move.cpu().numpy()
        return dict(delta=int(v[0]), move_index=int(np.uint32(v[1].view(np.uint32))), op=int(v[2]),
                    a=int(v[3]), b=int(v[4]), valid=bool(v[5]))

    def apply_current_move(self):
        """Apply the move last written by eval_best_move (device memory)."""
        tga_apply_move(self.ctx, self.move.data_ptr())

    def descend(self, max_steps: int = (1 << 62)) -> dict:
        return tga_descend(self.ctx, max_steps)

    def set_descent_mode(self, mode: int):
        tga_set_descent_mode(self.ctx, mode)
        return self

    def descent_mode(self):
        return tga_get_descent_mode(self.ctx)

    def stats(self) -> dict:
        return tga_get_stats(self.ctx)

    def set_tile(self, rows=0, warps=0, row_split=None):
        """Inter-route tile shape; row_split = 0 selects the strip-major
        kernel (tga_set_tile_strip)."""
        if row_split is None:
            tga_set_tile(self.ctx, rows, warps)
        elif row_split == 0:
            tga_set_tile_strip(self.ctx, rows, warps)
        else:
            tga_set_tile_shape(self.ctx, rows, warps, row_split)
        return tga_get_tile_shape(self.ctx)

    def solution(self):
        self.stream.synchronize()
        return self.tour.cpu().numpy().copy(), self.route_start.cpu().numpy().copy()

    def move_log(self):
        self.stream.synchronize()
        st = self.stats()
        k = min(int(st["evaluations"]), self.log.shape[0])
        return self.log[:k].cpu().numpy().view(np.uint64).copy()

    def close(self):
        if getattr(self, "ctx", None):
            tga_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack_key(key: int):
    return (int(key) >> 32) - (1 << 31), int(key) & 0xFFFFFFFF
