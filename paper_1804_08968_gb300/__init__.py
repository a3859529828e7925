"""GB300 dexel offsets: Python binding of libdexel (include/dexel.h).

Argument marshalling only: torch provides device memory and the CUDA stream, every step of
the computation runs in the library's CUDA kernels.  There is no CPU fallback -- if the
library cannot be loaded the import of ``lib()`` raises.

Typical use::

    import paper_1804_08968_gb300 as dx
    g = dx.Grid.from_host(nx, ny, h, col_off, z, dtype=torch.float64)   # CSR on the GPU
    d = dx.dilate(g, k=8.0)              # ball of radius 8 grid spacings
    e = dx.erode(g, k=8.0)
    c = dx.close(g, k=8.0)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Grid", "Context", "dilate", "erode", "close", "open_", "boolean", "shell", "lib",
           "DexelError", "FP64", "FP32_PRED64", "UNION", "INTERSECT", "DIFFERENCE",
           "dilate_slices", "erode_slices", "raycast"]

FP64 = 0
FP32_PRED64 = 1
DILATE, ERODE, CLOSE, OPEN = 0, 1, 2, 3
# dexel_status codes
OK, ERR_INVALID_ARG, ERR_BAD_CSR, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_NO_PLAN = (
    0, -1, -2, -3, -4, -5, -6, -7)
UNION, INTERSECT, DIFFERENCE = 0, 1, 2
# dexel_prim: int32 kind, int32 pad, 7 doubles
PRIM_DTYPE = np.dtype([("kind", "<i4"), ("pad", "<i4"), ("p", "<f8", (7,))])
PRIM_KIND = {"sphere": 0, "box": 1, "shell": 2}
STATUS = {0: "ok", -1: "invalid argument", -2: "malformed CSR dexel grid",
          -3: "capacity too small", -4: "CUDA runtime error", -5: "device wait timeout",
          -6: "out of memory"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libdexel.so")
_lib = None


class DexelError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class _In(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("h", ctypes.c_double),
                ("col_off", ctypes.c_void_p), ("z", ctypes.c_void_p), ("nseg", ctypes.c_int64)]


class _Out(ctypes.Structure):
    _fields_ = [("col_off", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("capacity_seg", ctypes.c_int64), ("nseg", ctypes.c_int64)]


def lib():
    """Load libdexel.so (built by ``paper_1804_08968_gb300.build``); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise ImportError(f"libdexel.so not built ({_LIBPATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(_LIBPATH)
        P = ctypes.c_void_p
        L.dexel_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
        L.dexel_ctx_destroy.argtypes = [P]
        L.dexel_ctx_destroy.restype = None
        for name in ("dexel_dilate", "dexel_erode"):
            f = getattr(L, name)
            f.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                          ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_offset_enqueue.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(_Out), P, ctypes.c_size_t,
                                           P, P]
        L.dexel_morph.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_validate.argtypes = [P, ctypes.POINTER(_In), ctypes.c_int, P, ctypes.c_size_t, P]
        L.dexel_raycast.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Out), P,
                                    ctypes.c_size_t, P]
        L.dexel_raycast_axis.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_offset_ldi.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_offset_slices.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_boolean.argtypes = [P, ctypes.c_int, ctypes.POINTER(_In), ctypes.POINTER(_In),
                                    ctypes.c_int, ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_shell.argtypes = [P, ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(_Out), P, ctypes.c_size_t, P]
        L.dexel_offset_batched.argtypes = [P, ctypes.c_int, ctypes.POINTER(_In),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                           ctypes.POINTER(_Out), P, ctypes.c_size_t, P, P]
        L.dexel_last_error_detail.argtypes = []
        L.dexel_last_error_detail.restype = ctypes.c_char_p
        L.dexel_set_batch_autotune.argtypes = [P, ctypes.c_int]
        L.dexel_set_batch_autotune.restype = None
        L.dexel_workspace_size.argtypes = [ctypes.POINTER(_In), ctypes.c_double, ctypes.c_int]
        L.dexel_workspace_size.restype = ctypes.c_size_t
        L.dexel_last_required.argtypes = [P]
        L.dexel_last_required.restype = ctypes.c_size_t
        L.dexel_last_launches.argtypes = [P]
        L.dexel_last_launches.restype = ctypes.c_int64
        L.dexel_status_string.argtypes = [ctypes.c_int]
        L.dexel_status_string.restype = ctypes.c_char_p
        L.dexel_set_profiling.argtypes = [P, ctypes.c_int]
        L.dexel_set_profiling.restype = None
        L.dexel_last_stage_ms.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.dexel_last_kernel_ms.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.dexel_last_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


class Grid:
    """A CSR dexel grid resident on the GPU (col_off int32, z (nseg, 2) float32/float64)."""

    def __init__(self, nx, ny, h, col_off, z):
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.col_off = col_off
        self.z = z

    @property
    def nseg(self) -> int:
        return int(self.z.shape[0])

    @property
    def mode(self) -> int:
        return FP64 if self.z.dtype == _torch().float64 else FP32_PRED64

    @classmethod
    def from_host(cls, nx, ny, h, col_off, z, dtype=None, device="cuda"):
        torch = _torch()
        dtype = dtype or (torch.float32 if np.asarray(z).dtype == np.float32 else torch.float64)
        off = torch.as_tensor(np.asarray(col_off, np.int32)).to(device)
        zz = torch.as_tensor(np.asarray(z).reshape(-1, 2)).to(device=device, dtype=dtype)
        return cls(nx, ny, h, off.contiguous(), zz.contiguous())

    @classmethod
    def from_synth(cls, g, dtype=None, device="cuda"):
        return cls.from_host(g.nx, g.ny, g.h, g.col_off, g.z, dtype=dtype, device=device)

    def to_host(self):
        return self.col_off.cpu().numpy().astype(np.int64), self.z.cpu().numpy()

    def _in(self) -> _In:
        torch = _torch()
        z = self.z if self.z.numel() else torch.zeros((1, 2), dtype=self.z.dtype, device=self.z.device)
        self._keep = z
        return _In(self.nx, self.ny, self.h, self.col_off.data_ptr(), z.data_ptr(), self.nseg)


class Context:
    """One libdexel context per device; owns the library's scratch between calls."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ptr = ctypes.c_void_p()
        rc = lib().dexel_ctx_create(ctypes.byref(self.ptr), device)
        if rc != 0:
            raise DexelError(rc, "dexel_ctx_create")
        self._cap_hint = {}

    def __del__(self):
        try:
            if self.ptr:
                lib().dexel_ctx_destroy(self.ptr)
        except Exception:  # pragma: no cover
            pass

    @property
    def last_launches(self) -> int:
        return int(lib().dexel_last_launches(self.ptr))

    def set_profiling(self, on: bool) -> None:
        """Bracket each stage of every call with CUDA events on the call's stream."""
        lib().dexel_set_profiling(self.ptr, 1 if on else 0)

    def stage_ms(self):
        """Device ms of [validate+tables, pass 1, pass 2, count+scan, write] of the last call."""
        a = (ctypes.c_double * 5)()
        n = lib().dexel_last_stage_ms(self.ptr, a, 5)
        return [a[i] for i in range(n)]

    def kernel_ms(self):
        """Device ms of [pass-1 window kernel, k_levels, k_lgather, S_mid float copy] of the
        last call (profiling on; 0 for a kernel that did not run)."""
        a = (ctypes.c_double * 4)()
        n = lib().dexel_last_kernel_ms(self.ptr, a, 4)
        return [a[i] for i in range(n)]

    def stats(self):
        """[input segments, S_mid pieces, pass-2 intervals, output segments, max pieces per
        S_mid column, columns redone by the fallback gather (sweep: max live state), status
        bits, attempts, pass-1 redo launches, blocks of y lines, pass-1 tiles walked twice,
        columns whose lists outgrew the gather's bucket, that bucket's size, the event room of a
        pass-1 tile, level lists longer than a lane's slots] of the last call."""
        a = (ctypes.c_int64 * 15)()
        n = lib().dexel_last_stats(self.ptr, a, 15)
        return [int(a[i]) for i in range(n)]

    def _stream(self, stream):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def run(self, op: int, g: Grid, k: float, stream=None, capacity=None) -> Grid:
        torch = _torch()
        key = (op, g.nx, g.ny, g.nseg, float(k), g.mode)
        cap = capacity or self._cap_hint.get(key) or max(2 * g.nseg + g.nx * g.ny // 4, 1024)
        gin = g._in()
        st = self._stream(stream)
        for _ in range(3):
            off = torch.empty(g.nx * g.ny + 1, dtype=torch.int32, device=g.col_off.device)
            z = torch.empty((cap, 2), dtype=g.z.dtype, device=g.z.device)
            out = _Out(off.data_ptr(), z.data_ptr(), cap, 0)
            if op == DILATE:
                rc = lib().dexel_dilate(self.ptr, ctypes.byref(gin), k, g.mode, ctypes.byref(out), None, 0, st)
            elif op == ERODE:
                rc = lib().dexel_erode(self.ptr, ctypes.byref(gin), k, g.mode, ctypes.byref(out), None, 0, st)
            else:
                rc = lib().dexel_morph(self.ptr, ctypes.byref(gin), k, op, g.mode, ctypes.byref(out), None, 0, st)
            if rc == -3 and out.nseg > cap:
                cap = int(out.nseg) + 16
                continue
            if rc != 0:
                detail = lib().dexel_last_error_detail().decode()
                raise DexelError(rc, f"dexel offset (stats {self.stats()}, "
                                     f"required {lib().dexel_last_required(self.ptr)} B{', ' + detail if detail else ''})")
            self._cap_hint[key] = cap
            return Grid(g.nx, g.ny, g.h, off, z[: out.nseg])
        raise DexelError(-3, "dexel offset (output capacity)")

    def last_required(self) -> int:
        """Workspace bytes the last call needed (dexel_last_required)."""
        return int(lib().dexel_last_required(self.ptr))

    def enqueue(self, op: int, g: Grid, k: float, ws, out_off, out_z, result, stream=None) -> int:
        """dexel_offset_enqueue: queue op (DILATE or ERODE) of g by k on the stream with no host
        synchronisation, replaying the plan a synchronous run() of the same offset recorded on
        this context.  ws: a uint8 device tensor of at least last_required() bytes after that
        run; out_off: int32 [nx*ny + 1]; out_z: [capacity, 2] of g's dtype; result: int64 [2]
        device tensor that receives [status, output segments] in stream order.  Returns the
        host-side status (0 queued; -7 no plan recorded for this offset)."""
        gin = g._in()
        out = _Out(out_off.data_ptr(), out_z.data_ptr(), int(out_z.shape[0]), 0)
        return int(lib().dexel_offset_enqueue(self.ptr, ctypes.byref(gin), float(k), op, g.mode,
                                              ctypes.byref(out), ctypes.c_void_p(ws.data_ptr()),
                                              ws.numel(), self._stream(stream),
                                              ctypes.c_void_p(result.data_ptr())))

    def _call_out(self, nx, ny, h, like, cap, fn, what):
        """Run fn(out) with an output of cap segments, growing it once to the reported need."""
        torch = _torch()
        for _ in range(3):
            off = torch.empty(nx * ny + 1, dtype=torch.int32, device=like.col_off.device)
            z = torch.empty((cap, 2), dtype=like.z.dtype, device=like.z.device)
            out = _Out(off.data_ptr(), z.data_ptr(), cap, 0)
            rc = fn(out)
            if rc == -3 and out.nseg > cap:
                cap = int(out.nseg) + 16
                continue
            if rc != 0:
                detail = lib().dexel_last_error_detail().decode()
                raise DexelError(rc, f"{what}{' (' + detail + ')' if detail else ''}")
            return Grid(nx, ny, h, off, z[: out.nseg])
        raise DexelError(-3, f"{what} (output capacity)")

    def boolean(self, op: int, a: Grid, b: Grid, stream=None) -> Grid:
        """op in UNION / INTERSECT / DIFFERENCE (dexel_boolean)."""
        if (a.nx, a.ny) != (b.nx, b.ny) or a.mode != b.mode:
            raise ValueError("grids of different sizes or precisions")
        ia, ib = a._in(), b._in()
        st = self._stream(stream)
        cap = max(a.nseg + b.nseg + 16, 1024)
        return self._call_out(a.nx, a.ny, a.h, a, cap, lambda out: lib().dexel_boolean(
            self.ptr, op, ctypes.byref(ia), ctypes.byref(ib), a.mode, ctypes.byref(out), None, 0, st),
            "dexel_boolean")

    def raycast(self, prims, nx: int, ny: int, h: float, dtype=None, stream=None, axis: int = 2) -> Grid:
        """Ray-cast primitives ("sphere", cx, cy, cz, R) / ("box", x0, x1, y0, y1, z0, z1) /
        ("shell", cx, cy, cz, R, t) at the column centres of an nx x ny grid of spacing h
        (dexel_raycast); dtype float64 (default) or float32 endpoints."""
        torch = _torch()
        dtype = dtype or torch.float64
        rec = np.zeros(len(prims), dtype=PRIM_DTYPE)
        for q, p in enumerate(prims):
            rec["kind"][q] = PRIM_KIND[p[0]]
            rec["p"][q, : len(p) - 1] = p[1:]
        dev = torch.device("cuda", self.device)
        buf = torch.from_numpy(rec.view(np.uint8).copy()).to(dev) if len(prims) else None
        st = self._stream(stream)
        mode = FP64 if dtype == torch.float64 else FP32_PRED64
        like = Grid(nx, ny, h, torch.empty(1, dtype=torch.int32, device=dev),
                    torch.empty((0, 2), dtype=dtype, device=dev))
        ptr = buf.data_ptr() if buf is not None else None
        return self._call_out(nx, ny, h, like, max(4 * nx * ny, 1024), lambda out: lib().dexel_raycast_axis(
            self.ptr, ptr, len(prims), axis, nx, ny, float(h), mode, ctypes.byref(out), None, 0, st),
            "dexel_raycast_axis")

    def offset_ldi(self, op: int, views, k: float, stream=None):
        """The three views of a layered depth image (rays along z, x, y) each offset by op
        (dexel_offset_ldi); returns three grids."""
        torch = _torch()
        if len(views) != 3 or any(v.mode != views[0].mode for v in views):
            raise ValueError("three views of one precision")
        ins = (_In * 3)(*[v._in() for v in views])
        st = self._stream(stream)
        caps = [max(4 * v.nseg + v.nx * v.ny // 4, 1024) for v in views]
        for _ in range(3):
            outs_t = []
            outs = (_Out * 3)()
            for q, v in enumerate(views):
                off = torch.empty(v.nx * v.ny + 1, dtype=torch.int32, device=v.col_off.device)
                z = torch.empty((caps[q], 2), dtype=v.z.dtype, device=v.z.device)
                outs_t.append((off, z))
                outs[q] = _Out(off.data_ptr(), z.data_ptr(), caps[q], 0)
            rc = lib().dexel_offset_ldi(self.ptr, ins, float(k), op, views[0].mode, outs, None, 0, st)
            if rc == -3 and any(outs[q].nseg > caps[q] for q in range(3)):
                caps = [max(caps[q], int(outs[q].nseg) + 16) for q in range(3)]
                continue
            if rc != 0:
                raise DexelError(rc, "dexel_offset_ldi")
            return [Grid(v.nx, v.ny, v.h, outs_t[q][0], outs_t[q][1][: outs[q].nseg])
                    for q, v in enumerate(views)]
        raise DexelError(-3, "dexel_offset_ldi (output capacity)")

    def slices(self, op: int, g: Grid, k: float, stream=None) -> Grid:
        """Every row of g a 2D image, dilated (op DILATE) or eroded (ERODE) by a disk of radius
        k spacings (dexel_offset_slices)."""
        gin = g._in()
        st = self._stream(stream)
        cap = max(2 * g.nseg + g.nx * g.ny // 4, 1024)
        return self._call_out(g.nx, g.ny, g.h, g, cap, lambda out: lib().dexel_offset_slices(
            self.ptr, ctypes.byref(gin), float(k), op, g.mode, ctypes.byref(out), None, 0, st),
            "dexel_offset_slices")

    def shell(self, g: Grid, k: float, stream=None) -> Grid:
        """Thick shell: dilation minus erosion by a ball of radius k spacings (dexel_shell)."""
        gin = g._in()
        st = self._stream(stream)
        cap = max(4 * g.nseg + g.nx * g.ny // 4, 1024)
        return self._call_out(g.nx, g.ny, g.h, g, cap, lambda out: lib().dexel_shell(
            self.ptr, ctypes.byref(gin), float(k), g.mode, ctypes.byref(out), None, 0, st),
            "dexel_shell")

    def run_batched(self, ops, grids, ks, stream=None, capacities=None):
        """Offsets of many grids in one batched call (dexel_offset_batched): ops[s] in
        DILATE / ERODE / CLOSE / OPEN, grids all FP64 or all FP32.  Returns the output grids;
        a shape whose output did not fit is run again with the size the library reported."""
        torch = _torch()
        n = len(grids)
        if n == 0:
            return []
        mode = grids[0].mode
        if any(g.mode != mode for g in grids):
            raise ValueError("all grids of a batch share one precision")
        caps = list(capacities) if capacities else [max(2 * g.nseg + g.nx * g.ny // 4, 1024) for g in grids]
        st = self._stream(stream)
        todo = list(range(n))
        res = [None] * n
        for _ in range(3):
            ins = (_In * len(todo))(*[grids[s]._in() for s in todo])
            outs_t = []
            outs = (_Out * len(todo))()
            for q, s in enumerate(todo):
                g = grids[s]
                off = torch.empty(g.nx * g.ny + 1, dtype=torch.int32, device=g.col_off.device)
                z = torch.empty((caps[s], 2), dtype=g.z.dtype, device=g.z.device)
                outs_t.append((off, z))
                outs[q] = _Out(off.data_ptr(), z.data_ptr(), caps[s], 0)
            kk = (ctypes.c_double * len(todo))(*[float(ks[s]) for s in todo])
            oo = (ctypes.c_int * len(todo))(*[int(ops[s]) for s in todo])
            dst = torch.zeros(len(todo), dtype=torch.int32, device=grids[todo[0]].col_off.device)
            rc = lib().dexel_offset_batched(self.ptr, len(todo), ins, kk, oo, mode, outs, None, 0,
                                            ctypes.c_void_p(dst.data_ptr()), st)
            stat = dst.cpu().numpy()
            again = []
            for q, s in enumerate(todo):
                if stat[q] == 0:
                    off, z = outs_t[q]
                    res[s] = Grid(grids[s].nx, grids[s].ny, grids[s].h, off, z[: outs[q].nseg])
                elif stat[q] == -3 and outs[q].nseg > caps[s]:
                    caps[s] = int(outs[q].nseg) + 16
                    again.append(s)
                else:
                    raise DexelError(int(stat[q]), f"dexel_offset_batched shape {s} (rc {rc})")
            if not again:
                return res
            todo = again
        raise DexelError(-3, "dexel_offset_batched (output capacity)")

    def set_batch_autotune(self, on: bool) -> None:
        lib().dexel_set_batch_autotune(self.ptr, 1 if on else 0)

    def validate(self, g: Grid, stream=None) -> int:
        gin = g._in()
        return int(lib().dexel_validate(self.ptr, ctypes.byref(gin), g.mode, None, 0, self._stream(stream)))


_ctx = {}


def _default_ctx(g: Grid) -> Context:
    dev = g.col_off.device.index or 0
    if dev not in _ctx:
        _ctx[dev] = Context(dev)
    return _ctx[dev]


def dilate(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Dilation by a ball of radius k grid spacings (exact on the dexel grid)."""
    return (ctx or _default_ctx(g)).run(DILATE, g, k, stream)


def erode(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Erosion by a ball of radius k grid spacings (complement of the dilated complement)."""
    return (ctx or _default_ctx(g)).run(ERODE, g, k, stream)


def close(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Closing: erosion of the dilation."""
    return (ctx or _default_ctx(g)).run(CLOSE, g, k, stream)


def open_(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Opening: dilation of the erosion."""
    return (ctx or _default_ctx(g)).run(OPEN, g, k, stream)


def boolean(op: int, a: Grid, b: Grid, ctx: Context | None = None, stream=None) -> Grid:
    """Union / intersection / difference of two grids (CSG in dexel space)."""
    return (ctx or _default_ctx(a)).boolean(op, a, b, stream)


def shell(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Thick shell: the dilation minus the erosion by a ball of radius k spacings."""
    return (ctx or _default_ctx(g)).shell(g, k, stream)


def dilate_slices(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Every row a 2D dexel image dilated by a disk of radius k spacings (Sec. 3.2)."""
    return (ctx or _default_ctx(g)).slices(DILATE, g, k, stream)


def erode_slices(g: Grid, k: float, ctx: Context | None = None, stream=None) -> Grid:
    """Every row a 2D dexel image eroded by a disk of radius k spacings."""
    return (ctx or _default_ctx(g)).slices(ERODE, g, k, stream)


def raycast(prims, nx: int, ny: int, h: float, dtype=None, device: int = 0, axis: int = 2) -> Grid:
    """Ray-cast analytic primitives into a dexel grid on the GPU (dexel_raycast_axis; rays
    along axis 2 = z by default)."""
    if device not in _ctx:
        _ctx[device] = Context(device)
    return _ctx[device].raycast(prims, nx, ny, h, dtype, axis=axis)
