"""FP64 CPU oracle for dexel dilation / erosion / closing / opening by a ball.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path (the CUDA
library and its binding) never imports it, and it imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain brute-force gather, see its header):
  * ``dilate``  -- Sec. 3.1 Eq. of D_r: union over in-grid columns c' with n = di^2+dj^2 <= k^2
                   of [a - w, b + w], w = h sqrt(k^2 - n)  (the Sec. 4 brute force, as a gather);
  * ``erode``   -- Sec. 3.1 "Erosion", written directly: intersection over c' of the union of
                   [a + w, b - w]; zero-length results dropped;
  * ``close`` = erode(dilate(S)), ``open`` = dilate(erode(S))   (Sec. 4 "Topological Cleaning");
  * ``union`` / ``intersection`` / ``difference`` -- CSG in dexel space (Sec. 2, "(3)"), from
                   point membership of each column's elementary intervals, then the closure;
  * ``shell`` = difference(dilate(S), erode(S))  (Sec. 4 "3D Printing", the teaser figure);
  * ``dilate_slices`` / ``erode_slices`` -- Sec. 3.2's 2D offsets for every row at once: the
                   same gather over the output column's own row only (a disk in the x-z plane);
  * ``raycast`` -- analytic spheres, boxes and hollow spheres cast at the column centres
                   (Sec. 1: implicit shapes to ray representations), chords united per column.
``complement`` builds the per-column complement with +-inf sentinels (Sec. 3.1: the complement
is trivial in a ray representation); tests use it to check erosion/dilation duality.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` (closed forms
with Pythagorean radii, point-membership brute force against the distance definition,
duality, monotonicity, union commutation, extensivity, idempotence, k = 0 identity) and, for
the Boolean operations and the shell, by ``tests/test_csg_oracle.py`` (closed forms of boxes
and concentric spheres, additivity of length, set identities, point membership, the golden
capsule, shell u erosion = dilation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (IEEE double, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_offset.restype = ctypes.c_int64
        lib.oracle_offset.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                      ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                      ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
        lib.oracle_offset_slices.restype = ctypes.c_int64
        lib.oracle_offset_slices.argtypes = lib.oracle_offset.argtypes
        lib.oracle_raycast.restype = ctypes.c_int64
        lib.oracle_raycast.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                       ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_boolean.restype = ctypes.c_int64
        lib.oracle_boolean.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                       ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class Columns:
    """Result of an oracle call: CSR over the requested columns (float64 endpoints)."""

    def __init__(self, off: np.ndarray, z: np.ndarray, cols):
        self.off = off
        self.z = z
        self.cols = cols

    def column(self, t: int) -> np.ndarray:
        return self.z[self.off[t]:self.off[t + 1]]

    def __len__(self):
        return len(self.off) - 1


def _run(grid, k: float, erode: int, cols=None, threads: int | None = None,
         slices: bool = False) -> Columns:
    lib = _load()
    off_in = np.ascontiguousarray(grid.col_off, dtype=np.int64)
    z_in = np.ascontiguousarray(grid.z, dtype=np.float64).reshape(-1)
    if z_in.size == 0:
        z_in = np.zeros(2, np.float64)
    if cols is not None:
        cols_arr = np.ascontiguousarray(cols, dtype=np.int64)
        ncols = cols_arr.size
        cptr = cols_arr.ctypes.data
    else:
        cols_arr = None
        ncols = grid.nx * grid.ny
        cptr = None
    po = ctypes.POINTER(ctypes.c_int64)()
    pz = ctypes.POINTER(ctypes.c_double)()
    fn = lib.oracle_offset_slices if slices else lib.oracle_offset
    total = fn(grid.nx, grid.ny, float(grid.h), float(k), off_in.ctypes.data,
               z_in.ctypes.data, erode, cptr, ncols,
               threads or default_threads(), ctypes.byref(po), ctypes.byref(pz))
    if total < 0:
        raise ValueError("oracle_offset rejected its arguments")
    off = np.ctypeslib.as_array(po, shape=(ncols + 1,)).copy()
    z = np.ctypeslib.as_array(pz, shape=(max(total, 1) * 2,))[: 2 * total].copy().reshape(-1, 2)
    lib.oracle_free(ctypes.cast(po, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(pz, ctypes.c_void_p))
    return Columns(off, z, cols_arr)


def _as_grid(template, res: Columns):
    from synth.shapes import DexelGrid  # container only
    return DexelGrid(template.nx, template.ny, template.h, res.off, res.z)


def dilate(grid, k: float, cols=None, threads=None):
    """Dilation by a ball of radius k*h.  With cols=None returns a full DexelGrid (float64)."""
    r = _run(grid, k, 0, cols, threads)
    return _as_grid(grid, r) if cols is None else r


def erode(grid, k: float, cols=None, threads=None):
    """Erosion by a ball of radius k*h (direct intersection form)."""
    r = _run(grid, k, 1, cols, threads)
    return _as_grid(grid, r) if cols is None else r


def dilate_slices(grid, k: float, cols=None, threads=None):
    """Every row of the grid a 2D dexel image dilated by a disk of radius k*h (Sec. 3.2)."""
    r = _run(grid, k, 0, cols, threads, slices=True)
    return _as_grid(grid, r) if cols is None else r


def erode_slices(grid, k: float, cols=None, threads=None):
    """Every row of the grid a 2D dexel image eroded by a disk of radius k*h."""
    r = _run(grid, k, 1, cols, threads, slices=True)
    return _as_grid(grid, r) if cols is None else r


def close(grid, k: float, threads=None):
    """Closing = erosion of the dilation."""
    return erode(dilate(grid, k, threads=threads), k, threads=threads)


def open_(grid, k: float, threads=None):
    """Opening = dilation of the erosion."""
    return dilate(erode(grid, k, threads=threads), k, threads=threads)


def _boolean(op: int, a, b):
    if (a.nx, a.ny) != (b.nx, b.ny):
        raise ValueError("grids of different sizes")
    lib = _load()
    oa = np.ascontiguousarray(a.col_off, dtype=np.int64)
    ob = np.ascontiguousarray(b.col_off, dtype=np.int64)
    za = np.ascontiguousarray(a.z, dtype=np.float64).reshape(-1)
    zb = np.ascontiguousarray(b.z, dtype=np.float64).reshape(-1)
    za = za if za.size else np.zeros(2)
    zb = zb if zb.size else np.zeros(2)
    ncols = a.nx * a.ny
    po = ctypes.POINTER(ctypes.c_int64)()
    pz = ctypes.POINTER(ctypes.c_double)()
    total = lib.oracle_boolean(op, ncols, oa.ctypes.data, za.ctypes.data, ob.ctypes.data,
                               zb.ctypes.data, ctypes.byref(po), ctypes.byref(pz))
    if total < 0:
        raise ValueError("oracle_boolean rejected its arguments")
    off = np.ctypeslib.as_array(po, shape=(ncols + 1,)).copy()
    z = np.ctypeslib.as_array(pz, shape=(max(total, 1) * 2,))[: 2 * total].copy().reshape(-1, 2)
    lib.oracle_free(ctypes.cast(po, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(pz, ctypes.c_void_p))
    return _as_grid(a, Columns(off, z, None))


def union(a, b):
    """Closed union of two grids, column by column (CSG in dexel space, Sec. 2)."""
    return _boolean(0, a, b)


def intersection(a, b):
    """Closed intersection; zero-length results dropped."""
    return _boolean(1, a, b)


def difference(a, b):
    """Closure of A minus B; zero-length results dropped."""
    return _boolean(2, a, b)


def shell(grid, k: float, threads=None):
    """Thick shell: the dilation minus the erosion (Sec. 4 "3D Printing", teaser figure)."""
    return difference(dilate(grid, k, threads=threads), erode(grid, k, threads=threads))


_KIND = {"sphere": 0, "box": 1, "shell": 2}


def prim_arrays(prims):
    """(kind int32[n], params float64[n, 8]) of primitive tuples ("sphere", cx, cy, cz, R),
    ("box", x0, x1, y0, y1, z0, z1), ("shell", cx, cy, cz, R, t)."""
    kind = np.array([_KIND[p[0]] for p in prims], np.int32)
    prm = np.zeros((max(len(prims), 1), 8), np.float64)
    for q, p in enumerate(prims):
        prm[q, : len(p) - 1] = p[1:]
    return kind, prm


def raycast(prims, nx: int, ny: int, h: float):
    """Ray-cast primitives at the column centres of an nx x ny grid of spacing h (Sec. 1,
    implicit shapes to ray representations; Sec. 3.1 dexels)."""
    from synth.shapes import DexelGrid  # container only
    lib = _load()
    kind, prm = prim_arrays(prims)
    po = ctypes.POINTER(ctypes.c_int64)()
    pz = ctypes.POINTER(ctypes.c_double)()
    total = lib.oracle_raycast(nx, ny, float(h), kind.ctypes.data, prm.ctypes.data, len(prims),
                               ctypes.byref(po), ctypes.byref(pz))
    if total < 0:
        raise ValueError("oracle_raycast rejected its arguments")
    n = nx * ny
    off = np.ctypeslib.as_array(po, shape=(n + 1,)).copy()
    z = np.ctypeslib.as_array(pz, shape=(max(total, 1) * 2,))[: 2 * total].copy().reshape(-1, 2)
    lib.oracle_free(ctypes.cast(po, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(pz, ctypes.c_void_p))
    return DexelGrid(nx, ny, h, off, z)


def round_float32(grid):
    """Each end rounded to the nearest float32, then segments that touch or overlap joined
    (a valid float32 grid: strictly positive gaps)."""
    from synth.shapes import DexelGrid  # container only
    n = grid.nx * grid.ny
    out_off = np.zeros(n + 1, np.int64)
    cols = []
    for c in range(n):
        segs = np.asarray(grid.z[grid.col_off[c]:grid.col_off[c + 1]], np.float64).astype(np.float32)
        res = []
        for a, b in segs:
            if res and a <= res[-1][1]:
                res[-1][1] = max(res[-1][1], b)
            else:
                res.append([a, b])
        cols.append(res)
        out_off[c + 1] = out_off[c] + len(res)
    z = np.array([s for col in cols for s in col], np.float32).reshape(-1, 2)
    return DexelGrid(grid.nx, grid.ny, grid.h, out_off, z)


def view_prims(prims, axis: int):
    """The primitives seen from rays along axis 0 (x) or 1 (y): coordinates cycled so that the
    ray runs along the third one (x rays: columns over (y, z); y rays: columns over (z, x));
    axis 2 leaves them as they are."""
    if axis == 2:
        return list(prims)
    u, v, w = (1, 2, 0) if axis == 0 else (2, 0, 1)
    out = []
    for p in prims:
        if p[0] == "box":
            b = p[1:]
            out.append(("box", b[2 * u], b[2 * u + 1], b[2 * v], b[2 * v + 1], b[2 * w], b[2 * w + 1]))
        else:
            c = p[1:4]
            out.append((p[0], c[u], c[v], c[w]) + tuple(p[4:]))
    return out


def raycast_axis(prims, axis: int, nx: int, ny: int, h: float):
    """Ray casting along axis 0, 1 or 2 (a view of a layered depth image, Sec. 5)."""
    return raycast(view_prims(prims, axis), nx, ny, h)


def complement(grid):
    """Per-column complement within the grid: (-inf, a1], [b1, a2], ..., [bn, +inf).

    An empty column becomes (-inf, +inf).  The closed complement intervals share endpoints
    with the shape; the difference is measure-zero and is what erosion's zero-length rule
    absorbs.
    """
    from synth.shapes import DexelGrid
    zin = np.asarray(grid.z, np.float64)
    cols = []
    for c in range(grid.nx * grid.ny):
        s0, s1 = grid.col_off[c], grid.col_off[c + 1]
        pts = np.concatenate([[-np.inf], zin[s0:s1].reshape(-1), [np.inf]]).reshape(-1, 2)
        # a shape piece reaching -inf or +inf leaves an empty (x, x) pair at that end
        keep = ~((pts[:, 0] == pts[:, 1]) & np.isinf(pts[:, 0]))
        cols.append(pts[keep])
    cnt = np.array([len(p) for p in cols], np.int64)
    off = np.zeros(grid.nx * grid.ny + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    z = np.concatenate(cols) if cols else np.zeros((0, 2))
    return DexelGrid(grid.nx, grid.ny, grid.h, off, z)
