"""FP64 Siddon projector of the oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this module. It wraps oracle/siddon_oracle.c (the plane-crossing Siddon
traversal) through ctypes and adds the geometry bookkeeping the BSGD oracle
needs: row blocks I_i, column blocks J_j (Sec. 2, Eq. 3), detector bands of a
column block and sub-detector cells (Sec. 2.1, Fig. 2).
"""
import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from .build import build_oracle

KINDS = {"par2d": 0, "fan2d": 1, "cone3d": 2}


class _OrcGeom(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("n_views", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
    ]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER
        g = P(_OrcGeom)
        lib.orc_trace_ray.argtypes = [g, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int]
        lib.orc_trace_ray.restype = ctypes.c_int
        lib.orc_fp_rows.argtypes = [g, P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        lib.orc_fp_rows.restype = ctypes.c_int
        lib.orc_bp_rows.argtypes = [g, P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        lib.orc_bp_rows.restype = ctypes.c_int
        lib.orc_count_rows.argtypes = [g, P(ctypes.c_int64), ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_count_rows.restype = ctypes.c_int64
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def num_threads() -> int:
    """OpenMP threads the oracle's projector uses."""
    return int(_lib().orc_num_threads())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


@dataclass
class Geometry:
    """Scan geometry. Angles default to uniform: a*pi/n for parallel beam,
    a*2*pi/n for fan and cone beam."""
    kind: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    n_views: int
    nu: int
    nv: int
    du: float
    dv: float
    dso: float = 0.0
    dsd: float = 0.0
    angles: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.angles is None:
            span = math.pi if self.kind == "par2d" else 2.0 * math.pi
            self.angles = np.arange(self.n_views, dtype=np.float64) * (span / self.n_views)
        self.angles = np.ascontiguousarray(self.angles, dtype=np.float64)
        self._c = _OrcGeom(KINDS[self.kind], self.nx, self.ny, self.nz,
                           self.dx, self.dy, self.dz, self.n_views,
                           _dptr(self.angles), self.nu, self.nv, self.du, self.dv,
                           self.dso, self.dsd)

    # sizes of A (Sec. 1: A in R^{r x c})
    @property
    def n_rows(self) -> int:
        return self.n_views * self.nv * self.nu

    @property
    def n_cols(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def block_axis(self) -> int:
        """Column blocks are slabs along z for volumes, along y for images."""
        return 2 if self.nz > 1 else 1

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.n_views, self.nv, self.nu)

    def axis_len(self, axis: int) -> int:
        return (self.nx, self.ny, self.nz)[axis]


# --------------------------------------------------------------------------
# Blocks (Sec. 2, Eq. 3)

def column_block(geom: Geometry, N: int, j: int):
    """Plane range [c0, c1) of column block J_j along the block axis."""
    n = geom.axis_len(geom.block_axis)
    return (j * n) // N, ((j + 1) * n) // N


def column_block_voxels(geom: Geometry, N: int, j: int) -> np.ndarray:
    """Flat voxel indices of J_j."""
    c0, c1 = column_block(geom, N, j)
    stride = geom.nx * geom.ny if geom.block_axis == 2 else geom.nx
    return np.arange(c0 * stride, c1 * stride, dtype=np.int64)


def row_block_views(geom: Geometry, M: int, i: int, view_block=None) -> np.ndarray:
    """Views of row block I_i: interleaved (a mod M == i) unless an explicit
    per-view block assignment is given."""
    a = np.arange(geom.n_views)
    if view_block is None:
        return a[a % M == i]
    return a[np.asarray(view_block) == i]


def rows_of_views(geom: Geometry, views) -> np.ndarray:
    per = geom.nv * geom.nu
    views = np.asarray(views, dtype=np.int64)
    return (views[:, None] * per + np.arange(per, dtype=np.int64)[None, :]).reshape(-1)


def cell_of_pixel(geom: Geometry, v, u, n_cells: int):
    """Sub-detector cell of pixel (v, u) (Fig. 2): halves in u for 2 cells,
    quadrants (v half * 2 + u half) for 4 cells, the whole detector for 1."""
    uh = (np.asarray(u) >= geom.nu // 2).astype(np.int64)
    vh = (np.asarray(v) >= geom.nv // 2).astype(np.int64)
    if n_cells == 1:
        return np.zeros_like(uh)
    if n_cells == 2:
        return uh
    if n_cells == 4:
        return vh * 2 + uh
    raise ValueError("n_cells must be 1, 2 or 4")


def rows_of_cell(geom: Geometry, view: int, cell: int, n_cells: int) -> np.ndarray:
    v, u = np.meshgrid(np.arange(geom.nv), np.arange(geom.nu), indexing="ij")
    sel = cell_of_pixel(geom, v, u, n_cells).reshape(-1) == cell
    base = view * geom.nv * geom.nu
    return base + np.nonzero(sel)[0].astype(np.int64)


# --------------------------------------------------------------------------
# Projector

def _block_args(geom, block):
    axis = geom.block_axis
    if block is None:
        return axis, 0, geom.axis_len(axis)
    return axis, int(block[0]), int(block[1])


def trace_ray(geom: Geometry, a: int, v: int, u: int):
    """(voxel indices, lengths) of every positive-length segment of one ray."""
    cap = geom.nx + geom.ny + geom.nz + 8
    vox = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap, dtype=np.float64)
    n = _lib().orc_trace_ray(ctypes.byref(geom._c), a, v, u, _iptr(vox), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError("orc_trace_ray failed")
    return vox[:n].copy(), ln[:n].copy()


def fp_rows(geom: Geometry, x, rows, block=None) -> np.ndarray:
    """(A_rows^J x_J) for the listed rows; block = (c0, c1) or None for all of x."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(rows.size, dtype=np.float64)
    axis, c0, c1 = _block_args(geom, block)
    rc = _lib().orc_fp_rows(ctypes.byref(geom._c), _dptr(x), _iptr(rows), rows.size,
                            axis, c0, c1, _dptr(out))
    if rc != 0:
        raise RuntimeError("orc_fp_rows failed (%d)" % rc)
    return out


def bp_rows(geom: Geometry, r_rows, rows, block=None, out=None) -> np.ndarray:
    """vol_J += (A_rows^J)^T r for the listed rows (r_rows[k] belongs to rows[k])."""
    r_rows = np.ascontiguousarray(np.asarray(r_rows, dtype=np.float64).reshape(-1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if out is None:
        out = np.zeros(geom.n_cols, dtype=np.float64)
    axis, c0, c1 = _block_args(geom, block)
    rc = _lib().orc_bp_rows(ctypes.byref(geom._c), _dptr(r_rows), _iptr(rows), rows.size,
                            axis, c0, c1, _dptr(out))
    if rc != 0:
        raise RuntimeError("orc_bp_rows failed (%d)" % rc)
    return out


def count_rows(geom: Geometry, rows, block=None) -> int:
    """Voxel-ray updates of one forward (or one back) projection over these
    rows and block: (ray, voxel) pairs longer than 1e-4 of the smallest voxel
    edge (shorter pieces are edge / corner crossings, zero in exact arithmetic)."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    axis, c0, c1 = _block_args(geom, block)
    n = _lib().orc_count_rows(ctypes.byref(geom._c), _iptr(rows), rows.size, axis, c0, c1)
    if n < 0:
        raise RuntimeError("orc_count_rows failed")
    return int(n)


def fp(geom: Geometry, x, views=None, block=None) -> np.ndarray:
    """Full-sinogram forward projection (rows of unlisted views are zero)."""
    views = np.arange(geom.n_views) if views is None else np.asarray(views)
    rows = rows_of_views(geom, views)
    y = np.zeros(geom.n_rows, dtype=np.float64)
    y[rows] = fp_rows(geom, x, rows, block)
    return y.reshape(geom.sino_shape)


def bp(geom: Geometry, r, views=None, block=None) -> np.ndarray:
    """A^T r over the listed views and block (full-volume array)."""
    views = np.arange(geom.n_views) if views is None else np.asarray(views)
    rows = rows_of_views(geom, views)
    r = np.asarray(r, dtype=np.float64).reshape(-1)
    return bp_rows(geom, r[rows], rows, block).reshape(geom.vol_shape)


def dense_matrix(geom: Geometry) -> np.ndarray:
    """Explicit A (rows x cols) assembled ray by ray from the traversal."""
    A = np.zeros((geom.n_rows, geom.n_cols))
    for a in range(geom.n_views):
        for v in range(geom.nv):
            for u in range(geom.nu):
                vox, ln = trace_ray(geom, a, v, u)
                np.add.at(A[(a * geom.nv + v) * geom.nu + u], vox, ln)
    return A


# --------------------------------------------------------------------------
# Detector footprint of a column block (used by the residual-norm weights)

def _box_corners(geom: Geometry, N: int, j: int) -> np.ndarray:
    c0, c1 = column_block(geom, N, j)
    lo = np.array([-0.5 * geom.nx * geom.dx, -0.5 * geom.ny * geom.dy, -0.5 * geom.nz * geom.dz])
    h = np.array([geom.dx, geom.dy, geom.dz])
    n = np.array([geom.nx, geom.ny, geom.nz], dtype=np.float64)
    blo, bhi = lo.copy(), lo + n * h
    ax = geom.block_axis
    blo[ax] = lo[ax] + c0 * h[ax]
    bhi[ax] = lo[ax] + c1 * h[ax]
    return np.array([[blo[0] if i & 1 == 0 else bhi[0],
                      blo[1] if i & 2 == 0 else bhi[1],
                      blo[2] if i & 4 == 0 else bhi[2]] for i in range(8)])


def view_cos_sin(t: float):
    """cos and sin of view angle t; within 1e-9 rad of a multiple of pi / 2 the
    angle is that multiple exactly (axis-aligned directions, as in the C
    traversal)."""
    k = round(t / (math.pi / 2))
    if abs(t - k * (math.pi / 2)) <= 1e-9:
        return ((1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0))[k % 4]
    return math.cos(t), math.sin(t)


def footprint(geom: Geometry, a: int, N: int, j: int):
    """Detector coordinates (u, v) of the 8 corners of J_j's box seen from view a:
    the shadow of a convex box is the convex hull of its corners' shadows."""
    X = _box_corners(geom, N, j)
    c, s = view_cos_sin(geom.angles[a])
    xu = -s * X[:, 0] + c * X[:, 1]
    if geom.kind == "par2d":
        return xu, np.zeros_like(xu)
    depth = geom.dso - (c * X[:, 0] + s * X[:, 1])
    t = geom.dsd / depth
    return t * xu, t * X[:, 2]


def v_band(geom: Geometry, a: int, N: int, j: int):
    """Detector rows [v_lo, v_hi] whose pixel centres fall inside the v-extent
    of J_j's shadow at view a (empty when v_lo > v_hi)."""
    if geom.nv == 1:
        return 0, 0
    _, v = footprint(geom, a, N, j)
    off = 0.5 * (geom.nv - 1)
    lo = math.ceil(v.min() / geom.dv + off)
    hi = math.floor(v.max() / geom.dv + off)
    return max(lo, 0), min(hi, geom.nv - 1)


def row_block_v_band(geom: Geometry, M: int, N: int, i: int, j: int, view_block=None):
    """Union over the views of I_i of the v-bands of J_j: the detector rows R_ij
    whose residual mass weights pair (i, j)."""
    lo, hi = geom.nv, -1
    for a in row_block_views(geom, M, i, view_block):
        l, h = v_band(geom, int(a), N, j)
        if l <= h:
            lo, hi = min(lo, l), max(hi, h)
    return lo, hi
