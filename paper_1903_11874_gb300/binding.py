"""Thin ctypes binding of the BSGD C ABI (include/bsgd.h).

Argument marshalling only: every function forwards to the entry point of the
same name in libbsgd.so, which runs the work in the library's CUDA kernels.
torch supplies device memory and the current stream. There is no fallback:
if the library cannot be loaded, every call raises.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

F32, BF16, F16 = 0, 1, 2
PAR2D, FAN2D, CONE3D = 0, 1, 2
KINDS = {"par2d": PAR2D, "fan2d": FAN2D, "cone3d": CONE3D}
STEP_STRIP, STEP_BLOCK, STEP_FIXED = 0, 1, 2
PAIRS_UNIFORM, PAIRS_RESIDUAL = 0, 1
CELLS_NONE, CELLS_GEOMETRIC, CELLS_UNIFORM = 0, 1, 2
SERVE_SHARED, SERVE_AGE = 0, 1

# Every symbol include/bsgd.h declares.
EXPORTS = (
    "bsgd_last_error", "bsgd_status_string", "bsgd_geometry_create", "bsgd_geometry_destroy",
    "bsgd_geometry_get_info", "bsgd_geometry_pair_rays", "bsgd_forward_project", "bsgd_back_project", "bsgd_count_updates",
    "bsgd_count_updates_noalloc", "bsgd_power_iteration", "bsgd_tv_prox", "bsgd_state_create", "bsgd_state_destroy",
    "bsgd_block_step", "bsgd_state_query", "bsgd_state_read_residual", "bsgd_trace_stride",
    "bsgd_state_read_trace", "bsgd_state_set_shard", "bsgd_shard_begin", "bsgd_shard_end",
    "bsgd_state_set_replay", "bsgd_state_profile", "bsgd_state_read_profile",
    "bsgd_state_set_split", "bsgd_state_set_sampling", "bsgd_state_checkpoint_bytes",
    "bsgd_state_save", "bsgd_state_restore", "bsgd_solve",
    "bsgd_request_bytes", "bsgd_server_create", "bsgd_server_destroy", "bsgd_server_submit",
    "bsgd_server_wait", "bsgd_server_read_trace", "bsgd_server_poll", "bsgd_server_get_stats",
)
STAGES = ("sample", "fp", "residual", "bp", "update", "tv", "fpbp")


class BSGDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, status), message))
        self.status = status


_STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timeout",
           5: "over budget", 6: "invalid state"}


class GeometryDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("n_views", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("view_block", ctypes.POINTER(ctypes.c_int32)),
    ]


class GeometryInfo(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
        ("M", ctypes.c_int), ("N", ctypes.c_int), ("block_axis", ctypes.c_int),
        ("max_views_per_block", ctypes.c_int), ("max_block_cols", ctypes.c_int64),
        ("compact_rows", ctypes.c_int64),
    ]


class SolveParamsC(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("gamma", ctypes.c_double), ("epochs", ctypes.c_int),
        ("step_rule", ctypes.c_int), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
        ("power_iters", ctypes.c_int), ("pair_sampling", ctypes.c_int), ("cells", ctypes.c_int),
        ("n_cells", ctypes.c_int), ("tv_lambda", ctypes.c_double), ("tv_iters", ctypes.c_int),
        ("storage", ctypes.c_int), ("seed", ctypes.c_uint64),
        ("auto_mu", ctypes.c_int), ("auto_window", ctypes.c_int), ("auto_eps", ctypes.c_double),
        ("auto_delta", ctypes.c_double), ("auto_t1", ctypes.c_double), ("auto_t2", ctypes.c_double),
        ("final_uniform_epochs", ctypes.c_int), ("zero_start", ctypes.c_int),
        ("image_plain", ctypes.c_int),
    ]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 7), ("ms", ctypes.c_double * 7)]


class Report(ctypes.Structure):
    _fields_ = [
        ("residual_norm", ctypes.c_double), ("mu", ctypes.c_double),
        ("iteration", ctypes.c_int64), ("epoch", ctypes.c_double), ("updates", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("device", ctypes.c_int),
                ("priority", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("resident", ctypes.c_int64),
        ("peak_resident", ctypes.c_int), ("bytes_resident", ctypes.c_size_t),
        ("peak_bytes", ctypes.c_size_t), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("updates", ctypes.c_int64),
        ("busy_s", ctypes.c_double), ("rounds", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_vp, _i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbsgd.so (building it first if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise BSGDError(3, "libbsgd.so not found at %s" % path)
    lib = ctypes.CDLL(path)
    st = ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "bsgd_last_error": (ctypes.c_char_p, []),
        "bsgd_status_string": (ctypes.c_char_p, [st]),
        "bsgd_geometry_create": (st, [P(GeometryDesc), ctypes.c_int, ctypes.c_int, P(_vp)]),
        "bsgd_geometry_destroy": (st, [_vp]),
        "bsgd_geometry_get_info": (st, [_vp, P(GeometryInfo)]),
        "bsgd_geometry_pair_rays": (st, [_vp, ctypes.c_int, ctypes.c_int, P(ctypes.c_int64)]),
        "bsgd_forward_project": (st, [_vp, _vp, st, _vp, st, _i32p, ctypes.c_int, _i32p,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
        "bsgd_back_project": (st, [_vp, _vp, st, _vp, st, _i32p, ctypes.c_int, _i32p,
                                   ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, _vp]),
        "bsgd_count_updates": (st, [_vp, _i32p, ctypes.c_int, _i32p, ctypes.c_int,
                                    P(ctypes.c_int64), _vp]),
        "bsgd_count_updates_noalloc": (st, [_vp, _i32p, ctypes.c_int, _i32p, ctypes.c_int,
                                            P(ctypes.c_int64), _vp]),
        "bsgd_power_iteration": (st, [_vp, ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int,
                                      P(ctypes.c_double), _vp]),
        "bsgd_tv_prox": (st, [_vp, _vp, st, ctypes.c_double, ctypes.c_int, _vp]),
        "bsgd_state_create": (st, [_vp, P(SolveParamsC), _vp, st, _vp, P(_vp)]),
        "bsgd_state_destroy": (st, [_vp]),
        "bsgd_block_step": (st, [_vp, _vp, ctypes.c_int, _vp]),
        "bsgd_state_query": (st, [_vp, P(Report), _vp]),
        "bsgd_state_read_residual": (st, [_vp, _vp, st, _vp]),
        "bsgd_state_set_shard": (st, [_vp, _i32p, ctypes.c_int, P(ctypes.c_int64)]),
        "bsgd_shard_begin": (st, [_vp, _vp, _vp, _vp]),
        "bsgd_shard_end": (st, [_vp, _vp, _vp, _vp]),
        "bsgd_trace_stride": (ctypes.c_int64, [_vp]),
        "bsgd_state_read_trace": (st, [_vp, _i32p, ctypes.c_int64, ctypes.c_int64, _vp]),
        "bsgd_state_set_replay": (st, [_vp, _i32p, ctypes.c_int64]),
        "bsgd_state_profile": (st, [_vp, ctypes.c_int]),
        "bsgd_state_set_split": (st, [_vp, ctypes.c_int]),
        "bsgd_state_checkpoint_bytes": (st, [_vp, P(ctypes.c_int64)]),
        "bsgd_state_save": (st, [_vp, _vp, ctypes.c_int64, _vp]),
        "bsgd_state_restore": (st, [_vp, _vp, ctypes.c_int64, _vp]),
        "bsgd_state_set_sampling": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
        "bsgd_state_read_profile": (st, [_vp, P(Profile), _vp]),
        "bsgd_solve": (st, [_vp, P(SolveParamsC), _vp, st, _vp, st, P(Report), _vp]),
        "bsgd_request_bytes": (st, [P(GeometryDesc), ctypes.c_int, ctypes.c_int, P(SolveParamsC),
                                    P(ctypes.c_size_t)]),
        "bsgd_server_create": (st, [P(ServerParams), P(_vp)]),
        "bsgd_server_destroy": (st, [_vp]),
        "bsgd_server_submit": (st, [_vp, P(GeometryDesc), ctypes.c_int, ctypes.c_int,
                                    P(SolveParamsC), _vp, st, ctypes.POINTER(ctypes.c_float),
                                    P(ctypes.c_int64)]),
        "bsgd_server_wait": (st, [_vp, ctypes.c_int64, ctypes.c_int, P(Report)]),
        "bsgd_server_read_trace": (st, [_vp, ctypes.c_int64, _i32p, ctypes.c_int64,
                                        P(ctypes.c_int64), P(ctypes.c_int64)]),
        "bsgd_server_poll": (st, [_vp, ctypes.c_int64, P(ctypes.c_int)]),
        "bsgd_server_get_stats": (st, [_vp, P(ServerStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status):
    if status != 0:
        msg = load().bsgd_last_error()
        raise BSGDError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# torch marshalling helpers (torch is imported lazily: the build and the CPU
# tests do not need a GPU)

def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    m = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
    if t.dtype not in m:
        raise BSGDError(1, "unsupported dtype %s" % t.dtype)
    return m[t.dtype]


def _dev_ptr(t, what):
    if not t.is_cuda:
        raise BSGDError(1, "%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise BSGDError(1, "%s must be contiguous" % what)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ids(ids):
    if ids is None:
        return None, 0, None
    arr = np.ascontiguousarray(np.asarray(ids, dtype=np.int32).reshape(-1))
    return arr.ctypes.data_as(_i32p), int(arr.size), arr


# ---------------------------------------------------------------------------
# Geometry

def make_desc(kind, nx, ny, nz, dx, dy, dz, n_views, nu, nv, du, dv, dso=0.0, dsd=0.0,
              angles=None, view_block=None):
    """A bsgd_geometry_desc and the arrays it points to (keep them alive)."""
    ang = None if angles is None else np.ascontiguousarray(angles, dtype=np.float64)
    vb = None if view_block is None else np.ascontiguousarray(view_block, dtype=np.int32)
    d = GeometryDesc(KINDS[kind] if isinstance(kind, str) else int(kind), int(nx), int(ny), int(nz),
                     float(dx), float(dy), float(dz), int(n_views),
                     None if ang is None else ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     int(nu), int(nv), float(du), float(dv), float(dso), float(dsd),
                     None if vb is None else vb.ctypes.data_as(_i32p))
    return d, (ang, vb)


class Geometry:
    """Owning handle of a bsgd_geometry (bsgd_geometry_create / _destroy)."""

    def __init__(self, kind, nx, ny, nz, dx, dy, dz, n_views, nu, nv, du, dv, dso=0.0, dsd=0.0,
                 angles=None, view_block=None, M=1, N=1):
        lib = load()
        self.kind = kind
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz = float(dx), float(dy), float(dz)
        self.n_views, self.nu, self.nv = int(n_views), int(nu), int(nv)
        self.du, self.dv, self.dso, self.dsd = float(du), float(dv), float(dso), float(dsd)
        d, self._keep = make_desc(kind, nx, ny, nz, dx, dy, dz, n_views, nu, nv, du, dv, dso, dsd,
                                  angles, view_block)
        h = ctypes.c_void_p()
        _check(lib.bsgd_geometry_create(ctypes.byref(d), int(M), int(N), ctypes.byref(h)))
        self.handle = h
        info = GeometryInfo()
        _check(lib.bsgd_geometry_get_info(h, ctypes.byref(info)))
        self.info = info
        self.M, self.N = info.M, info.N

    @property
    def n_rows(self):
        return int(self.info.n_rows)

    @property
    def compact_rows(self):
        return int(self.info.compact_rows)

    @property
    def n_cols(self):
        return int(self.info.n_cols)

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.n_views, self.nv, self.nu)

    def pair_rays(self, i, j) -> int:
        out = ctypes.c_int64()
        _check(load().bsgd_geometry_pair_rays(self.handle, int(i), int(j), ctypes.byref(out)))
        return int(out.value)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(load().bsgd_geometry_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bsgd_geometry_create(**kw) -> Geometry:
    return Geometry(**kw)


def bsgd_forward_project(geom, x, y, row_blocks=None, col_blocks=None, accumulate=False,
                         batch=1, stream=None):
    rp, nr, _ra = _ids(row_blocks)
    cp, nc, _ca = _ids(col_blocks)
    _check(load().bsgd_forward_project(geom.handle, _dev_ptr(x, "x"), dtype_code(x),
                                       _dev_ptr(y, "y"), dtype_code(y), rp, nr, cp, nc,
                                       int(bool(accumulate)), int(batch), _stream(stream)))
    return y


def bsgd_back_project(geom, r, x, row_blocks=None, col_blocks=None, scale=1.0, accumulate=False,
                      batch=1, stream=None):
    rp, nr, _ra = _ids(row_blocks)
    cp, nc, _ca = _ids(col_blocks)
    _check(load().bsgd_back_project(geom.handle, _dev_ptr(r, "r"), dtype_code(r),
                                    _dev_ptr(x, "x"), dtype_code(x), rp, nr, cp, nc,
                                    float(scale), int(bool(accumulate)), int(batch),
                                    _stream(stream)))
    return x


def bsgd_count_updates(geom, row_blocks=None, col_blocks=None, stream=None) -> int:
    rp, nr, _ra = _ids(row_blocks)
    cp, nc, _ca = _ids(col_blocks)
    out = ctypes.c_int64()
    _check(load().bsgd_count_updates(geom.handle, rp, nr, cp, nc, ctypes.byref(out),
                                     _stream(stream)))
    return int(out.value)


def bsgd_count_updates_noalloc(geom, row_blocks=None, col_blocks=None, stream=None) -> int:
    """bsgd_count_updates for callers that cannot allocate device memory: the
    library keeps its counters in a fixed device array (at most 16384 views)."""
    rp, nr, _ra = _ids(row_blocks)
    cp, nc, _ca = _ids(col_blocks)
    out = ctypes.c_int64()
    _check(load().bsgd_count_updates_noalloc(geom.handle, rp, nr, cp, nc, ctypes.byref(out),
                                             _stream(stream)))
    return int(out.value)


def bsgd_power_iteration(geom, col_block, iters=30, row_blocks=None, stream=None) -> float:
    rp, nr, _ra = _ids(row_blocks)
    out = ctypes.c_double()
    _check(load().bsgd_power_iteration(geom.handle, int(col_block), int(iters), rp, nr,
                                       ctypes.byref(out), _stream(stream)))
    return float(out.value)


def bsgd_tv_prox(geom, x, kappa, iters=20, stream=None):
    _check(load().bsgd_tv_prox(geom.handle, _dev_ptr(x, "x"), dtype_code(x), float(kappa),
                               int(iters), _stream(stream)))
    return x


# ---------------------------------------------------------------------------
# Solver

@dataclass
class SolveParams:
    alpha: float
    gamma: float
    epochs: int = 1
    step_rule: int = STEP_STRIP
    mu: float = 0.0
    rho: float = 0.25
    power_iters: int = 30
    pair_sampling: int = PAIRS_UNIFORM
    cells: int = CELLS_NONE
    n_cells: int = 1
    tv_lambda: float = 0.0
    tv_iters: int = 20
    storage: int = F32
    seed: int = 1
    # Algorithm 3 (automatic step length); defaults: eps and the cosine
    # thresholds are readings, delta = 0.4 as in Sec. 5
    auto_mu: bool = False
    auto_window: int = 0
    auto_eps: float = 0.1
    auto_delta: float = 0.4
    auto_t1: float = 0.2
    auto_t2: float = 0.5
    # bsgd_solve: last epochs without importance sampling (after Algorithm 2)
    final_uniform_epochs: int = 0
    # bsgd_solve: start from x0 = 0 without reading x (otherwise x holds x0)
    zero_start: bool = False
    # 16-bit storage: the image without its low-order term (2 B / voxel)
    image_plain: bool = False

    def c(self):
        return SolveParamsC(self.alpha, self.gamma, self.epochs, self.step_rule, self.mu, self.rho,
                            self.power_iters, self.pair_sampling, self.cells, self.n_cells,
                            self.tv_lambda, self.tv_iters, self.storage, self.seed,
                            int(bool(self.auto_mu)), self.auto_window, self.auto_eps,
                            self.auto_delta, self.auto_t1, self.auto_t2,
                            int(self.final_uniform_epochs), int(bool(self.zero_start)),
                            int(bool(self.image_plain)))


class State:
    """Owning handle of a bsgd_state."""

    def __init__(self, geom, params: SolveParams, y, stream=None):
        self.geom, self.params = geom, params
        self._pc = params.c()
        h = ctypes.c_void_p()
        _check(load().bsgd_state_create(geom.handle, ctypes.byref(self._pc), _dev_ptr(y, "y"),
                                        dtype_code(y), _stream(stream), ctypes.byref(h)))
        self.handle = h

    def block_step(self, x, n_iters, stream=None):
        _check(load().bsgd_block_step(self.handle, _dev_ptr(x, "x"), int(n_iters), _stream(stream)))
        return x

    def query(self, stream=None) -> dict:
        rep = Report()
        _check(load().bsgd_state_query(self.handle, ctypes.byref(rep), _stream(stream)))
        return rep.as_dict()

    def read_residual(self, out, stream=None):
        """r = y - sum_j z^j into the device tensor out (n_rows elements)."""
        _check(load().bsgd_state_read_residual(self.handle, _dev_ptr(out, "out"), dtype_code(out),
                                               _stream(stream)))
        return out

    def set_shard(self, owned_blocks) -> int:
        """Mark the column blocks this process owns (owner-computes sharding);
        returns the length (floats) of the exchange buffer."""
        ids = np.ascontiguousarray(np.asarray(list(owned_blocks), dtype=np.int32))
        n = ctypes.c_int64()
        _check(load().bsgd_state_set_shard(self.handle, ids.ctypes.data_as(_i32p), int(ids.size),
                                           ctypes.byref(n)))
        return int(n.value)

    def shard_begin(self, x, exchange, stream=None):
        _check(load().bsgd_shard_begin(self.handle, _dev_ptr(x, "x"), _dev_ptr(exchange, "exchange"),
                                       _stream(stream)))

    def shard_end(self, x, exchange, stream=None):
        _check(load().bsgd_shard_end(self.handle, _dev_ptr(x, "x"), _dev_ptr(exchange, "exchange"),
                                     _stream(stream)))

    @property
    def trace_stride(self) -> int:
        return int(load().bsgd_trace_stride(self.handle))

    def save(self, stream=None) -> bytes:
        """Checkpoint of the state (bsgd_state_save); x and y are not in it."""
        n = ctypes.c_int64(0)
        _check(load().bsgd_state_checkpoint_bytes(self.handle, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(max(1, n.value))
        _check(load().bsgd_state_save(self.handle, ctypes.cast(buf, _vp), n.value, _stream(stream)))
        return buf.raw[: n.value]

    def restore(self, blob: bytes, stream=None):
        """Load a checkpoint of a state with the same geometry, parameters and y
        (bsgd_state_restore); continue with the x of the save."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(load().bsgd_state_restore(self.handle, ctypes.cast(buf, _vp), len(blob), _stream(stream)))

    def read_trace(self, n_iters, stream=None) -> np.ndarray:
        s = self.trace_stride
        buf = np.zeros(max(1, n_iters * s), dtype=np.int32)
        _check(load().bsgd_state_read_trace(self.handle, buf.ctypes.data_as(_i32p), buf.size,
                                            int(n_iters), _stream(stream)))
        return buf[: n_iters * s].reshape(n_iters, s)

    def set_replay(self, trace: np.ndarray):
        t = np.ascontiguousarray(trace, dtype=np.int32)
        n = 0 if t.size == 0 else t.shape[0]
        _check(load().bsgd_state_set_replay(self.handle, t.ctypes.data_as(_i32p), int(n)))

    def profile(self, enable=True):
        _check(load().bsgd_state_profile(self.handle, int(bool(enable))))

    def set_sampling(self, pair_sampling, cells=0, n_cells=1, stream=None):
        _check(load().bsgd_state_set_sampling(self.handle, int(pair_sampling), int(cells),
                                              int(n_cells), _stream(stream)))

    def set_split(self, split=True):
        _check(load().bsgd_state_set_split(self.handle, int(bool(split))))

    def read_profile(self, stream=None) -> dict:
        pr = Profile()
        _check(load().bsgd_state_read_profile(self.handle, ctypes.byref(pr), _stream(stream)))
        return {name: {"launches": int(pr.launches[k]), "ms": float(pr.ms[k])}
                for k, name in enumerate(STAGES)}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(load().bsgd_state_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bsgd_state_create(geom, params, y, stream=None) -> State:
    return State(geom, params, y, stream)


def bsgd_block_step(state: State, x, n_iters, stream=None):
    return state.block_step(x, n_iters, stream)


def bsgd_state_query(state: State, stream=None) -> dict:
    return state.query(stream)


def _any_ptr(t):
    """Device pointer for CUDA tensors, host pointer for CPU tensors / arrays."""
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise BSGDError(1, "array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    if not t.is_contiguous():
        raise BSGDError(1, "tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _any_dtype(t):
    if isinstance(t, np.ndarray):
        if t.dtype == np.float32:
            return F32
        if t.dtype == np.float16:
            return F16
        raise BSGDError(1, "numpy arrays must be float32 or float16")
    return dtype_code(t)


def bsgd_solve(geom, params: SolveParams, y, x, stream=None) -> dict:
    """One-call reconstruction; y and x may live on the host or the device."""
    pc = params.c()
    rep = Report()
    _check(load().bsgd_solve(geom.handle, ctypes.byref(pc), _any_ptr(y), _any_dtype(y),
                             _any_ptr(x), _any_dtype(x), ctypes.byref(rep), _stream(stream)))
    return rep.as_dict()


# ---------------------------------------------------------------------------
# Serving

def bsgd_request_bytes(geo: dict, M: int, N: int, params: SolveParams) -> int:
    """Device bytes a request holds while resident (the admission model)."""
    d, _keep = make_desc(**geo)
    pc = params.c()
    out = ctypes.c_size_t()
    _check(load().bsgd_request_bytes(ctypes.byref(d), int(M), int(N), ctypes.byref(pc),
                                     ctypes.byref(out)))
    return int(out.value)


class Server:
    """Owning handle of a bsgd_server: submit reconstructions, wait for them."""

    def __init__(self, budget_bytes, max_slots=16, device=0, priority=None):
        h = ctypes.c_void_p()
        prm = ServerParams(int(budget_bytes), int(max_slots), int(device),
                           SERVE_SHARED if priority is None else int(priority))
        _check(load().bsgd_server_create(ctypes.byref(prm), ctypes.byref(h)))
        self.handle = h
        self._pending = {}

    def submit(self, geo: dict, M: int, N: int, params: SolveParams, y: np.ndarray) -> int:
        """Queue a reconstruction of y (host float32 / float16 array); returns its id."""
        d, keep = make_desc(**geo)
        pc = params.c()
        y = np.ascontiguousarray(y)
        yt = {np.dtype(np.float32): F32, np.dtype(np.float16): F16}[y.dtype]
        nx, ny, nz = int(geo["nx"]), int(geo["ny"]), int(geo["nz"])
        x = np.zeros(nx * ny * nz, dtype=np.float32)
        rid = ctypes.c_int64()
        _check(load().bsgd_server_submit(self.handle, ctypes.byref(d), int(M), int(N),
                                         ctypes.byref(pc), ctypes.c_void_p(y.ctypes.data), yt,
                                         x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         ctypes.byref(rid)))
        self._pending[rid.value] = (x, keep)
        return int(rid.value)

    def wait(self, rid: int, timeout_ms: int = 600000):
        """(x, report) once request rid is done; BSGDError(TIMEOUT) if not in time."""
        rep = Report()
        _check(load().bsgd_server_wait(self.handle, int(rid), int(timeout_ms), ctypes.byref(rep)))
        x, _keep = self._pending[rid]
        return x, rep.as_dict()

    def read_trace(self, rid: int) -> np.ndarray:
        """Draws of finished request rid: an (iterations, stride) int32 array in
        the layout of State.read_trace."""
        stride, n = ctypes.c_int64(), ctypes.c_int64()
        _check(load().bsgd_server_read_trace(self.handle, int(rid), None, 0, ctypes.byref(stride),
                                             ctypes.byref(n)))
        buf = np.zeros(max(1, n.value * stride.value), dtype=np.int32)
        _check(load().bsgd_server_read_trace(self.handle, int(rid),
                                             buf.ctypes.data_as(_i32p), buf.size,
                                             ctypes.byref(stride), ctypes.byref(n)))
        return buf[:n.value * stride.value].reshape(n.value, stride.value)

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int()
        _check(load().bsgd_server_poll(self.handle, int(rid), ctypes.byref(done)))
        return bool(done.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().bsgd_server_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(load().bsgd_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
