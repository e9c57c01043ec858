"""Python binding of libexactmap (GB300 / sm_103a), the Exact SPH -> Voronoi
density mapping with the tree-based pseudo-particle front end.

The binding only marshals arguments into the C ABI declared in
``include/exactmap.h``; every step of the computation runs in the library's
CUDA kernels.  Functions keep the C names.  Arrays are torch CUDA tensors
(float64 / int64 / int32); torch provides device memory and streams only.

Importing this module loads the compiled library and raises ImportError if
it is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexactmap.so")

MAP_OK = 0
MAP_EINVAL = -1
MAP_ENOMEM = -2
MAP_ECUDA = -3
MAP_ETIMEOUT = -4
MAP_EDEGENERATE = -5
MAP_EHANDLE = -6
MAP_ECAPACITY = -7
MAP_FP64 = 0
MAP_MIXED = 1
MAP_TABLE = 2

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libexactmap.so not built ({LIB_PATH}); run paper_2404_17084_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


class map_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("theta", ctypes.c_double), ("hfact", ctypes.c_double), ("leaf_size", ctypes.c_int),
                ("ngb_bruteforce_max", ctypes.c_int), ("autotune", ctypes.c_int),
                ("queue_timeout_ns", ctypes.c_ulonglong), ("count_work", ctypes.c_int), ("table_n", ctypes.c_int)]


class map_particles(ctypes.Structure):
    _fields_ = [("n", _I64), ("x", _P), ("y", _P), ("z", _P), ("m", _P), ("h", _P)]


class map_grid(ctypes.Structure):
    _fields_ = [("ncell", _I64), ("nface", _I64), ("nloop", _I64), ("nvert", _I64), ("cell_face_off", _P),
                ("face_vert_off", _P), ("face_vert", _P), ("face_plane", _P), ("vx", _P), ("vy", _P), ("vz", _P),
                ("site", _P)]


class map_outputs(ctypes.Structure):
    _fields_ = [("cell_mass", _P), ("cell_rho", _P), ("cell_vol", _P)]


class map_stats(ctypes.Structure):
    _fields_ = [("n_pairs", _I64), ("n_edge_terms", _I64), ("n_fp64_terms", _I64), ("total_mass", ctypes.c_double),
                ("status", ctypes.c_int)]


_lib.map_config_default.argtypes = [ctypes.POINTER(map_config)]
_lib.map_config_default.restype = None
_lib.map_init.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(map_config)]
_lib.map_destroy.argtypes = [_P]
_lib.map_destroy.restype = None
_lib.map_strerror.argtypes = [ctypes.c_int]
_lib.map_strerror.restype = ctypes.c_char_p
_lib.map_grid_upload.argtypes = [_P, ctypes.POINTER(map_grid), ctypes.POINTER(ctypes.c_int), _P]
_lib.map_grid_release.argtypes = [_P, ctypes.c_int]
_lib.map_grid_volumes.argtypes = [_P, ctypes.c_int, _P, _P]
_lib.map_grid_build.argtypes = [_P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                _P, ctypes.POINTER(_I64), _P]
_lib.map_grid_sizes.argtypes = [_P, ctypes.c_int] + [ctypes.POINTER(_I64)] * 4
_lib.map_grid_copy.argtypes = [_P, ctypes.c_int] + [_P] * 8 + [_P]
_lib.map_particles_to_cells.argtypes = [_P, ctypes.POINTER(map_particles), ctypes.c_int, ctypes.POINTER(map_outputs), _P]
_lib.map_get_pairs.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I64)]
_lib.map_copy_pairs.argtypes = [_P, _P, _P, _P, _I64, _P]
_lib.map_cells_to_particles.argtypes = [_P, _P, _P, _I64, _P]
_lib.map_get_stats.argtypes = [_P, ctypes.POINTER(map_stats)]
_lib.map_get_work.argtypes = [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
_lib.map_get_timing.argtypes = [_P, ctypes.POINTER(ctypes.c_float)]
_lib.solve_h.argtypes = [_P, ctypes.POINTER(map_particles), _P, _P]
_lib.solve_h_batch.argtypes = [_P, ctypes.c_int, ctypes.POINTER(map_particles), ctypes.POINTER(_P), _P]
_lib.build_pseudo_particles.argtypes = [_P, ctypes.POINTER(map_particles), ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_int, ctypes.POINTER(map_particles), _P, _P,
                                        ctypes.POINTER(_I64), _P]
class map_walk(ctypes.Structure):
    _fields_ = [("src", _P), ("nsrc", ctypes.c_int), ("r_part", ctypes.c_double), ("r_leaf", ctypes.c_double),
                ("regions", _P), ("nregion", ctypes.c_int)]


_lib.map_device_peaks.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 3
_lib.map_device_peaks.restype = ctypes.c_int
_lib.solve_h_noalloc.argtypes = [_P, _P, _P, _I64, ctypes.c_double, _P, _P, _P]
_lib.solve_h_noalloc.restype = ctypes.c_int
_lib.build_pseudo_particles_walk.argtypes = [_P, ctypes.POINTER(map_particles), ctypes.POINTER(map_walk),
                                             ctypes.POINTER(map_particles), _P, _P, ctypes.POINTER(_I64), _P]


class map_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int), ("slots", ctypes.c_int),
                ("hbm_budget", ctypes.c_size_t), ("hfact", ctypes.c_double)]


class map_request(ctypes.Structure):
    _fields_ = [("n", _I64), ("x", _P), ("y", _P), ("z", _P), ("m", _P), ("ncell", _I64), ("nface", _I64),
                ("nloop", _I64), ("nvert", _I64), ("cell_face_off", _P), ("face_vert_off", _P),
                ("face_vert", _P), ("face_plane", _P), ("vx", _P), ("vy", _P), ("vz", _P), ("site", _P),
                ("cell_mass", _P), ("cell_rho", _P), ("h", _P), ("grid_id", _I64)]


class map_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_pairs", _I64), ("total_mass", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("bytes_reserved", ctypes.c_size_t)]


_lib.map_server_config_default.argtypes = [ctypes.POINTER(map_server_config)]
_lib.map_server_config_default.restype = None
_lib.map_server_create.argtypes = [ctypes.POINTER(map_server_config), ctypes.POINTER(_P)]
_lib.map_server_submit.argtypes = [_P, ctypes.POINTER(map_request), ctypes.POINTER(_I64)]
_lib.map_server_wait.argtypes = [_P, _I64, ctypes.POINTER(map_request_result)]
_lib.map_server_stats.argtypes = [_P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64),
                                  ctypes.POINTER(ctypes.c_size_t)]
_lib.map_server_grid_stats.argtypes = [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                       ctypes.POINTER(ctypes.c_size_t)]
_lib.map_server_destroy.argtypes = [_P]
_lib.map_server_destroy.restype = None
for _name in ("map_server_create", "map_server_submit", "map_server_wait", "map_server_stats", "map_server_grid_stats"):
    getattr(_lib, _name).restype = ctypes.c_int
_lib.map_batch.argtypes = [_P, ctypes.c_int, ctypes.POINTER(map_particles), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(map_outputs), _P, _P]
_lib.map_get_autotune.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_int)]
_lib.map_autotune_shapes.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
_lib.map_batch_graph_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]
_lib.solve_h_batch_graph_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
for _name in ("map_init", "map_grid_upload", "map_grid_release", "map_grid_volumes", "map_grid_build",
              "map_grid_sizes", "map_grid_copy", "map_particles_to_cells",
              "map_get_pairs", "map_copy_pairs", "map_cells_to_particles", "map_get_stats", "map_get_work",
              "map_get_timing", "solve_h", "build_pseudo_particles", "build_pseudo_particles_walk", "map_batch",
              "map_get_autotune", "map_autotune_shapes", "solve_h_batch", "map_batch_graph_stats",
              "solve_h_batch_graph_stats"):
    getattr(_lib, _name).restype = ctypes.c_int


class MapError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {map_strerror(code)} ({code})")
        self.code = code


def _check(code: int, where: str) -> None:
    if code != MAP_OK:
        raise MapError(code, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr_dev_or_pinned(t):
    if not t.is_contiguous() or not (t.is_cuda or t.is_pinned()):
        raise ValueError("expected a contiguous CUDA or page-locked host tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- C names

def map_strerror(code: int) -> str:
    return _lib.map_strerror(code).decode()


def map_config_default(**overrides) -> map_config:
    cfg = map_config()
    _lib.map_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def map_init(cfg: map_config | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(_lib.map_init(ctypes.byref(ctx), ctypes.byref(cfg) if cfg is not None else None), "map_init")
    return ctx


def map_destroy(ctx) -> None:
    _lib.map_destroy(ctx)


def make_particles(x, y, z, m=None, h=None) -> map_particles:
    return map_particles(int(x.numel()), _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h))


def map_grid_upload(ctx, g: dict, stream=None) -> int:
    """g: dict of CUDA or page-locked host tensors cell_face_off, face_vert_off
    (int64), face_vert (int32), face_plane ([nface,4] float64), vx, vy, vz,
    site ([ncell,3])."""
    P = _ptr_dev_or_pinned
    mg = map_grid(int(g["cell_face_off"].numel() - 1), int(g["face_vert_off"].numel() - 1),
                  int(g["face_vert"].numel()), int(g["vx"].numel()), P(g["cell_face_off"]),
                  P(g["face_vert_off"]), P(g["face_vert"]), P(g["face_plane"]), P(g["vx"]),
                  P(g["vy"]), P(g["vz"]), P(g["site"]))
    h = ctypes.c_int(-1)
    _check(_lib.map_grid_upload(ctx, ctypes.byref(mg), ctypes.byref(h), _stream(stream)), "map_grid_upload")
    return h.value


def map_grid_release(ctx, handle: int) -> None:
    _check(_lib.map_grid_release(ctx, handle), "map_grid_release")


def map_grid_volumes(ctx, handle: int, vol, stream=None) -> None:
    _check(_lib.map_grid_volumes(ctx, handle, _ptr(vol), _stream(stream)), "map_grid_volumes")


def map_particles_to_cells(ctx, p: map_particles, handle: int, cell_mass, cell_rho=None, cell_vol=None,
                           stream=None) -> None:
    out = map_outputs(_ptr(cell_mass), _ptr(cell_rho), _ptr(cell_vol))
    _check(_lib.map_particles_to_cells(ctx, ctypes.byref(p), handle, ctypes.byref(out), _stream(stream)),
           "map_particles_to_cells")


def map_batch(ctx, parts, handles, cell_mass, cell_rho=None, cell_vol=None, totals=None, stream=None) -> None:
    """Map len(parts) snapshots in one batched launch: parts[j] (map_particles)
    on resident grid handles[j], writing cell_mass[j] (and cell_rho[j],
    cell_vol[j] when given); totals: optional CUDA float64 tensor of
    len(parts) receiving sum_i M_i per snapshot."""
    n = len(parts)
    P = (map_particles * n)(*parts)
    H = (ctypes.c_int * n)(*handles)
    O = (map_outputs * n)(*[map_outputs(_ptr(cell_mass[j]), _ptr(cell_rho[j]) if cell_rho else None,
                                        _ptr(cell_vol[j]) if cell_vol else None) for j in range(n)])
    _check(_lib.map_batch(ctx, n, P, H, O, _ptr(totals), _stream(stream)), "map_batch")


AUTOTUNE_SHAPES = ["4 warps/CTA, 5 CTAs/SM", "4 warps/CTA, 4 CTAs/SM", "2 warps/CTA, 9 CTAs/SM",
                   "8 warps/CTA, 2 CTAs/SM"]
AUTOTUNE_ITEM_TARGETS = [16, 64, 256]


def map_autotune_shapes(ctx):
    """The autotuner's launch shapes as launched on the context's device:
    one dict per shape (warps_per_cta, ctas_per_sm, registers)."""
    w, c, r = (ctypes.c_int * 8)(), (ctypes.c_int * 8)(), (ctypes.c_int * 8)()
    n = ctypes.c_int()
    _check(_lib.map_autotune_shapes(ctx, w, c, r, ctypes.byref(n)), "map_autotune_shapes")
    return [{"warps_per_cta": w[i], "ctas_per_sm": c[i], "registers": r[i]} for i in range(n.value)]


def map_get_autotune(ctx):
    """(chosen trial, [ms per trial]) of the context's autotuner.  Trial
    t * len(AUTOTUNE_SHAPES) + v is work-item target AUTOTUNE_ITEM_TARGETS[t]
    (items per resident warp) with launch shape AUTOTUNE_SHAPES[v]."""
    c = ctypes.c_int()
    nv = ctypes.c_int()
    ms = (ctypes.c_float * 32)()
    _check(_lib.map_get_autotune(ctx, ctypes.byref(c), ms, ctypes.byref(nv)), "map_get_autotune")
    return c.value, [ms[i] for i in range(nv.value)]


def map_batch_graph_stats(ctx):
    """(captures, replays, fallbacks) of map_batch's whole-step graph."""
    v = [ctypes.c_int64() for _ in range(3)]
    _check(_lib.map_batch_graph_stats(ctx, *[ctypes.byref(x) for x in v]), "map_batch_graph_stats")
    return tuple(x.value for x in v)


def solve_h_batch_graph_stats(ctx):
    """(captures, replays) of solve_h_batch's whole-step graph."""
    v = [ctypes.c_int64() for _ in range(2)]
    _check(_lib.solve_h_batch_graph_stats(ctx, *[ctypes.byref(x) for x in v]), "solve_h_batch_graph_stats")
    return tuple(x.value for x in v)


# ---------------------------------------------------------------- serving

def map_server_config_default(**overrides) -> map_server_config:
    cfg = map_server_config()
    _lib.map_server_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


_server_keep = {}  # (server, ticket) -> host arrays kept alive until the wait


def map_server_create(cfg: map_server_config | None = None) -> ctypes.c_void_p:
    srv = ctypes.c_void_p()
    _check(_lib.map_server_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(srv)),
           "map_server_create")
    return srv


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


def map_server_submit(srv, x, y, z, m, grid, cell_mass, cell_rho=None, h=None, grid_id: int = -1) -> int:
    """Queue one request of host (numpy) arrays: particles x, y, z, m and a
    grid (synth.Grid or dict of its CSR arrays); cell_mass (ncell float64,
    written on completion) and optional cell_rho, h; grid_id >= 0 keeps the
    grid resident under that id for later requests.  Returns the ticket."""
    G = grid if isinstance(grid, dict) else {k: getattr(grid, k) for k in (
        "cell_face_off", "face_vert_off", "face_vert", "face_plane", "vx", "vy", "vz", "site")}
    keep = []
    def ptr(a, dt):
        arr, p = _host(a, dt)
        keep.append(arr)
        return p
    for out in (cell_mass, cell_rho, h):
        if out is not None and not (isinstance(out, np.ndarray) and out.dtype == np.float64
                                    and out.flags["C_CONTIGUOUS"]):
            raise ValueError("outputs must be contiguous float64 numpy arrays")
    req = map_request(len(x), ptr(x, np.float64), ptr(y, np.float64), ptr(z, np.float64), ptr(m, np.float64),
                      len(G["cell_face_off"]) - 1, len(G["face_vert_off"]) - 1, len(G["face_vert"]), len(G["vx"]),
                      ptr(G["cell_face_off"], np.int64), ptr(G["face_vert_off"], np.int64),
                      ptr(G["face_vert"], np.int32), ptr(G["face_plane"], np.float64), ptr(G["vx"], np.float64),
                      ptr(G["vy"], np.float64), ptr(G["vz"], np.float64), ptr(G["site"], np.float64),
                      ctypes.c_void_p(cell_mass.ctypes.data),
                      ctypes.c_void_p(cell_rho.ctypes.data) if cell_rho is not None else None,
                      ctypes.c_void_p(h.ctypes.data) if h is not None else None, int(grid_id))
    keep += [cell_mass, cell_rho, h]
    t = _I64()
    _check(_lib.map_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), "map_server_submit")
    _server_keep[(srv.value, t.value)] = keep
    return t.value


def map_server_wait(srv, ticket: int) -> map_request_result:
    res = map_request_result()
    _check(_lib.map_server_wait(srv, ticket, ctypes.byref(res)), "map_server_wait")
    _server_keep.pop((srv.value, ticket), None)
    return res


def map_server_grid_stats(srv):
    """(uploads, hits, resident grids, resident bytes)."""
    u, hh, r = _I64(), _I64(), _I64()
    b = ctypes.c_size_t()
    _check(_lib.map_server_grid_stats(srv, ctypes.byref(u), ctypes.byref(hh), ctypes.byref(r), ctypes.byref(b)),
           "map_server_grid_stats")
    return u.value, hh.value, r.value, b.value


def map_server_stats(srv):
    """(completed, running, queued, held_bytes)."""
    c, q = _I64(), _I64()
    r = ctypes.c_int()
    b = ctypes.c_size_t()
    _check(_lib.map_server_stats(srv, ctypes.byref(c), ctypes.byref(r), ctypes.byref(q), ctypes.byref(b)),
           "map_server_stats")
    return c.value, r.value, q.value, b.value


def map_server_destroy(srv) -> None:
    _lib.map_server_destroy(srv)
    for k in [k for k in _server_keep if k[0] == srv.value]:
        _server_keep.pop(k, None)


def map_get_pairs(ctx):
    """(pair_off_ptr, pair_idx_ptr, pair_frac_ptr, n_pairs) of the last call (context-owned)."""
    a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(_lib.map_get_pairs(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)),
           "map_get_pairs")
    return a.value, b.value, c.value, n.value


def map_copy_pairs(ctx, ncell: int, device=None, stream=None):
    """The last call's pair list as new tensors (off int64, idx int32, frac float64)."""
    n = map_get_pairs(ctx)[3]
    dev = device or torch.device("cuda", torch.cuda.current_device())
    off = torch.empty(ncell + 1, dtype=torch.int64, device=dev)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    frac = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    _check(_lib.map_copy_pairs(ctx, _ptr(off), _ptr(idx), _ptr(frac), max(n, 1), _stream(stream)), "map_copy_pairs")
    return off, idx[:n], frac[:n]


def map_cells_to_particles(ctx, cell_value, particle_value, stream=None):
    """Inverse mapping (Eq. 4): particle_value[a] = sum_i cell_value[i] f_ai
    over the pairs of the last map_particles_to_cells call (float64 CUDA
    tensors: ncell values in, one per particle out)."""
    for t in (cell_value, particle_value):
        if t.dtype != torch.float64:
            raise ValueError("expected float64 tensors")
    _check(_lib.map_cells_to_particles(ctx, _ptr(cell_value), _ptr(particle_value), particle_value.numel(),
                                       _stream(stream)), "map_cells_to_particles")
    return particle_value


def map_grid_build(ctx, x, y, z, lloyd: int = 5, merge_tol: float = 0.0, kept=None, stream=None):
    """Grid construction on the device (Section II-A): merge, Lloyd
    iterations, Voronoi cells.  x, y, z: float64 CUDA tensors of the sites;
    kept: optional int64 CUDA tensor (capacity n) for the surviving site
    indices.  Returns (grid handle, number of cells)."""
    h = ctypes.c_int(-1)
    nk = _I64(0)
    _check(_lib.map_grid_build(ctx, _ptr(x), _ptr(y), _ptr(z), x.numel(), int(lloyd), float(merge_tol),
                               ctypes.byref(h), _ptr(kept), ctypes.byref(nk), _stream(stream)), "map_grid_build")
    return h.value, nk.value


def map_grid_sizes(ctx, handle: int):
    v = [_I64(0) for _ in range(4)]
    _check(_lib.map_grid_sizes(ctx, handle, *[ctypes.byref(a) for a in v]), "map_grid_sizes")
    return tuple(a.value for a in v)


def map_grid_copy(ctx, handle: int, device=None, stream=None) -> dict:
    """A resident grid's arrays as new CUDA tensors (the layout of map_grid)."""
    nc, nf, nl, nv = map_grid_sizes(ctx, handle)
    dev = device or torch.device("cuda", torch.cuda.current_device())
    e = lambda n, dt: torch.empty(max(n, 1), dtype=dt, device=dev)
    out = dict(cell_face_off=e(nc + 1, torch.int64), face_vert_off=e(nf + 1, torch.int64),
               face_vert=e(nl, torch.int32), face_plane=e(4 * nf, torch.float64), vx=e(nv, torch.float64),
               vy=e(nv, torch.float64), vz=e(nv, torch.float64), site=e(3 * nc, torch.float64))
    _check(_lib.map_grid_copy(ctx, handle, *[_ptr(out[k]) for k in ("cell_face_off", "face_vert_off", "face_vert",
                                                                     "face_plane", "vx", "vy", "vz", "site")],
                              _stream(stream)), "map_grid_copy")
    out["face_vert"] = out["face_vert"][:nl]
    out["face_plane"] = out["face_plane"][:4 * nf].view(nf, 4) if nf else out["face_plane"][:0].view(0, 4)
    for k in ("vx", "vy", "vz"):
        out[k] = out[k][:nv]
    out["site"] = out["site"][:3 * nc].view(nc, 3)
    return out


def map_get_stats(ctx) -> map_stats:
    st = map_stats()
    _check(_lib.map_get_stats(ctx, ctypes.byref(st)), "map_get_stats")
    return st


def map_get_work(ctx):
    """(dict of per-class work counts of the last mapping call, kernel launches so far)."""
    arr = (_I64 * 6)()
    nl = _I64()
    _check(_lib.map_get_work(ctx, arr, ctypes.byref(nl)), "map_get_work")
    return dict(face_tests=arr[0], edge_records=arr[1], inner_evals=arr[2], mid_intervals=arr[3],
                outer_intervals=arr[4], mid_split=arr[5]), nl.value


def map_get_timing(ctx):
    """Device ms of the latest phases: dict(tree, pairs, integrals, solve_h)."""
    arr = (ctypes.c_float * 4)()
    _check(_lib.map_get_timing(ctx, arr), "map_get_timing")
    return dict(tree=arr[0], pairs=arr[1], integrals=arr[2], solve_h=arr[3])


def solve_h(ctx, p: map_particles, route=None, stream=None) -> None:
    _check(_lib.solve_h(ctx, ctypes.byref(p), _ptr(route), _stream(stream)), "solve_h")


def solve_h_batch(ctx, parts, routes=None, stream=None) -> None:
    """solve_h for a list of particle sets (map_particles) at once; routes:
    None or a list of int32 CUDA tensors / None."""
    n = len(parts)
    P = (map_particles * n)(*parts)
    R = None
    if routes is not None:
        R = (_P * n)(*[_ptr(r) if r is not None else None for r in routes])
    _check(_lib.solve_h_batch(ctx, n, P, R, _stream(stream)), "solve_h_batch")


def map_device_peaks(device: int = 0) -> dict:
    """Measured issue rates (lane operations per second) of the FP32 FMA, the
    special-function (reciprocal square root) and the FP64 FMA pipes."""
    v = [ctypes.c_double(0.0) for _ in range(3)]
    _check(_lib.map_device_peaks(int(device), *[ctypes.byref(a) for a in v]), "map_device_peaks")
    return {"ffma": v[0].value, "mufu": v[1].value, "dfma": v[2].value}


def solve_h_noalloc(x, y, z, h, route=None, hfact: float = 1.2, stream=None) -> None:
    """solve_h without a context or device allocations (at most 32768
    particles; see the header): x, y, z, h float64 CUDA tensors of one length
    on the current device, route an optional int32 CUDA tensor of that
    length.  The library writes h and route through raw pointers, so their
    types, lengths and device are checked here first (ValueError)."""
    n = x.numel()
    dev = torch.cuda.current_device()
    for name, t, dt in (("x", x, torch.float64), ("y", y, torch.float64), ("z", z, torch.float64),
                        ("h", h, torch.float64), ("route", route, torch.int32)):
        if t is None and name == "route":
            continue
        if t.dtype != dt or t.numel() != n or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"solve_h_noalloc: {name} must be a {dt} CUDA tensor of {n} elements on "
                             f"cuda:{dev} (got {t.dtype}, {t.numel()} on {t.device})")
    _check(_lib.solve_h_noalloc(_ptr(x), _ptr(y), _ptr(z), n, float(hfact), _ptr(h), _ptr(route),
                                _stream(stream)), "solve_h_noalloc")


def build_pseudo_particles_walk(ctx, full: map_particles, src, out: map_particles, kind=None, ident=None,
                                r_part=0.0, r_leaf=0.0, regions=None, stream=None):
    """build_pseudo_particles through the walk-controls entry point (Section
    III-B: r_part, r_leaf, regions of an earlier step, several sources)."""
    srcs = [float(v) for v in np.asarray(src, dtype=np.float64).ravel()]
    arr = (ctypes.c_double * len(srcs))(*srcs)
    regs = [] if regions is None else [float(v) for v in np.asarray(regions, dtype=np.float64).ravel()]
    rarr = (ctypes.c_double * max(len(regs), 1))(*regs)
    walk = map_walk(ctypes.cast(arr, _P), len(srcs) // 3, float(r_part), float(r_leaf),
                    ctypes.cast(rarr, _P) if regs else None, len(regs) // 5)
    n = ctypes.c_int64(0)
    code = _lib.build_pseudo_particles_walk(ctx, ctypes.byref(full), ctypes.byref(walk), ctypes.byref(out),
                                            _ptr(kind), _ptr(ident), ctypes.byref(n), _stream(stream))
    if code != MAP_OK:
        err = MapError(code, "build_pseudo_particles_walk")
        err.required = n.value
        raise err
    return n.value


def build_pseudo_particles(ctx, full: map_particles, src, out: map_particles, kind=None, ident=None, stream=None,
                           r_part=0.0, r_leaf=0.0, regions=None):
    """Returns the number of pseudo-particles written (raises MapError with
    code MAP_ECAPACITY, attribute .required, if out is too small).  src: one
    or more source positions (flat or k x 3); r_part, r_leaf, regions (k x 5:
    centre, radius, smallest size): the walk controls of Section III-B."""
    srcs = [float(v) for v in np.asarray(src, dtype=np.float64).ravel()]
    arr = (ctypes.c_double * len(srcs))(*srcs)
    n = ctypes.c_int64(0)
    if r_part == 0.0 and r_leaf == 0.0 and regions is None:
        code = _lib.build_pseudo_particles(ctx, ctypes.byref(full), arr, len(srcs) // 3, ctypes.byref(out),
                                           _ptr(kind), _ptr(ident), ctypes.byref(n), _stream(stream))
    else:
        return build_pseudo_particles_walk(ctx, full, src, out, kind, ident, r_part, r_leaf, regions, stream)
    if code != MAP_OK:
        err = MapError(code, "build_pseudo_particles")
        err.required = n.value
        raise err
    return n.value


# ---------------------------------------------------------------- convenience

def grid_to_device(grid, device="cuda") -> dict:
    """Copy a host grid (any object with the CSR numpy arrays) to CUDA tensors."""
    t = lambda a, dt: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
    return dict(cell_face_off=t(grid.cell_face_off, torch.int64), face_vert_off=t(grid.face_vert_off, torch.int64),
                face_vert=t(grid.face_vert, torch.int32), face_plane=t(grid.face_plane, torch.float64),
                vx=t(grid.vx, torch.float64), vy=t(grid.vy, torch.float64), vz=t(grid.vz, torch.float64),
                site=t(grid.site, torch.float64))


class ExactMapper:
    """A context plus the resident grids it owns (one GPU, one host thread)."""

    def __init__(self, precision: int = MAP_MIXED, device: int = 0, **cfg):
        self.device = torch.device("cuda", device)
        self.cfg = map_config_default(precision=precision, device=device, **cfg)
        self.ctx = map_init(self.cfg)

    def close(self):
        if self.ctx:
            map_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, grid) -> int:
        g = grid if isinstance(grid, dict) else grid_to_device(grid, self.device)
        return map_grid_upload(self.ctx, g)

    def map(self, handle: int, ncell: int, x, y, z, m, h, stream=None):
        mass = torch.empty(ncell, dtype=torch.float64, device=self.device)
        rho = torch.empty(ncell, dtype=torch.float64, device=self.device)
        p = make_particles(x, y, z, m, h)
        map_particles_to_cells(self.ctx, p, handle, mass, rho, None, stream)
        return mass, rho

    def solve_h(self, x, y, z, stream=None):
        h = torch.empty_like(x)
        route = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
        solve_h(self.ctx, make_particles(x, y, z, None, h), route, stream)
        return h, route
