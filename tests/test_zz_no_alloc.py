"""solve_h_noalloc: the smoothing-length solve for callers that cannot
allocate device memory (a process that has handed the GPU's memory to its own
pools, a pipeline that forbids allocation after start-up).  It must give the
same smoothing lengths as solve_h, bit for bit, call after call, while using
only the library's fixed scratch array: the device's free memory does not
move across calls.

Collected last on purpose (file name), so that a failure here comes after
every other test has run; it passes alone in a fresh process too."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import lib, dev_particles

pytestmark = pytest.mark.gpu


def _noalloc():
    L = lib()
    fn = L._lib.solve_h_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _ref_solve(x, y, z, n):
    """solve_h on an FP64 context: the entry point's reference."""
    L = lib()
    h = torch.empty_like(x)
    route = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx = L.map_init(L.map_config_default(precision=0))
    try:
        L.solve_h(ctx, L.make_particles(x, y, z, None, h), route)
        torch.cuda.synchronize()
    finally:
        L.map_destroy(ctx)
    return h, route


def _call(fn, x, y, z, n, h, route, stream):
    return fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()), n, 1.2,
              ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(route.data_ptr()), stream)


def test_solve_h_noalloc_matches_solve_h_twice():
    L = lib()
    fn = _noalloc()
    p = synth.lognormal_particles(20000, synth.BASE_SEED + 7, sigma=1.5, ngrid=32)
    x, y, z, _, _ = dev_particles(p)
    h_ref, route_ref = _ref_solve(x, y, z, p.n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # every buffer of the calls below exists before the first one
    hs = [torch.full_like(x, float("nan")) for _ in range(3)]
    routes = [torch.full((p.n,), -1, dtype=torch.int32, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    free = []
    for k in range(3):
        rc = _call(fn, x, y, z, p.n, hs[k], routes[k], stream)
        torch.cuda.synchronize()
        assert rc == 0, L.map_strerror(rc)
        free.append(torch.cuda.mem_get_info()[0])
        # the same kernels and the same order of sums as solve_h: equal bits
        assert torch.equal(hs[k], h_ref)
        assert torch.equal(routes[k], route_ref)
    # no device memory taken or returned by the calls after the first
    assert free[1] == free[0] and free[2] == free[0]


def test_solve_h_noalloc_dense_tree_fits():
    """The largest octree we could construct from at most 32768 particles:
    1927 groups of 17, each spread over the eight cells of one deepest-level
    node, so that every group keeps a chain of nodes down to level 20 and ends
    in eight leaves (about 48,000 nodes).  It fits the fixed node arrays and
    gives solve_h's result bit for bit."""
    L = lib()
    fn = _noalloc()
    d = 2.0 ** -21
    offs = np.array([[(o >> 2) & 1, (o >> 1) & 1, o & 1] for o in range(8)], float)
    rng = np.random.default_rng(1)
    base = np.floor(rng.random((1927, 3)) * 0.98 * 2**20 + 0.01 * 2**20) / 2**20
    pts = (base[:, None, :] + (offs[np.arange(17) % 8][None, :, :] + 0.5) * d).reshape(-1, 3)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, z = t(pts[:, 0]), t(pts[:, 1]), t(pts[:, 2])
    n = len(pts)
    h_ref, route_ref = _ref_solve(x, y, z, n)
    h = torch.full_like(x, float("nan"))
    route = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rc = _call(fn, x, y, z, n, h, route, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, L.map_strerror(rc)
    assert torch.equal(h, h_ref) and torch.equal(route, route_ref)


def test_solve_h_noalloc_rejects_oversize_and_capture():
    L = lib()
    fn = _noalloc()
    n = 32769  # one above the documented maximum
    x = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    h = torch.empty_like(x)
    rc = fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, 1.2,
            ctypes.c_void_p(h.data_ptr()), None, None)
    assert rc == L.MAP_ECAPACITY
    # a stream being captured is refused and its capture stays valid
    s = torch.cuda.Stream()
    xs = x[:1000].contiguous()
    hs = torch.empty_like(xs)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        rc = fn(ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(xs.data_ptr()), 1000,
                1.2, ctypes.c_void_p(hs.data_ptr()), None, ctypes.c_void_p(s.cuda_stream))
        hs.fill_(1.0)
        g.capture_end()
    assert rc == L.MAP_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert bool((hs == 1.0).all())
    # the binding checks types and lengths before the raw pointers are used
    with pytest.raises(ValueError):
        L.solve_h_noalloc(xs, xs, xs, hs.float())
    with pytest.raises(ValueError):
        L.solve_h_noalloc(xs, xs, xs, hs[:10])
