"""solve_h_noalloc: the smoothing-length solve for callers that cannot
allocate device memory (a fixed memory reservation, an allocation-free
pipeline).  It must give the same smoothing lengths as solve_h, call after
call, while using only the library's fixed scratch array.

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


def test_solve_h_noalloc_matches_solve_h_twice():
    L = lib()
    fn = _noalloc()
    p = synth.lognormal_particles(20000, synth.BASE_SEED + 7, sigma=1.5, ngrid=32)
    x, y, z, _, h_ref = dev_particles(p)
    route_ref = torch.empty(p.n, dtype=torch.int32, device="cuda")
    ctx = L.map_init(L.map_config_default(precision=0))
    try:
        L.solve_h(ctx, L.make_particles(x, y, z, None, h_ref), route_ref)
    finally:
        L.map_destroy(ctx)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        h = torch.full_like(x, float("nan"))
        route = torch.full((p.n,), -1, dtype=torch.int32, device="cuda")
        rc = fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()), p.n,
                1.2, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(route.data_ptr()), stream)
        torch.cuda.synchronize()
        assert rc == 0, L.map_strerror(rc)
        hd, hr = h.cpu().numpy(), h_ref.cpu().numpy()
        assert np.all(np.isfinite(hd))
        assert np.max(np.abs(hd / hr - 1)) < 1e-9
        assert torch.equal(route, route_ref)


def test_solve_h_noalloc_rejects_oversize():
    L = lib()
    fn = _noalloc()
    n = 32769  # one above the documented maximum
    x = torch.full((n,), 0.5, dtype=torch.float64, device="cuda")
    h = torch.empty_like(x)
    rc = fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, 1.2,
            ctypes.c_void_p(h.data_ptr()), None, None)
    assert rc == L.MAP_ECAPACITY
