"""Serving loop (continuous batching): every request's result is the same
alone and in a mix of concurrent requests (bit-identical: each request runs
on its own context and stream and depends on its own inputs only), admission
holds the HBM budget, grids stay resident by id (reused without an upload,
evicted when memory runs short), and a served FP64 result matches the
oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import lib, dev_particles, oracle_h, rel_err, sample_cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def requests_():
    out = []
    for spec in synth.batch_specs(6, synth.BASE_SEED + 5, 10.0, 13.0):
        p = synth.batch_particles(spec)
        out.append((p, synth.voronoi(p.pos())))
    return out


def serve(reqs, precision=1, slots=4, budget=0, order=None):
    L = lib()
    srv = L.map_server_create(L.map_server_config_default(precision=precision, slots=slots, hbm_budget=budget))
    try:
        outs = [np.full(g.ncell, -1.0) for _, g in reqs]
        hs = [np.zeros(p.n) for p, _ in reqs]
        order = list(range(len(reqs))) if order is None else order
        tickets = {}
        for j in order:
            p, g = reqs[j]
            tickets[j] = L.map_server_submit(srv, p.x, p.y, p.z, p.m, g, outs[j], h=hs[j])
        res = {j: L.map_server_wait(srv, tickets[j]) for j in order}
        stats = L.map_server_stats(srv)
        return outs, hs, res, stats
    finally:
        L.map_server_destroy(srv)


def test_serve_same_alone_and_in_mix(requests_):
    alone = [serve([r], slots=1) for r in requests_]
    mix, hmix, res, stats = serve(requests_, slots=4, order=[3, 0, 5, 1, 4, 2])
    assert stats[0] == len(requests_) and stats[1] == 0 and stats[2] == 0
    for j in range(len(requests_)):
        assert res[j].status == 0 and res[j].latency_ms >= res[j].queue_ms >= 0.0
        assert np.array_equal(mix[j], alone[j][0][0]), j
        assert np.array_equal(hmix[j], alone[j][1][0]), j
        assert res[j].n_pairs == alone[j][2][0].n_pairs


def test_serve_matches_plain_api(requests_):
    """A served request equals solve_h + map_particles_to_cells on one context."""
    L = lib()
    outs, hs, res, _ = serve(requests_[:2], slots=2)
    for j, (p, g) in enumerate(requests_[:2]):
        ctx = L.map_init(L.map_config_default(precision=1))
        try:
            handle = L.map_grid_upload(ctx, L.grid_to_device(g))
            x, y, z, m, hh = dev_particles(p)
            L.solve_h(ctx, L.make_particles(x, y, z, None, hh))
            mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
            L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass)
            torch.cuda.synchronize()
            assert np.array_equal(outs[j], mass.cpu().numpy())
            assert np.array_equal(hs[j], hh.cpu().numpy())
        finally:
            L.map_destroy(ctx)


def test_serve_admission_budget(requests_):
    """A budget that fits one request at a time: the others queue, results
    are unchanged; a request larger than the budget fails alone."""
    L = lib()
    ref, _, _, _ = serve(requests_, slots=4)
    big = max(range(len(requests_)), key=lambda j: requests_[j][0].n)
    # estimate of the largest request (as the server computes it) + one small one's worth
    p, g = requests_[big]
    est = int(1.25 * (48.0 * p.n + 200.0 * p.n + 2560.0 * p.n + 96.0 * g.ncell + 130.0 * g.nface
                      + 160.0 * len(g.face_vert) + 48.0 * len(g.vx) + 24.0 * g.ncell)) + (64 << 20)
    outs, _, res, _ = serve(requests_, slots=4, budget=est + (8 << 20))
    queued = sum(1 for r in res.values() if r.queue_ms > 0.5)
    assert queued >= 1
    for j in range(len(requests_)):
        assert res[j].status == 0
        assert np.array_equal(outs[j], ref[j])
    # too large for the budget even alone
    outs2, _, res2, _ = serve(requests_[:2], slots=2, budget=32 << 20)
    assert all(r.status == L.MAP_ENOMEM for r in res2.values())


def test_serve_fp64_vs_oracle(requests_):
    outs, hs, res, _ = serve(requests_[:1], precision=0, slots=1)
    p, g = requests_[0]
    h_ref, _ = oracle_h(p)
    assert np.max(np.abs(hs[0] / h_ref - 1)) < 1e-9
    cells = sample_cells(g.ncell, 60, 1)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, hs[0], cells=cells)
    assert rel_err(outs[0][cells], ref["mass"]).max() < 1e-9


def _est(p, g):
    """The server's admission estimate (work, grid) of a mixed request, in bytes."""
    work = int(1.25 * ((48.0 + 200.0 + 2560.0) * p.n + 24.0 * g.ncell)) + (64 << 20)
    grid = int(1.25 * (96.0 * g.ncell + 146.0 * g.nface + 64.0 * len(g.face_vert) + 48.0 * len(g.vx)))
    return work, grid


def test_serve_resident_grid_reused(requests_):
    """Requests on one grid id: the first uploads the grid, the later ones
    (two at once, on different slots) map onto the resident copy without an
    upload, and every result equals the request served with a grid of its
    own.  Another particle field on the same resident grid (masses doubled)
    gives exactly twice the cell masses."""
    L = lib()
    p, g = requests_[0]
    ref, href, _, _ = serve([requests_[0]], slots=1)
    srv = L.map_server_create(L.map_server_config_default(precision=1, slots=2))
    try:
        outs = [np.full(g.ncell, -1.0) for _ in range(4)]
        hs = [np.zeros(p.n) for _ in range(3)]
        t0 = L.map_server_submit(srv, p.x, p.y, p.z, p.m, g, outs[0], h=hs[0], grid_id=7)
        assert L.map_server_wait(srv, t0).status == 0
        assert L.map_server_grid_stats(srv)[:3] == (1, 0, 1)
        t1 = L.map_server_submit(srv, p.x, p.y, p.z, p.m, g, outs[1], h=hs[1], grid_id=7)
        t2 = L.map_server_submit(srv, p.x, p.y, p.z, p.m, g, outs[2], h=hs[2], grid_id=7)
        t3 = L.map_server_submit(srv, p.x, p.y, p.z, 2.0 * p.m, g, outs[3], grid_id=7)
        assert all(L.map_server_wait(srv, t).status == 0 for t in (t1, t2, t3))
        uploads, hits, resident, nbytes = L.map_server_grid_stats(srv)
        assert (uploads, hits, resident) == (1, 3, 1) and nbytes > 0
    finally:
        L.map_server_destroy(srv)
    for j in range(3):
        assert np.array_equal(outs[j], ref[0]), j
        assert np.array_equal(hs[j], href[0]), j
    assert np.array_equal(outs[3], 2.0 * ref[0])


def test_serve_resident_grid_evicted_under_budget(requests_):
    """A budget with room for the larger of two requests and a quarter of the
    smaller one's grid: a request on the second grid id evicts the first
    (least recently used, unused) resident grid, and the first id uploads
    again afterwards; results are unchanged."""
    L = lib()
    ja, jb = sorted(range(2), key=lambda j: requests_[j][0].n)  # a: the smaller request
    (pa, ga), (pb, gb) = requests_[ja], requests_[jb]
    wa, gra = _est(pa, ga)
    wb, grb = _est(pb, gb)
    budget = wb + grb + gra // 4
    refa, _, _, _ = serve([requests_[ja]], slots=1)
    refb, _, _, _ = serve([requests_[jb]], slots=1)
    srv = L.map_server_create(L.map_server_config_default(precision=1, slots=1, hbm_budget=budget))
    try:
        oa, ob, oa2 = np.empty(ga.ncell), np.empty(gb.ncell), np.empty(ga.ncell)
        t = L.map_server_submit(srv, pa.x, pa.y, pa.z, pa.m, ga, oa, grid_id=1)
        assert L.map_server_wait(srv, t).status == 0
        assert L.map_server_grid_stats(srv)[:3] == (1, 0, 1)
        t = L.map_server_submit(srv, pb.x, pb.y, pb.z, pb.m, gb, ob, grid_id=2)
        assert L.map_server_wait(srv, t).status == 0
        assert L.map_server_grid_stats(srv)[:3] == (2, 0, 1)  # the first grid made room
        t = L.map_server_submit(srv, pa.x, pa.y, pa.z, pa.m, ga, oa2, grid_id=1)
        assert L.map_server_wait(srv, t).status == 0
        assert L.map_server_grid_stats(srv)[:2] == (3, 0)  # evicted, so uploaded again
    finally:
        L.map_server_destroy(srv)
    assert np.array_equal(oa, refa[0]) and np.array_equal(oa2, refa[0]) and np.array_equal(ob, refb[0])
