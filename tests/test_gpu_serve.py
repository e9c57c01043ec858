"""Serving loop (continuous batching): every request's result is the same
alone and in a mix of concurrent requests (bit-identical: each request runs
on its own context and stream and depends on its own inputs only), admission
holds the HBM budget, and a served FP64 result matches the oracle."""
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
