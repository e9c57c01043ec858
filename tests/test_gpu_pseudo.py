"""Pseudo-particles on the GPU (Section III-A/B, Eq. 5) and their smoothing
lengths (Section III-C/D) against the oracle's octree, walk and h solve."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import lib, oracle_h, gpu_map, rel_err

pytestmark = pytest.mark.gpu


def gpu_pseudo(p, h, src, theta=0.5, ngb_max=10000, **walk):
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=0, theta=theta, ngb_bruteforce_max=ngb_max))
    try:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        x, y, z, m, hh = t(p.x), t(p.y), t(p.z), t(p.m), t(h)
        cap = p.n
        ox, oy, oz, om, oh = (torch.empty(cap, dtype=torch.float64, device="cuda") for _ in range(5))
        kind = torch.empty(cap, dtype=torch.int32, device="cuda")
        ident = torch.empty(cap, dtype=torch.int64, device="cuda")
        n = L.build_pseudo_particles(ctx, L.make_particles(x, y, z, m, hh), src, L.make_particles(ox, oy, oz, om, oh),
                                     kind, ident, **walk)
        torch.cuda.synchronize()
        out = {k: v[:n].cpu().numpy() for k, v in dict(x=ox, y=oy, z=oz, m=om, h=oh, kind=kind, ident=ident).items()}
        return out
    finally:
        L.map_destroy(ctx)


def oracle_pseudo(p, h, src, theta=0.5, hfact=oracle.HFACT, **walk):
    t = oracle.Tree(p.x, p.y, p.z, p.m)
    acc, opened = t.walk(src, theta, **walk)
    # h of accepted nodes over the member set (brute force), Eq. (7)-(9)
    hn, _ = oracle.pseudo_h(t, acc, opened, h, hfact=hfact)
    return t, acc, opened, hn


@pytest.fixture(scope="module")
def cloud():
    p = synth.lognormal_particles(1 << 15, synth.BASE_SEED + 3)
    h, _ = oracle_h(p)
    a = int(np.argmin(h))  # densest particle: smallest h, lowest index on ties
    src = p.pos()[a]
    return p, h, src


def walk_cases(p, h, src):
    """Plain walk; r_part and r_leaf annuli around two sources; a region
    recorded around a large node of the plain walk."""
    t = oracle.Tree(p.x, p.y, p.z, p.m)
    acc0, _ = t.walk(src, 0.5)
    big = acc0[np.argmax(t.size[acc0])]
    second = p.pos()[int(np.argsort(h)[len(h) // 2])]
    return [dict(src=src), dict(src=np.stack([src, second]), r_part=0.03, r_leaf=0.08),
            dict(src=src, r_leaf=0.1, regions=np.array([[*t.com[big], t.size[big], 0.3 * t.size[big]]]))]


@pytest.mark.parametrize("ngb_max,case", [(10000, 0), (50, 0), (10000, 1), (50, 1), (10000, 2)])
def test_pseudo_particles_match_oracle(cloud, ngb_max, case):
    p, h, src0 = cloud
    walk = walk_cases(p, h, src0)[case]
    src = walk.pop("src")
    out = gpu_pseudo(p, h, src, ngb_max=ngb_max, **walk)
    t, acc, opened, h_acc = oracle_pseudo(p, h, src, **walk)
    if case:
        t0 = oracle.Tree(p.x, p.y, p.z, p.m)
        acc0, op0 = t0.walk(src0, 0.5)
        assert len(out["m"]) > len(acc0) + int(t0.count[op0].sum())  # the controls resolve more
    # the set of pseudo-particles: node labels and extracted particle indices
    gpu_nodes = np.sort(out["ident"][out["kind"] == 0])
    gpu_parts = np.sort(out["ident"][out["kind"] == 1])
    ref_nodes = np.sort(t.label[acc])
    ref_parts = np.sort(np.concatenate([t.particles_of(i) for i in opened])) if len(opened) else np.zeros(0, np.int64)
    assert np.array_equal(gpu_nodes, ref_nodes)
    assert np.array_equal(gpu_parts, ref_parts)
    # mass conservation and node properties
    assert abs(out["m"].sum() - p.m.sum()) < 1e-12 * p.m.sum()
    lab2acc = {int(l): k for k, l in enumerate(t.label[acc])}
    sel = np.nonzero(out["kind"] == 0)[0]
    k = np.array([lab2acc[int(l)] for l in out["ident"][sel]])
    com = t.com[acc][k]
    assert np.max(np.abs(out["x"][sel] - com[:, 0])) < 1e-13
    assert np.max(np.abs(out["m"][sel] / t.mass[acc][k] - 1)) < 1e-13
    # extracted particles keep their h; nodes get the solved h
    ps = np.nonzero(out["kind"] == 1)[0]
    assert np.array_equal(out["h"][ps], h[out["ident"][ps]])
    assert np.max(np.abs(out["h"][sel] / h_acc[k] - 1)) < 1e-9
    # depth-first order: pseudo-particles listed by Morton position, so the
    # walk output is a partition with no duplicates
    assert len(np.unique(out["ident"][sel])) == len(sel)


def test_pseudo_mapping_reduces_pairs(cloud):
    """Map the pseudo set onto its own Voronoi grid: parity with the oracle,
    and fewer pairs than the full set on its grid."""
    p, h, src = cloud
    out = gpu_pseudo(p, h, src)
    keep = synth.dedupe_sites(np.stack([out["x"], out["y"], out["z"]], 1))
    sites = np.stack([out["x"], out["y"], out["z"]], 1)[keep]
    g = synth.voronoi(sites)
    q = synth.Particles(out["x"].copy(), out["y"].copy(), out["z"].copy(), out["m"].copy())
    res = gpu_map(g, q, out["h"], 1)
    ref = oracle.map_cells(g, q.x, q.y, q.z, q.m, out["h"])
    assert np.array_equal(res["idx"], ref["idx"])
    assert rel_err(res["mass"], ref["mass"]).max() < 1e-5
    assert abs(res["mass"].sum() - ref["mass"].sum()) < 1e-7 * ref["mass"].sum()
    assert res["n_pairs"] < 0.5 * 100 * p.n
