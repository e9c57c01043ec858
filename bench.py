#!/usr/bin/env python
"""Benchmark: particle-cell pair integrals per second on GB300.

Workload (one step = the whole mapping path on one snapshot): the clumpy
cloud -- 2^20 equal-mass particles sampled from a log-normal density field
(Gaussian random field with P(k) ~ k^-4 on a 128^3 grid, sigma_ln_rho = 1.5)
in the unit cube, its clipped Voronoi grid (host-generated input, resident on
the device), and per step: smoothing-length solve, octree, pair-list build,
pair integrals and cell sums in the mixed FP32/FP64 build.

value = pair integrals per second (pairs of the snapshot / device time per
step), inputs resident in HBM.  e2e = the same metric with the particles and
the grid copied from pinned host memory and the cell masses read back inside
the timed region.  The FP64 build is timed on the same snapshot and reported
under "fp64".  cpu_baseline = the FP64 CPU oracle on a bounded sample of
cells of the same snapshot, on the host's cores.

--impl reference times that oracle alone (one sample of cells per step).
Multi-GPU (torchrun): every rank maps its own snapshot (weak scaling; no
collective on the data path); time = max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import platform
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_PARTICLES = 1 << 20
SIGMA = 1.5
OUTDIR = [os.path.join(ROOT, "bench_out")]  # clock samples and --dump output
WORKLOAD_BASE = ("clumpy cloud: 2^20 equal-mass particles, log-normal field (GRF P(k)~k^-4, 128^3, sigma_ln_rho=1.5), "
                 "clipped Voronoi grid")
WORKLOAD = WORKLOAD_BASE + ", mixed FP32/FP64"


# ----------------------------------------------------------------------------- helpers

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int):
    """One process per GPU: NCCL with GPUs, gloo without (host-logic tests)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def rank_seed(base: int, rank: int) -> int:
    """Each rank maps its own snapshot (weak scaling, no data-path collective)."""
    return base + 1000 * rank


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: the job's time."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def emit(line: dict, rank: int) -> bool:
    """Rank 0 prints the JSON line; the others print nothing."""
    if rank == 0:
        print(json.dumps(line), flush=True)
        return True
    return False


def make_snapshot(rank: int, n: int):
    import synth
    p = synth.lognormal_particles(n, rank_seed(synth.BASE_SEED + 2, rank), sigma=SIGMA)
    g = synth.voronoi(p.pos())
    return p, g


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(OUTDIR[0], f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# Algorithmic operation model of the pair-integral kernel (per counted unit):
# (FP32-pipe ops, MUFU ops), counted from the formulas as written, with an
# IEEE divide = 1 MUFU + 8, sqrt = 1 MUFU + 3, atan/atan2 = 1 MUFU + 18-22,
# asinh = 2 MUFU + 20.
OPS = {
    "face_tests": (6, 0),            # r0 = d'/h - n.y, side, |.|
    "edge_records": (11, 0),         # R0, along-edge a_a, a_b, side
    "edge_terms": (15, 2),           # c^2, s2, s1, clamps (split_edge)
    "inner_evals": (96, 6),          # one antiderivative: U, Omega, L, P2..P5
    "mid_intervals_mixed": (200, 14),  # 6-node Gauss-Legendre panel + setup + kappa dPhi
    "mid_split_mixed": (200, 14),    # the second piece of an interval split at the foot
    "mid_intervals_fp64": (240, 14),  # two closed-form evaluations + kappa dPhi
    "outer_intervals": (45, 2),      # -c0 dPhi (both branches of c0 evaluated)
}


# DRAM traffic of the mixed pair-integral kernel per pair:
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the 2^16
# clumpy case (385 MB for 7,813,809 pairs), scaled to a launch by its pair
# count (the kernel streams the same per-pair data at any size).  It belongs
# to the kernel as captured: set it to None when the kernel changes.
INTEGRAL_DRAM_BYTES_PER_PAIR = 49.3
# DRAM bytes per pair of one inverse-mapping sum (inv_apply, Morton-ordered
# gather): 449.6 MB read + written for 32,168,427 pairs in ncu on the 2^18
# clumpy snapshot, scaled by pair count like the figure above; None once the
# kernel changes.
INVERSE_DRAM_BYTES_PER_PAIR = 13.97


def counted_work(L, torch, precision, device, grids, dev, parts):
    """Work tally of the pair-integral kernel for the operation count: one
    untimed mapping call (map_particles_to_cells, or map_batch for a list of
    snapshots) of a context created with count_work = 1, whose kernel keeps
    the tally; the timed contexts run the kernel without it."""
    ctx = L.map_init(L.map_config_default(precision=precision, device=device, count_work=1))
    try:
        if isinstance(grids, list):
            handles = [L.map_grid_upload(ctx, L.grid_to_device(g, dev)) for g in grids]
            outs = [torch.empty(g.ncell, dtype=torch.float64, device=dev) for g in grids]
            L.map_batch(ctx, parts, handles, outs)
        else:
            handle = L.map_grid_upload(ctx, L.grid_to_device(grids, dev))
            out = torch.empty(grids.ncell, dtype=torch.float64, device=dev)
            L.map_particles_to_cells(ctx, parts, handle, out)
        torch.cuda.synchronize()
        st = L.map_get_stats(ctx)
        work, _ = L.map_get_work(ctx)
        return st.n_edge_terms, work
    finally:
        L.map_destroy(ctx)


def algorithmic_ops(work: dict, terms: int, mixed: bool):
    f = m = 0
    units = [("face_tests", work["face_tests"]), ("edge_records", work["edge_records"]),
             ("edge_terms", terms), ("inner_evals", work["inner_evals"]),
             ("outer_intervals", work["outer_intervals"]),
             ("mid_intervals_mixed" if mixed else "mid_intervals_fp64", work["mid_intervals"])]
    if mixed:
        units.append(("mid_split_mixed", work["mid_split"]))
    for key, cnt in units:
        f += OPS[key][0] * cnt
        m += OPS[key][1] * cnt
    return f, m


def alu_roofline(L, local, f32, mufu, launch_ms, sm_count, f_clk):
    """The integral kernel's roofline: its time bound is the slower of its
    FP32 ops at the measured FP32 FMA issue rate and its MUFU ops at the
    measured MUFU rate (map_device_peaks, this run); frac = bound / launch
    time, achieved = frac x the FP32 rate.  Falls back to the nominal rates,
    said so."""
    nominal_ops = sm_count * 128 * f_clk * 1e6       # FP32 lane-ops per second
    try:
        meas = L.map_device_peaks(local)
        peak_ops, peak_mufu = meas["ffma"], meas["mufu"]
        source = ("measured: FP32 FMA and MUFU issue microbenchmarks (map_device_peaks), "
                  f"nominal {nominal_ops / 1e12:.2f} = {sm_count} SMs x 128 lanes x {f_clk:.0f} MHz")
    except Exception as exc:  # the nominal rates, said so
        meas = None
        peak_ops, peak_mufu = nominal_ops, nominal_ops / 8.0
        source = f"nominal (microbenchmark failed: {exc}): {sm_count} SMs x 128 FP32 lanes x {f_clk:.0f} MHz"
    bound_s = max(f32 / peak_ops, mufu / peak_mufu)
    frac = bound_s / (launch_ms * 1e-3)
    return {"achieved": frac * peak_ops / 1e12, "peak": peak_ops / 1e12, "frac": frac, "peak_source": source,
            "measured_peaks_Tops": (None if meas is None else {k: round(v / 1e12, 3) for k, v in meas.items()})}


def oracle_errors(g, p, h, mass_gpu, ncells, seed):
    """Per-cell error of a GPU result against the FP64 oracle, run on the same
    particles and the GPU's own h, on a seeded random sample of cells (the
    floor of the relative error is 1e-12 of the largest reference mass)."""
    import oracle
    rng = np.random.default_rng(seed)
    cells = np.sort(rng.choice(g.ncell, min(ncells, g.ncell), replace=False)).astype(np.int64)
    r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells, nthreads=os.cpu_count() or 1)
    ref = r["mass"]
    scale = np.maximum(np.abs(ref), 1e-12 * np.abs(ref).max())
    e = np.abs(np.asarray(mass_gpu)[cells] - ref) / scale
    return {"cells": int(len(cells)), "max_rel": float(e.max()), "p99_rel": float(np.percentile(e, 99))}


def merge_errors(errs):
    """One error summary for several sampled snapshots."""
    errs = [e for e in errs if e]
    return {"cells": int(sum(e["cells"] for e in errs)), "max_rel": float(max(e["max_rel"] for e in errs)),
            "p99_rel": float(max(e["p99_rel"] for e in errs)), "snapshots": len(errs),
            "note": "per-cell mass against the FP64 oracle run on the same particles and the GPU's h; p99 is the "
                    "largest per-snapshot p99"}


def autotune_table(L, chosen, ms, shapes):
    """The autotuner's two-dimensional table: ms[target][shape]; the shapes
    as launched (warps per CTA, CTAs per SM, registers), read from the
    library."""
    ns = len(shapes)
    label = [f"{s['warps_per_cta']} warps/CTA, {s['ctas_per_sm']} CTAs/SM, {s['registers']} registers" for s in shapes]
    return {"chosen": {"item_target": L.AUTOTUNE_ITEM_TARGETS[chosen // ns], "shape": label[chosen % ns]},
            "shapes": label, "item_targets_per_warp": L.AUTOTUNE_ITEM_TARGETS,
            "ms": [[round(ms[t * ns + v], 3) for v in range(ns)] for t in range(len(L.AUTOTUNE_ITEM_TARGETS))]}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import paper_2404_17084_gb300 as L

    rank, world, local = dist_env()
    dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    p, g = make_snapshot(rank, args.n)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
    h = torch.empty_like(x)
    mass = torch.empty(g.ncell, dtype=torch.float64, device=dev)
    rho = torch.empty_like(mass)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def setup(precision):
        # the first warm-up step of the mixed build runs the autotuner (item size x launch shape)
        ctx = L.map_init(L.map_config_default(precision=precision, device=local, autotune=1))
        handle = L.map_grid_upload(ctx, L.grid_to_device(g, dev))
        return ctx, handle

    def step(ctx, handle):
        L.solve_h(ctx, L.make_particles(x, y, z, None, h))
        L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, h), handle, mass, rho)

    def timed(ctx, handle, steps, warmup, sampler=None):
        for _ in range(warmup):
            step(ctx, handle)
        barrier()
        _, l0 = L.map_get_work(ctx)
        integ_ms = []
        if sampler:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step(ctx, handle)
            integ_ms.append(L.map_get_timing(ctx)["integrals"])
        e1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        st = L.map_get_stats(ctx)
        work, l1 = L.map_get_work(ctx)
        phases = L.map_get_timing(ctx)
        return ms, st, work, (l1 - l0) // steps * steps, float(np.mean(integ_ms)), phases, clocks

    # ---- mixed build (headline)
    ctx, handle = setup(L.MAP_MIXED)
    sampler = ClockSampler(local)
    ms, st, work, launches, integ_ms, phases, clocks = timed(ctx, handle, args.steps, args.warmup, sampler)
    tune_chosen, tune_ms = L.map_get_autotune(ctx)
    tune_shapes = L.map_autotune_shapes(ctx)
    n_pairs = st.n_pairs
    mass_mixed = mass.cpu().numpy()
    h_mixed = h.cpu().numpy()
    inverse = inverse_run(L, torch, ctx, g, args.n, n_pairs, mass, m, dev)
    terms, work = counted_work(L, torch, L.MAP_MIXED, local, g, dev, L.make_particles(x, y, z, m, h))
    # ---- e2e through the public API with host buffers
    e2e = None if args.skip_e2e else e2e_run(L, torch, ctx, p, g, dev, args, barrier, world)
    L.map_destroy(ctx)
    # ---- the metric's latency half: a short serving pass at 50% and 90% of capacity
    import synth
    serving = None if args.skip_serve else serving_latency(L, local, rank_seed(synth.BASE_SEED + 5, rank) + 77)

    # ---- FP64 build (one timed step: GB300's FP64 rate makes it ~70x slower)
    fp64 = None
    table = None
    mass_fp64 = None
    h_fp64 = None
    mass_mixed_h64 = None
    if not args.skip_fp64:
        ctx64, handle64 = setup(L.MAP_FP64)
        ms64, st64, work64, _, integ64, phases64, _ = timed(ctx64, handle64, 1, 0)
        mass_fp64 = mass.cpu().numpy()
        h_fp64 = h.cpu().numpy()
        L.map_destroy(ctx64)
        # the mixed build on the FP64 build's h: integration error alone, every cell
        ctxm, handlem = setup(L.MAP_MIXED)
        L.map_particles_to_cells(ctxm, L.make_particles(x, y, z, m, h), handlem, mass, rho)
        torch.cuda.synchronize()
        mass_mixed_h64 = mass.cpu().numpy()
        L.map_destroy(ctxm)
        if args.dump:
            os.makedirs(OUTDIR[0], exist_ok=True)
            np.savez(os.path.join(OUTDIR[0], "cells.npz"), mass_mixed=mass_mixed, mass_fp64=mass_fp64,
                     mass_mixed_h64=mass_mixed_h64, h_mixed=h_mixed, h_fp64=h_fp64)
        fp64 = {"value": st64.n_pairs * world / (ms64 * 1e-3), "ms_per_step": ms64, "steps": 1, "warmup": 0,
                "integrals_ms": integ64, "phases_ms": {k: round(v, 3) for k, v in phases64.items()}}
        # the FP64 kernel against the measured FP64 FMA rate: the op model of
        # the FP64 form (closed-form middle pieces), every op on the FP64 pipe
        # (its divides, square roots and arctangents are FP64 sequences; the
        # model counts each as one MUFU op, so this bound is a lower one)
        try:
            h64 = torch.from_numpy(h_fp64).to(dev)  # kept alive through the call
            terms64, work64 = counted_work(L, torch, L.MAP_FP64, local, g, dev, L.make_particles(x, y, z, m, h64))
            f64_ops, f64_mufu = algorithmic_ops(work64, terms64, False)
            dfma = L.map_device_peaks(local)["dfma"]
            frac64 = (f64_ops + f64_mufu) / dfma / (integ64 * 1e-3)
            fp64["roofline"] = {"bound": "fp64", "kernel": "pair_integrals<double>", "achieved": frac64 * dfma / 1e12,
                                "peak": dfma / 1e12, "unit": "Tops/s (FP64 FMA issue)", "frac": frac64,
                                "ops": int(f64_ops + f64_mufu), "launch_ms": integ64,
                                "peak_source": "measured: FP64 FMA microbenchmark (map_device_peaks)"}
        except Exception as exc:  # reported, not fatal
            fp64["roofline"] = {"error": str(exc)}
        # the table variant (the paper's production route): its own timed
        # steps, then one mapping on the FP64 build's h for its error alone
        ctxt, handlet = setup(L.MAP_TABLE)
        mst, stt, _, _, integ_t, phases_t, _ = timed(ctxt, handlet, 3, 1)
        h.copy_(torch.from_numpy(h_fp64).to(dev))
        L.map_particles_to_cells(ctxt, L.make_particles(x, y, z, m, h), handlet, mass, rho)
        torch.cuda.synchronize()
        mass_table = mass.cpu().numpy()
        tot_table = L.map_get_stats(ctxt).total_mass
        L.map_destroy(ctxt)
        sc = np.maximum(np.abs(mass_fp64), 1e-12 * np.abs(mass_fp64).max())
        et = np.abs(mass_table - mass_fp64) / sc
        table = {"value": stt.n_pairs * world / (mst * 1e-3), "ms_per_step": mst, "steps": 3, "warmup": 1,
                 "integrals_ms": integ_t, "phases_ms": {k: round(v, 3) for k, v in phases_t.items()},
                 "table_n": int(L.map_config_default().table_n),
                 "vs_fp64_all_cells": {"max_rel": float(et.max()), "p99_rel": float(np.percentile(et, 99)),
                                       "p50_rel": float(np.percentile(et, 50))},
                 "total_mass_rel_vs_fp64": float(abs(tot_table - mass_fp64.sum()) / mass_fp64.sum()),
                 "note": "pyramid integrals interpolated trilinearly (texture unit) in a table of I(r0, R0, phi); "
                         "errors against the FP64 closed form on the same h"}

    f32, mufu = algorithmic_ops(work, terms, True)
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    f_clk = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = alu_roofline(L, local, f32, mufu, integ_ms, sm_count, f_clk)
    line = {
        "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
        "value": n_pairs * world / (ms * 1e-3),
        "unit": "pair integrals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_particles": args.n, "n_cells": g.ncell, "n_pairs": int(n_pairs),
                   "n_faces": g.nface, "l2": "inputs larger than L2 (grid and pair list several GB)",
                   "step": "solve_h + octree + pair list + pair integrals + cell sums"},
        "phases_ms": {k: round(v, 3) for k, v in phases.items()},
        "fp64": fp64,
        "table_variant": table,
        "roofline": {"bound": "alu", "kernel": "pair_integrals_mixed", "achieved": roof["achieved"],
                     "peak": roof["peak"], "unit": "Tops/s (FP32 issue slots)", "frac": roof["frac"],
                     "traffic": (None if INTEGRAL_DRAM_BYTES_PER_PAIR is None
                                 else INTEGRAL_DRAM_BYTES_PER_PAIR * n_pairs),
                     "ops_fp32": int(f32), "ops_mufu": int(mufu), "launch_ms": integ_ms,
                     "peak_source": roof["peak_source"], "measured_peaks_Tops": roof["measured_peaks_Tops"]},
        "e2e": e2e,
        "latency_ms": (None if serving is None else
                       {**serving["loads"]["0.9"]["latency_ms"], "at": "90% of the serving capacity",
                        "p50_at_50pct": serving["loads"]["0.5"]["latency_ms"]["p50"],
                        "p99_at_50pct": serving["loads"]["0.5"]["latency_ms"]["p99"]}),
        "serving": serving,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "autotune": autotune_table(L, tune_chosen, tune_ms, tune_shapes),
        "stats": {"edge_terms": int(terms), "total_mass": st.total_mass, **{k: int(v) for k, v in work.items()},
                  "counted_by": "one untimed call of a count_work context on the same particles and h"},
        "inverse_mapping": inverse,
        "secondary": {"edge_integrals_per_s": terms * world / (ms * 1e-3),
                      "note": "edge integrals K'_e with a nonzero term per second of the step; each stands for "
                              "the two vertex pyramids (wedges) that share the edge's foot"},
    }
    if mass_fp64 is not None:
        scale = np.maximum(np.abs(mass_fp64), 1e-12 * np.abs(mass_fp64).max())
        e = np.abs(mass_mixed_h64 - mass_fp64) / scale
        e2 = np.abs(mass_mixed - mass_fp64) / scale
        line["mixed_vs_fp64_all_cells"] = {
            "max_rel": float(e.max()), "p99_rel": float(np.percentile(e, 99)),
            "n_above_1e-5": int((e > 1e-5).sum()),
            "note": "every cell, both builds on the FP64 build's h (FP64 build: 2.5e-13 from the oracle)",
            "with_own_h": {"max_rel": float(e2.max()), "p99_rel": float(np.percentile(e2, 99))}}
    if rank == 0 and not args.no_cpu_baseline:
        base, acc = cpu_baseline(p, g, h_mixed, mass_mixed, h_fp64, mass_fp64, args)
        line["cpu_baseline"] = base
        line["accuracy_vs_oracle"] = acc
    if world > 1:
        torch.distributed.barrier()
    emit(line, rank)
    if world > 1:
        torch.distributed.destroy_process_group()


BATCH_WORKLOAD = ("batched uneven instances: {n} snapshots, particle counts log-uniform in [2^10, 2^18], half uniform, "
                  "half log-normal clumpy (sigma_ln_rho 1.0-2.0, 64^3 GRF), clipped Voronoi grids, one persistent "
                  "launch, mixed FP32/FP64")


def run_batch(args):
    """Batched workload: every step solves h for each snapshot and maps all of
    them with one map_batch call (one persistent integral launch through a
    CUDA graph; launch shape chosen by the autotuner in the first warm-up)."""
    import torch
    import paper_2404_17084_gb300 as L
    import synth

    rank, world, local = dist_env()
    dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = synth.batch_specs(args.nsnap, rank_seed(synth.BASE_SEED + 4, rank))
    t0 = time.perf_counter()
    snaps = []
    for spec in specs:
        p = synth.batch_particles(spec)
        snaps.append((p, synth.voronoi(p.pos())))
    gen_s = time.perf_counter() - t0
    ctx = L.map_init(L.map_config_default(precision=L.MAP_MIXED, device=local, autotune=1))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    handles, parts, hparts, keep, mass = [], [], [], [], []
    for p, g in snaps:
        handles.append(L.map_grid_upload(ctx, L.grid_to_device(g, dev)))
        x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
        h = torch.empty_like(x)
        keep.append((x, y, z, m, h))
        parts.append(L.make_particles(x, y, z, m, h))
        hparts.append(L.make_particles(x, y, z, None, h))
        mass.append(torch.empty(g.ncell, dtype=torch.float64, device=dev))
    totals = torch.empty(len(snaps), dtype=torch.float64, device=dev)

    def step():
        L.solve_h_batch(ctx, hparts)
        L.map_batch(ctx, parts, handles, mass, totals=totals)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    _, l0 = L.map_get_work(ctx)
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    integ = []
    g0 = L.map_batch_graph_stats(ctx)
    h0 = L.solve_h_batch_graph_stats(ctx)
    e0.record()
    for _ in range(args.steps):
        step()
        integ.append(L.map_get_timing(ctx)["integrals"])
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    st = L.map_get_stats(ctx)
    work, l1 = L.map_get_work(ctx)
    chosen, tune_ms = L.map_get_autotune(ctx)
    tune_shapes = L.map_autotune_shapes(ctx)
    g1 = L.map_batch_graph_stats(ctx)
    h1 = L.solve_h_batch_graph_stats(ctx)
    phases = L.map_get_timing(ctx)
    graph = {"captures": g1[0] - g0[0], "replays": g1[1] - g0[1], "fallbacks": g1[2] - g0[2],
             "solve_h_batch": {"captures": h1[0] - h0[0], "replays": h1[1] - h0[1]},
             "note": "calls of the timed steps that replayed their whole captured step as one graph launch: "
                     "map_batch (validation, octrees, pair lists, work items, integral launch, sums) and "
                     "solve_h_batch (validation, octrees, h solve)",
             "phases_ms_last_step": {k: round(v, 3) for k, v in phases.items()}}
    integ_ms = float(np.mean(integ))
    batch_mass = [mm.cpu().numpy() for mm in mass]
    # the same snapshots one call at a time (mapping only, h as solved above)
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    single_mass = []
    for j, (p, g) in enumerate(snaps):
        out = torch.empty(g.ncell, dtype=torch.float64, device=dev)
        L.map_particles_to_cells(ctx, parts[j], handles[j], out)
        single_mass.append(out)
    torch.cuda.synchronize()
    single_s = time.perf_counter() - s0
    same = all(np.array_equal(a, b.cpu().numpy()) for a, b in zip(batch_mass, single_mass))
    # error against the FP64 oracle: 8 snapshots spread over the sizes, 25 cells each
    pick = np.linspace(0, len(snaps) - 1, 8).astype(int)
    batch_err = merge_errors([oracle_errors(snaps[j][1], snaps[j][0], keep[j][4].cpu().numpy(), batch_mass[j], 25,
                                            100 + int(j)) for j in pick])
    # the batch's grids take most of the GPU's memory (edge records of 1.1e7
    # cells): release them before the counting context uploads its own copy
    L.map_destroy(ctx)
    del single_mass
    torch.cuda.empty_cache()
    terms, work = counted_work(L, torch, L.MAP_MIXED, local, [g for _, g in snaps], dev, parts)
    f32, mufu = algorithmic_ops(work, terms, True)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    f_clk = (clocks or {}).get("sm_max_mhz") or 2070.0
    roof = alu_roofline(L, local, f32, mufu, integ_ms, sm_count, f_clk)
    n_part = int(sum(p.n for p, _ in snaps))
    line = {
        "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
        "value": st.n_pairs * world / (ms * 1e-3),
        "unit": "pair integrals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(n=len(snaps)), "n_snapshots": len(snaps),
                   "n_particles": n_part, "n_pairs": int(st.n_pairs),
                   "l2": "inputs larger than L2 (grids and pair lists several GB)",
                   "step": "per snapshot solve_h, then one map_batch (octree + pair list per snapshot, one "
                           "persistent integral launch over all snapshots)"},
        "batch": {"integrals_ms": integ_ms, "integral_launch_pairs_per_s": st.n_pairs / (integ_ms * 1e-3),
                  "autotune": autotune_table(L, chosen, tune_ms, tune_shapes),
                  "one_call_per_snapshot_mapping_s": single_s, "batched_equals_single": bool(same),
                  "graph": graph,
                  "host_input_generation_s": gen_s},
        "accuracy_vs_oracle": batch_err,
        "roofline": {"bound": "alu", "kernel": "pair_integrals_mixed (batched launch)",
                     "achieved": roof["achieved"], "peak": roof["peak"], "unit": "Tops/s (FP32 issue slots)",
                     "frac": roof["frac"],
                     "traffic": (None if INTEGRAL_DRAM_BYTES_PER_PAIR is None
                                 else INTEGRAL_DRAM_BYTES_PER_PAIR * int(st.n_pairs)),
                     "ops_fp32": int(f32), "ops_mufu": int(mufu), "launch_ms": integ_ms,
                     "peak_source": roof["peak_source"], "measured_peaks_Tops": roof["measured_peaks_Tops"]},
        "e2e": None,
        "gpu_launches": int((l1 - l0) // max(args.steps, 1) * args.steps),
        "clocks": clocks,
        "stats": {"edge_terms": int(terms), "total_mass": st.total_mass,
                  **{k: int(v) for k, v in work.items()},
                  "counted_by": "one untimed map_batch of a count_work context on the same snapshots and h"},
    }
    if world > 1:
        torch.distributed.barrier()
    emit(line, rank)
    if world > 1:
        torch.distributed.destroy_process_group()


SERVE_WORKLOAD = ("serving loop: Poisson stream of {n} mapping requests ({pool} distinct, each on its own grid kept "
                  "resident by id), particle counts log-normal in log2 (median 2^15, sigma 1.5) clipped to [2^12, "
                  "2^{hi}], random uniform / log-normal clumpy fields, host inputs and outputs, {slots} slots "
                  "admitted by HBM, mixed FP32/FP64")


def serve_specs(k: int, seed: int, log2_hi: float = 21.0):
    rng = np.random.default_rng(seed)
    l2 = np.clip(rng.normal(15.0, 1.5, k), 12.0, log2_hi)
    kinds = rng.choice(["uniform", "clumpy"], size=k)
    sig = rng.uniform(1.0, 2.0, k)
    seeds = rng.integers(1, 2**31, k)
    return [(int(2.0 ** l2[j]), str(kinds[j]), float(sig[j]), int(seeds[j])) for j in range(k)]


class ServeSession:
    """A server over a pool of distinct requests (host arrays), each request
    on its own grid id so that its grid stays resident after its first use;
    Poisson streams of requests drawn from the pool, timed on the host clock
    from submission to results in host memory."""

    def __init__(self, L, local, pool, slots):
        self.L, self.pool = L, pool
        self.srv = L.map_server_create(L.map_server_config_default(device=local, precision=L.MAP_MIXED, slots=slots))
        self.outs = [np.empty(g.ncell) for _, g in pool]
        self.hs = [np.empty(p.n) for p, _ in pool]

    def submit(self, j, out, h=None):
        p, g = self.pool[j]
        return self.L.map_server_submit(self.srv, p.x, p.y, p.z, p.m, g, out, h=h, grid_id=j)

    def burst(self, idx, first=False):
        ts = [self.submit(j, self.outs[j], self.hs[j] if first else None) for j in idx]
        return [self.L.map_server_wait(self.srv, t) for t in ts]

    def capacity(self):
        """Requests per second with the whole pool queued at once, the better of two passes."""
        best = float("inf")
        for _ in range(2):
            c0 = time.perf_counter()
            self.burst(range(len(self.pool)))
            best = min(best, time.perf_counter() - c0)
        return len(self.pool) / best

    def stream(self, rate, nreq, seed, sampler=None):
        import threading
        rng = np.random.default_rng(seed)
        order = rng.integers(0, len(self.pool), nreq)
        gaps = rng.exponential(1.0 / rate, nreq)
        tickets = [None] * nreq
        bufs = [np.empty(self.pool[j][1].ncell) for j in order]

        def submitter():
            t_next = time.perf_counter()
            for i, j in enumerate(order):
                t_next += gaps[i]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = self.submit(int(j), bufs[i])

        if sampler:
            sampler.start()
        w0 = time.perf_counter()
        th = threading.Thread(target=submitter)
        th.start()
        res = []
        for i in range(nreq):
            while tickets[i] is None:
                time.sleep(0.0005)
            res.append(self.L.map_server_wait(self.srv, tickets[i]))
        wall = time.perf_counter() - w0
        th.join()
        clocks = sampler.stop() if sampler else None
        lat = np.array([r.latency_ms for r in res])
        que = np.array([r.queue_ms for r in res])
        return {"order": order, "results": res, "wall": wall, "clocks": clocks,
                "summary": {"arrival_rate_per_s": rate, "requests_per_s": nreq / wall,
                            "pairs_per_s": sum(r.n_pairs for r in res) / wall,
                            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                           "max": float(lat.max())},
                            "queue_ms": {"p50": float(np.percentile(que, 50)), "p99": float(np.percentile(que, 99))},
                            "all_ok": all(r.status == 0 for r in res),
                            "results_equal_to_first_pass": all(np.array_equal(bufs[i], self.outs[order[i]])
                                                               for i in range(nreq))}}

    def errors(self, k, seed):
        """Error of served results against the FP64 oracle (the served h): k pool entries, 40 cells each."""
        pick = np.argsort([p.n for p, _ in self.pool])[np.linspace(0, len(self.pool) - 1, k).astype(int)]
        return merge_errors([oracle_errors(self.pool[j][1], self.pool[j][0], self.hs[j], self.outs[j], 40,
                                           seed + int(j)) for j in pick])

    def close(self):
        grid = self.L.map_server_grid_stats(self.srv)
        self.L.map_server_destroy(self.srv)
        return {"uploads": grid[0], "hits": grid[1], "resident": grid[2], "resident_bytes": grid[3]}


def serve_pool(k, seed, log2_hi=21.0):
    import synth
    pool = []
    for spec in serve_specs(k, seed, log2_hi):
        p = synth.batch_particles(spec)
        pool.append((p, synth.voronoi(p.pos())))
    return pool


def serving_latency(L, local, seed, pool_size=16, nreq=64, slots=4):
    """The metric's latency half for the default line: a short serving pass
    (a pool of distinct requests of 2^12 to 2^18 particles on resident grids)
    at 50% and 90% of the measured capacity."""
    t0 = time.perf_counter()
    pool = serve_pool(pool_size, seed, 18.0)
    gen_s = time.perf_counter() - t0
    S = ServeSession(L, local, pool, slots)
    try:
        S.burst(range(len(pool)), first=True)  # uploads every grid once: resident from here on
        cap = S.capacity()
        loads = {}
        for load in (0.5, 0.9):
            loads[str(load)] = S.stream(load * cap, nreq, seed + int(load * 10))["summary"]
        err = S.errors(3, 300)
    finally:
        grid = S.close()
    return {"workload": SERVE_WORKLOAD.format(n=nreq, pool=pool_size, slots=slots, hi=18), "capacity_per_s": cap,
            "loads": loads, "accuracy_vs_oracle": err, "grids": grid, "host_input_generation_s": gen_s,
            "n_particles_p50": int(np.median([p.n for p, _ in pool]))}


def run_serve(args):
    """Serving workload: requests (host arrays) arrive as a Poisson stream and
    go through the library's serving loop (continuous batching over slots,
    admission by HBM, grids resident by id); throughput and p50/p99 latency
    are measured on the host clock from submission to results in host memory."""
    import torch
    import paper_2404_17084_gb300 as L
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    pool = serve_pool(args.pool, rank_seed(synth.BASE_SEED + 5, rank))
    gen_s = time.perf_counter() - t0
    S = ServeSession(L, local, pool, args.slots)
    try:
        for _ in range(max(1, args.warmup // 3)):
            S.burst(range(len(pool)), first=True)
        capacity = S.capacity()
        # the headline stream at 80% of capacity, then the latency at 50% and 90%
        rate = args.rate if args.rate > 0 else 0.8 * capacity
        main = S.stream(rate, args.requests, synth.BASE_SEED + 6, ClockSampler(local))
        sweep = {str(load): S.stream(load * capacity, args.requests, synth.BASE_SEED + 6 + int(load * 10))["summary"]
                 for load in (0.5, 0.9)}
        err = S.errors(4, 400)
    finally:
        grid = S.close()
    summ = main["summary"]
    order, results, wall = main["order"], main["results"], main["wall"]
    pairs = int(sum(r.n_pairs for r in results))
    line = {
        "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
        "value": pairs / wall,
        "unit": "pair integrals/s",
        "n_gpus": 1,
        "steps": args.requests,
        "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / args.requests,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD.format(n=args.requests, pool=len(pool), slots=args.slots, hi=21),
                   "arrival_rate_per_s": rate, "capacity_per_s": capacity,
                   "step": "one request: copy-in, solve_h, octree, pair list, pair integrals, copy-out (its grid "
                           "uploaded by its first request only)"},
        "latency_ms": summ["latency_ms"],
        "serving": {**summ, "n_particles_p50": int(np.median([pool[j][0].n for j in order])),
                    "host_input_generation_s": gen_s, "load_sweep": sweep, "grids": grid},
        "accuracy_vs_oracle": err,
        "e2e": {"value": pairs / wall, "unit": "pair integrals/s",
                "h2d_bytes_per_step": int(np.mean([pool[j][0].n * 32 for j in order])),
                "d2h_bytes_per_step": int(np.mean([pool[j][1].ncell * 8 for j in order])),
                "note": "grids resident by id: after a grid's first request, a request copies in its particles only"},
        "gpu_launches": None,
        "clocks": main["clocks"],
    }
    emit(line, rank)


def _step_timer(torch, step, steps, warmup):
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_uniform(args):
    """Plain Exact mapping, FP64: 4096 equal-mass particles uniform in the
    cube; every cell against the oracle, and mass conservation on interior
    particles (support inside the cube)."""
    import torch
    import paper_2404_17084_gb300 as L
    import oracle
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = synth.uniform_particles(4096, rank_seed(synth.BASE_SEED + 1, rank))
    g = synth.voronoi(p.pos())
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
    res = {}
    for prec, name in ((L.MAP_FP64, "fp64"), (L.MAP_MIXED, "mixed")):
        ctx = L.map_init(L.map_config_default(precision=prec, device=local))
        hd = L.map_grid_upload(ctx, L.grid_to_device(g, dev))
        h = torch.empty_like(x)
        mass = torch.empty(g.ncell, dtype=torch.float64, device=dev)

        def step():
            L.solve_h(ctx, L.make_particles(x, y, z, None, h))
            L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, h), hd, mass)

        ms = _step_timer(torch, step, args.steps, max(args.warmup, 3))
        st = L.map_get_stats(ctx)
        off, idx, frac = L.map_copy_pairs(ctx, g.ncell)
        res[name] = dict(ms=ms, n_pairs=int(st.n_pairs), mass=mass.cpu().numpy(), h=h.cpu().numpy(),
                         idx=idx.cpu().numpy(), frac=frac.cpu().numpy(), phases=L.map_get_timing(ctx))
        L.map_destroy(ctx)
    h64 = res["fp64"]["h"]
    t0 = time.perf_counter()
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h64)
    cpu_s = time.perf_counter() - t0
    scale = np.maximum(np.abs(ref["mass"]), 1e-12 * np.abs(ref["mass"]).max())
    e64 = np.abs(res["fp64"]["mass"] - ref["mass"]) / scale
    tot = np.zeros(p.n)
    np.add.at(tot, res["fp64"]["idx"], res["fp64"]["frac"])
    pos = p.pos()
    interior = np.all((pos >= 2 * h64[:, None]) & (pos <= 1 - 2 * h64[:, None]), axis=1)
    ref_m = oracle.map_cells(g, p.x, p.y, p.z, p.m, res["mixed"]["h"])
    em = np.abs(res["mixed"]["mass"] - ref_m["mass"]) / np.maximum(np.abs(ref_m["mass"]),
                                                                   1e-12 * np.abs(ref_m["mass"]).max())
    line = {
        "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
        "value": res["fp64"]["n_pairs"] / (res["fp64"]["ms"] * 1e-3), "unit": "pair integrals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": res["fp64"]["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "plain Exact mapping: 4096 equal-mass particles (m = 1/4096) uniform in the unit "
                               "cube, clipped Voronoi grid, h = 1.2 (m/rho)^(1/3), FP64", "n_cells": g.ncell,
                   "n_pairs": res["fp64"]["n_pairs"], "l2": "inputs smaller than L2 (a 4096-particle case)",
                   "step": "solve_h + octree + pair list + pair integrals + cell sums"},
        "mixed": {"value": res["mixed"]["n_pairs"] / (res["mixed"]["ms"] * 1e-3), "ms_per_step": res["mixed"]["ms"],
                  "all_cells_vs_oracle": {"max_rel": float(em.max()), "p99_rel": float(np.percentile(em, 99))}},
        "accuracy_vs_oracle": {"cells": g.ncell, "fp64_max_rel": float(e64.max()),
                               "fp64_p99_rel": float(np.percentile(e64, 99)),
                               "total_mass_rel": float(abs(res["fp64"]["mass"].sum() - ref["mass"].sum())
                                                       / ref["mass"].sum()),
                               "interior_particles": int(interior.sum()),
                               "interior_sum_f_max_dev": float(np.max(np.abs(tot[interior] - 1)))},
        "cpu_baseline": {"value": len(ref["idx"]) / cpu_s, "unit": "pair integrals/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": f"every cell ({g.ncell}), {cpu_s:.1f} s"},
        "phases_ms": {k: round(v, 3) for k, v in res["fp64"]["phases"].items()},
        "e2e": None, "gpu_launches": None,
    }
    emit(line, rank)


def run_inverse(args):
    """Inverse mapping (Eq. 4) on the clumpy-cloud snapshot: the mapping runs
    once (untimed), then a step is one call carrying random per-cell values
    (an ionic-fraction field) back to every particle with the mapping's pair
    integrals.  The first warm-up call builds the particle-major copy of the
    pair list.  e2e: cell values from pinned host memory in, particle values
    out, every step."""
    import torch
    import paper_2404_17084_gb300 as L
    import oracle

    rank, world, local = dist_env()
    dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, g = make_snapshot(rank, args.n)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
    h = torch.empty_like(x)
    mass = torch.empty(g.ncell, dtype=torch.float64, device=dev)
    ctx = L.map_init(L.map_config_default(precision=L.MAP_MIXED, device=local))
    handle = L.map_grid_upload(ctx, L.grid_to_device(g, dev))
    L.solve_h(ctx, L.make_particles(x, y, z, None, h))
    L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, h), handle, mass)
    n_pairs = L.map_get_stats(ctx).n_pairs
    rng = np.random.default_rng(rank_seed(12, rank))
    cv_host = [torch.from_numpy(rng.random(g.ncell)).pin_memory() for _ in range(2)]
    cv = [c.to(dev) for c in cv_host]
    out = torch.empty(p.n, dtype=torch.float64, device=dev)
    k = [0]

    def step():
        L.map_cells_to_particles(ctx, cv[k[0] & 1], out)
        k[0] += 1

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()  # builds the particle-major copy of the pair list
    torch.cuda.synchronize()
    first_ms = (time.perf_counter() - t0) * 1e3
    sampler = ClockSampler(local)
    warm = max(args.warmup, 3)
    w0 = time.perf_counter()
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    # a call takes about a millisecond: the clock sampler (5 samples a
    # second, after its own start-up) runs through two more seconds of
    # untimed calls before the timed ones, so that it sees the GPU under
    # this load
    soak = int(np.ceil(2.0 / max((time.perf_counter() - w0) / warm, 1e-5)))
    sampler.start()
    for _ in range(soak):
        step()
    torch.cuda.synchronize()
    _, l0 = L.map_get_work(ctx)
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    _, l1 = L.map_get_work(ctx)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    launches = l1 - l0
    # the mass-weighted totals of a call: sum_a m_a out_a = sum_i v_i M_i
    L.map_cells_to_particles(ctx, cv[0], out)
    ident = abs(float(torch.dot(m, out)) - float(torch.dot(cv[0], mass))) / float(torch.dot(cv[0], mass))
    # e2e: host cell values in, host particle values out
    out_host = torch.empty(p.n, dtype=torch.float64).pin_memory()
    e2e_steps = max(args.steps, 5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(e2e_steps):
        cv[0].copy_(cv_host[j & 1], non_blocking=True)
        L.map_cells_to_particles(ctx, cv[0], out)
        out_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    L.map_destroy(ctx)
    nbytes = 12 * n_pairs + 24 * p.n + 8 * g.ncell
    peak = load_peaks().get("hbm_gbs")
    gbs = nbytes / (ms * 1e-3) / 1e9
    line = {
        "metric": "pair terms/s of the inverse mapping (Eq. 4)",
        "value": n_pairs * world / (ms * 1e-3), "unit": "pair terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm + soak, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("mixed FP32/FP64", "inverse mapping of random per-cell values "
                                                "with the mixed build's pair integrals"),
                   "n_particles": p.n, "n_cells": g.ncell, "n_pairs": int(n_pairs),
                   "l2": "inputs larger than L2 (particle-major pair list %d MB)" % ((12 * n_pairs) >> 20),
                   "step": "one map_cells_to_particles call (the particle-major copy built before timing)"},
        "first_call_ms": first_ms,
        "roofline": {"bound": "hbm", "kernel": "inv_apply", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": (gbs / peak) if peak else None,
                     "traffic": INVERSE_DRAM_BYTES_PER_PAIR * n_pairs if INVERSE_DRAM_BYTES_PER_PAIR else None,
                     "algorithmic_bytes": int(nbytes),
                     "note": "per pair cell index + f_ai (12 B), per particle two offsets and the result (24 B), "
                             "per cell its value (8 B); peak = measured copy bandwidth"},
        "mass_identity_rel": ident,
        "e2e": {"value": n_pairs * world / (e2e_ms * 1e-3), "unit": "pair terms/s",
                "h2d_bytes_per_step": 8 * g.ncell, "d2h_bytes_per_step": 8 * p.n, "ms_per_step": e2e_ms,
                "steps": e2e_steps},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's sum on a pair list of the same shape (cell-major, the
        # same pairs per cell on average), bounded to about args.cpu_seconds
        npc = max(1, int(round(n_pairs / g.ncell)))
        ncell_s = max(1, min(g.ncell, int(2e6 // npc)))
        ns = ncell_s * npc
        off = np.arange(ncell_s + 1, dtype=np.int64) * npc
        idx = rng.integers(0, p.n, ns).astype(np.int32)
        fr = rng.random(ns)
        vals = rng.random(ncell_s)
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0) or reps == 0:
            oracle.inverse_map(off, idx, fr, vals, p.n)
            reps += 1
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": reps * ns / cpu_s, "unit": "pair terms/s", "cores": 1, "kind": "oracle",
                                "sample": f"{ns} pairs ({ncell_s} cells x {npc}, random particles) x {reps} calls "
                                          f"of the numpy sum, {cpu_s:.1f} s"}
    if world > 1:
        torch.distributed.barrier()
    emit(line, rank)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_tessellate(args):
    """Grid construction on the device (Section II-A) for the clumpy-cloud
    snapshot's 2^20 particle positions: merge sites closer than 1e-6 of the
    mean spacing, 5 Lloyd iterations, then the clipped Voronoi cells, left
    resident for the mapping.  A step is one map_grid_build (and the release
    of its grid).  e2e: the sites from pinned host memory in, the grid's
    arrays back to pinned host memory."""
    import torch
    import paper_2404_17084_gb300 as L
    import oracle
    import synth

    rank, world, local = dist_env()
    dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = synth.lognormal_particles(args.n, rank_seed(synth.BASE_SEED + 2, rank), sigma=SIGMA)
    n = p.n
    tol = 1e-6 * (1.0 / n) ** (1.0 / 3.0)
    hx, hy, hz = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (p.x, p.y, p.z))
    x, y, z = hx.to(dev), hy.to(dev), hz.to(dev)
    ctx = L.map_init(L.map_config_default(precision=L.MAP_MIXED, device=local))
    info = {}

    def step():
        hd, nk = L.map_grid_build(ctx, x, y, z, 5, tol)
        info["ncell"] = nk
        info["sizes"] = L.map_grid_sizes(ctx, hd)
        L.map_grid_release(ctx, hd)

    sampler = ClockSampler(local)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    _, l0 = L.map_get_work(ctx)
    if world > 1:
        torch.distributed.barrier()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    _, l1 = L.map_get_work(ctx)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)

    def final_only():
        hd, _ = L.map_grid_build(ctx, x, y, z, 0, tol)
        L.map_grid_release(ctx, hd)

    one_ms = _step_timer(torch, final_only, 3, 1)
    # e2e: host sites in, host grid out
    nc, nf, nl, nv = info["sizes"]
    host = {k: torch.empty(sz, dtype=dt).pin_memory() for k, sz, dt in (
        ("cfo", nc + 1, torch.int64), ("fvo", nf + 1, torch.int64), ("fv", nl, torch.int32),
        ("fpl", 4 * nf, torch.float64), ("vx", nv, torch.float64), ("vy", nv, torch.float64),
        ("vz", nv, torch.float64), ("site", 3 * nc, torch.float64))}
    e2e_steps = max(args.steps, 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(hx, non_blocking=True); y.copy_(hy, non_blocking=True); z.copy_(hz, non_blocking=True)
        hd, _ = L.map_grid_build(ctx, x, y, z, 5, tol)
        L._check(L._lib.map_grid_copy(ctx, hd, *[ctypes.c_void_p(host[k].data_ptr()) for k in
                                                  ("cfo", "fvo", "fv", "fpl", "vx", "vy", "vz", "site")],
                                      L._stream(None)), "map_grid_copy")
        torch.cuda.synchronize()
        L.map_grid_release(ctx, hd)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    d2h = sum(t.numel() * t.element_size() for t in host.values())
    L.map_destroy(ctx)
    line = {
        "metric": "Voronoi cells/s of the grid construction (merge + 5 Lloyd iterations + clipped cells)",
        "value": n * world / (ms * 1e-3), "unit": "sites/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"grid construction for the clumpy cloud: 2^{int(np.log2(n))} particle positions "
                               "(log-normal field, sigma_ln_rho = 1.5) as sites, merge within 1e-6 of the mean "
                               "spacing, 5 Lloyd iterations, cells clipped to the unit cube",
                   "n_sites": n, "n_cells": int(info["ncell"]), "n_faces": int(nf), "n_loop_entries": int(nl),
                   "step": "one map_grid_build (6 tessellations, 5 centroid passes, CSR packing, grid "
                           "preparation) + release"},
        "final_tessellation_ms": one_ms,
        "e2e": {"value": n * world / (e2e_ms * 1e-3), "unit": "sites/s", "h2d_bytes_per_step": 24 * n,
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "steps": e2e_steps},
        "gpu_launches": int((l1 - l0) // max(args.steps, 1) * args.steps), "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's brute-force cells on a sample of the sites (no Lloyd)
        pos = p.pos()
        rng = np.random.default_rng(5)
        t0, k = time.perf_counter(), 0
        sample = rng.choice(n, 400, replace=False)
        while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0) and k < len(sample):
            oracle.voronoi_cells_of(pos, [int(sample[k])])
            k += 1
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k / cpu_s, "unit": "sites/s", "cores": 1, "kind": "oracle",
                                "sample": f"{k} random cells of the {n} sites (no Lloyd step), {cpu_s:.1f} s"}
        t0 = time.perf_counter()
        synth.voronoi(pos)
        line["host_generator_s"] = {"seconds": time.perf_counter() - t0, "threads": os.cpu_count(),
                                    "note": "the package's host C++ tessellation of the same sites (no Lloyd)"}
    if world > 1:
        torch.distributed.barrier()
    emit(line, rank)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_pseudo(args):
    """Pseudo-particle path: 2^22 particles from the log-normal field, h from
    the GPU solve, the source at the densest particle; the octree walk turns
    nodes into pseudo-particles (theta = 0.5, leaf 16) with their own h; the
    pseudo set is mapped onto its own Voronoi grid, and the full set onto the
    same grid for the full-resolution comparison."""
    import torch
    import paper_2404_17084_gb300 as L
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n if args.n != N_PARTICLES else 1 << 22
    p = synth.lognormal_particles(n, rank_seed(synth.BASE_SEED + 3, rank), sigma=SIGMA)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
    h = torch.empty_like(x)
    ctx = L.map_init(L.map_config_default(precision=L.MAP_MIXED, device=local, autotune=1))
    L.solve_h(ctx, L.make_particles(x, y, z, None, h))
    torch.cuda.synchronize()
    hn = h.cpu().numpy()
    src = p.pos()[int(np.argmin(hn))]
    cap = n
    ox, oy, oz, om, oh = (torch.empty(cap, dtype=torch.float64, device=dev) for _ in range(5))
    full = L.make_particles(x, y, z, m, h)
    outp = L.make_particles(ox, oy, oz, om, oh)
    npseudo = [0]

    def build():
        npseudo[0] = L.build_pseudo_particles(ctx, full, src, outp)

    build_ms = _step_timer(torch, build, args.steps, max(args.warmup, 3))
    k = npseudo[0]
    pos = np.stack([ox[:k].cpu().numpy(), oy[:k].cpu().numpy(), oz[:k].cpu().numpy()], 1)
    keep = synth.dedupe_sites(pos)
    g = synth.voronoi(pos[keep])
    hd = L.map_grid_upload(ctx, L.grid_to_device(g, dev))
    mass_p = torch.empty(g.ncell, dtype=torch.float64, device=dev)
    mass_f = torch.empty_like(mass_p)
    pseudo = L.make_particles(ox[:k], oy[:k], oz[:k], om[:k], oh[:k])

    def map_pseudo():
        L.map_particles_to_cells(ctx, pseudo, hd, mass_p)

    map_ms = _step_timer(torch, map_pseudo, args.steps, max(args.warmup, 3))
    st_p = L.map_get_stats(ctx)

    def map_full():
        L.map_particles_to_cells(ctx, full, hd, mass_f)

    full_ms = _step_timer(torch, map_full, 1, 1)
    st_f = L.map_get_stats(ctx)
    full_phases = L.map_get_timing(ctx)
    mp, mf = mass_p.cpu().numpy(), mass_f.cpu().numpy()
    pq = synth.Particles(ox[:k].cpu().numpy(), oy[:k].cpu().numpy(), oz[:k].cpu().numpy(), om[:k].cpu().numpy())
    pseudo_err = oracle_errors(g, pq, oh[:k].cpu().numpy(), mp, 300, 21)
    rel = np.abs(mp - mf) / np.maximum(mf, 1e-12 * mf.max())
    step_ms = build_ms + map_ms
    mass_plain = float(abs(om[:k].sum().item() - m.sum().item()) / m.sum().item())
    # the walk controls of Section III-B around the same source: particles
    # within r_part, at least leaves out to r_leaf
    kind = torch.empty(cap, dtype=torch.int32, device=dev)
    controls = {}
    for r_part, r_leaf in ((0.02, 0.05), (0.05, 0.1)):
        def build_c():
            npseudo[0] = L.build_pseudo_particles(ctx, full, src, outp, kind=kind, r_part=r_part, r_leaf=r_leaf)
        ms_c = _step_timer(torch, build_c, args.steps, max(args.warmup, 3))
        kc = npseudo[0]
        controls[f"r_part={r_part},r_leaf={r_leaf}"] = {
            "build_ms": ms_c, "n_pseudo": kc, "particles": int((kind[:kc] == 1).sum().item()),
            "mass_rel": float(abs(om[:kc].sum().item() - m.sum().item()) / m.sum().item())}
    line = {
        "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
        "value": st_p.n_pairs / (step_ms * 1e-3), "unit": "pair integrals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"pseudo-particle path: 2^{int(np.log2(n))} particles, log-normal field "
                               "(sigma_ln_rho = 1.5), octree leaf 16, source at the densest particle, theta = 0.5, "
                               "pseudo h on ~58 neighbours, pseudo set mapped onto its own Voronoi grid, mixed",
                   "n_particles": n, "n_pseudo": k, "n_cells": g.ncell, "n_pairs_pseudo": int(st_p.n_pairs),
                   "step": "build_pseudo_particles (walk + pseudo h) + mapping of the pseudo set"},
        "pseudo": {"build_ms": build_ms, "map_ms": map_ms,
                   "reduction": {"particles": n / k, "pairs_full_on_same_grid": int(st_f.n_pairs),
                                 "pairs_ratio": st_f.n_pairs / max(st_p.n_pairs, 1)},
                   "full_resolution_map_ms": full_ms,
                   "full_resolution_phases_ms": {k: round(v, 3) for k, v in full_phases.items()},
                   "vs_full_resolution_per_cell_rel": {"p50": float(np.percentile(rel, 50)),
                                                        "p90": float(np.percentile(rel, 90)),
                                                        "p99": float(np.percentile(rel, 99))},
                   "mass_pseudo_vs_full": mass_plain,
                   "walk_controls": controls},
        "accuracy_vs_oracle": pseudo_err,
        "e2e": None, "gpu_launches": None,
    }
    L.map_destroy(ctx)
    emit(line, rank)


def inverse_run(L, torch, ctx, g, n, n_pairs, mass, m, dev, reps=20):
    """Eq. 4 on the last step's mapping: random per-cell values carried back to
    the particles.  The first call also builds the particle-major copy of the
    pair list; later calls only sum.  Algorithmic bytes of a sum: per pair its
    cell index and f_ai (12 B), per particle two offsets and the result
    (24 B), per cell its value (8 B); FP64 work: one FMA per pair."""
    rng = np.random.default_rng(12)
    vals = [torch.as_tensor(rng.random(g.ncell), dtype=torch.float64, device=dev) for _ in range(2)]
    out = torch.empty(n, dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    L.map_cells_to_particles(ctx, vals[0], out)
    ev[1].record()
    for k in range(reps):
        L.map_cells_to_particles(ctx, vals[(k + 1) & 1], out)
    ev[2].record()
    torch.cuda.synchronize()
    first_ms = ev[0].elapsed_time(ev[1])
    apply_ms = ev[1].elapsed_time(ev[2]) / reps
    # reps is even: out holds vals[0] carried back
    lhs = float(torch.dot(m, out))
    rhs = float(torch.dot(vals[0], mass))
    nbytes = 12 * n_pairs + 24 * n + 8 * g.ncell
    peak = load_peaks().get("hbm_gbs")
    gbs = nbytes / (apply_ms * 1e-3) / 1e9
    return {"first_call_ms": first_ms, "apply_ms": apply_ms, "index_build_ms": first_ms - apply_ms,
            "pairs_per_s": n_pairs / (apply_ms * 1e-3), "bytes_per_apply": int(nbytes), "achieved_GBps": gbs,
            "frac_of_hbm": (gbs / peak) if peak else None,
            "fp64_fma_G_per_s": n_pairs / (apply_ms * 1e-3) / 1e9,
            "mass_identity_rel": abs(lhs - rhs) / abs(rhs),
            "note": "sum_a m_a out_a vs sum_i v_i M_i on the same mapping; apply = mean of %d calls, inputs "
                    "(index %d MB) larger than L2" % (reps, (12 * n_pairs) >> 20)}


def e2e_run(L, torch, ctx, p, g, dev, args, barrier, world):
    """Same metric through the public API: pinned host inputs copied in (the
    particles by torch, the grid by map_grid_upload itself), the grid
    prepared, solve_h + mapping, cell masses read back.  The h solve needs
    only the particles, so it runs on a second context and stream while the
    grid is copied in and prepared (calls of one context run in order).  Both
    streams are created ones: work on the legacy default stream would wait
    for the side stream's h solve instead of running beside it."""
    pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hp = [pin(a, torch.float64) for a in (p.x, p.y, p.z, p.m)]
    hg = dict(cell_face_off=pin(g.cell_face_off, torch.int64), face_vert_off=pin(g.face_vert_off, torch.int64),
              face_vert=pin(g.face_vert, torch.int32), face_plane=pin(g.face_plane, torch.float64),
              vx=pin(g.vx, torch.float64), vy=pin(g.vy, torch.float64), vz=pin(g.vz, torch.float64),
              site=pin(g.site, torch.float64))
    out_host = torch.empty(g.ncell, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hp) + sum(t.numel() * t.element_size() for t in hg.values())
    d2h = out_host.numel() * out_host.element_size()

    ctx_h = L.map_init(L.map_config_default(precision=L.MAP_MIXED, device=dev.index or 0))
    main = torch.cuda.Stream(device=dev)
    side = torch.cuda.Stream(device=dev)

    def one():
        with torch.cuda.stream(main):
            dp = [t.to(dev, non_blocking=True) for t in hp]
            hh = torch.empty_like(dp[0])
            side.wait_stream(main)
            with torch.cuda.stream(side):
                L.solve_h(ctx_h, L.make_particles(dp[0], dp[1], dp[2], None, hh), stream=side)
            handle = L.map_grid_upload(ctx, hg, stream=main)
            main.wait_stream(side)
            mass = torch.empty(g.ncell, dtype=torch.float64, device=dev)
            L.map_particles_to_cells(ctx, L.make_particles(dp[0], dp[1], dp[2], dp[3], hh), handle, mass,
                                     stream=main)
            out_host.copy_(mass, non_blocking=True)
        torch.cuda.synchronize()
        L.map_grid_release(ctx, handle)
        return L.map_get_stats(ctx).n_pairs

    try:
        steps = max(1, args.steps // 2)
        one()
        barrier()
        t0 = time.perf_counter()
        npairs = 0
        step_ms = []
        for _ in range(steps):
            ts = time.perf_counter()
            npairs = one()
            step_ms.append((time.perf_counter() - ts) * 1e3)
        barrier()
        sec = (time.perf_counter() - t0) / steps
    finally:
        L.map_destroy(ctx_h)
    return {"value": npairs * world / sec, "unit": "pair integrals/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": sec * 1e3, "steps": steps,
            "ms_each_step": [round(v, 2) for v in step_ms],
            "note": "solve_h on a second context and stream, beside the grid upload"}


def oracle_sample(p, g, h, ncells: int, seed: int = 7):
    """Time the oracle on a seeded random sample of ncells cells."""
    import oracle
    rng = np.random.default_rng(seed)
    cells = np.sort(rng.permutation(g.ncell)[:min(ncells, g.ncell)])
    ncores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells, nthreads=ncores)
    dt = time.perf_counter() - t0
    return cells, r, dt, ncores


def cpu_baseline(p, g, h, mass_mixed, h_fp64, mass_fp64, args):
    """Oracle timing on a bounded sample of cells, and the per-cell error of
    each GPU build against the oracle run on that build's own h."""
    import oracle
    # a seeded random 1% of the cells, at least 2000
    cells, r, dt, ncores = oracle_sample(p, g, h, max(2000, g.ncell // 100))
    npairs = len(r["idx"])

    def err(mass_gpu, ref):
        scale = np.maximum(np.abs(ref), 1e-12 * np.abs(ref).max())
        return np.abs(mass_gpu[cells] - ref) / scale

    err_mixed = err(mass_mixed, r["mass"])
    acc = {"cells": int(len(cells)), "mixed_max_rel": float(err_mixed.max()),
           "mixed_p99_rel": float(np.percentile(err_mixed, 99))}
    if mass_fp64 is not None:
        # the FP64 build on the first 2000 of those cells (its own h)
        c64 = cells[:2000]
        r64 = oracle.map_cells(g, p.x, p.y, p.z, p.m, h_fp64, cells=c64, nthreads=ncores)
        scale = np.maximum(np.abs(r64["mass"]), 1e-12 * np.abs(r64["mass"]).max())
        err_fp64 = np.abs(mass_fp64[c64] - r64["mass"]) / scale
        acc.update(fp64_cells=int(len(c64)), fp64_max_rel=float(err_fp64.max()),
                   fp64_p99_rel=float(np.percentile(err_fp64, 99)))
    acc["note"] = "per-cell mass vs the FP64 oracle on the same cells, each build with its own GPU-solved h"
    # the same oracle on one core, on a sixteenth of the sample
    c1 = cells[:max(4, len(cells) // 16)]
    t1 = time.perf_counter()
    r1 = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=c1, nthreads=1)
    dt1 = time.perf_counter() - t1
    base = {"value": npairs / dt, "unit": "pair integrals/s", "cores": ncores, "kind": "oracle",
            "sample": f"{len(cells)} random cells (max(2000, 1% of the cells)) of the same snapshot ({npairs} pairs; "
                      f"pair list by brute force over all {p.n} particles + adaptive-quadrature pair integrals), "
                      f"{dt:.1f} s",
            "value_1core": len(r1["idx"]) / dt1,
            "sample_1core": f"the first {len(c1)} of those cells ({len(r1['idx'])} pairs) on one core, {dt1:.1f} s",
            "cpu": platform.processor() or platform.machine()}
    return base, acc


# ----------------------------------------------------------------------------- reference arm (oracle)

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    p, g = make_snapshot(0, args.n)
    tree = oracle.Tree(p.x, p.y, p.z, p.m)
    h, _ = oracle.solve_h(p.x, p.y, p.z, oracle.particle_h_guess(tree))
    rng = np.random.default_rng(11)
    ncores = os.cpu_count() or 1
    per_step = args.ref_cells
    total_pairs = 0
    for _ in range(args.warmup):
        cells = np.sort(rng.choice(g.ncell, per_step, replace=False))
        oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells, nthreads=ncores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cells = np.sort(rng.choice(g.ncell, per_step, replace=False))
        r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells, nthreads=ncores)
        total_pairs += len(r["idx"])
    dt = time.perf_counter() - t0
    v = total_pairs / dt
    line = {"impl": "reference", "metric": "particle-cell pair integrals/sec at 1 GB300 (mixed vs FP64 form) + p50/p99 latency",
            "value": v, "unit": "pair integrals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_BASE + ", FP64 CPU oracle (brute-force pair list + adaptive "
                                   "quadrature of the pair integrals) on a random sample of cells per step",
                       "n_particles": args.n, "n_cells": g.ncell,
                       "sample_per_step": f"{per_step} random cells (pair list + pair integrals)"},
            "cpu_baseline": {"value": v, "unit": "pair integrals/s", "cores": ncores, "kind": "oracle",
                             "sample": f"{per_step} random cells per step"},
            "e2e": {"value": v, "unit": "pair integrals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_PARTICLES)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-cells", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-serve", action="store_true", help="no serving pass (latency) in the default line")
    ap.add_argument("--dump", action="store_true", help="save per-cell results to <outdir>/cells.npz")
    ap.add_argument("--outdir", default=os.path.join(ROOT, "bench_out"),
                    help="folder for the clock samples and --dump output")
    ap.add_argument("--workload", default="clumpy",
                    choices=["clumpy", "batch", "serve", "uniform", "pseudo", "inverse", "tessellate"],
                    help="clumpy: one 2^20 snapshot (default); batch: uneven snapshots in one launch; "
                         "serve: Poisson stream of requests through the serving loop; uniform: 4096 uniform "
                         "particles, FP64; pseudo: 2^22 particles reduced to pseudo-particles; inverse: "
                         "per-cell values carried back to the 2^20 snapshot's particles (Eq. 4); tessellate: "
                         "the grid built on the device from the 2^20 snapshot's positions")
    ap.add_argument("--pool", type=int, default=32, help="distinct requests of the serve workload")
    ap.add_argument("--requests", type=int, default=160, help="requests submitted in the serve workload")
    ap.add_argument("--rate", type=float, default=0.0, help="serve arrival rate (req/s); 0 = 80%% of capacity")
    ap.add_argument("--slots", type=int, default=4, help="serving slots")
    ap.add_argument("--nsnap", type=int, default=256, help="snapshots of the batch workload")
    args = ap.parse_args()
    OUTDIR[0] = args.outdir
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "uniform":
        run_uniform(args)
    elif args.workload == "pseudo":
        run_pseudo(args)
    elif args.workload == "inverse":
        run_inverse(args)
    elif args.workload == "tessellate":
        run_tessellate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
