"""Host logic of bench.py that needs no GPU: the autotuner's table (trial
t * nshapes + v is item target t with launch shape v, labelled from the
shapes the library reports as launched) and the merge of per-snapshot error
summaries."""
import importlib.util
import os
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_autotune_table_layout_and_labels():
    b = _bench()
    L = types.SimpleNamespace(AUTOTUNE_ITEM_TARGETS=[16, 64, 256])
    shapes = [{"warps_per_cta": 4, "ctas_per_sm": 5, "registers": 95},
              {"warps_per_cta": 4, "ctas_per_sm": 4, "registers": 96},
              {"warps_per_cta": 2, "ctas_per_sm": 9, "registers": 95},
              {"warps_per_cta": 8, "ctas_per_sm": 2, "registers": 96}]
    ms = [100.0 + t * 10 + v for t in range(3) for v in range(4)]  # trial t * 4 + v
    tab = b.autotune_table(L, 2 * 4 + 3, ms, shapes)
    assert tab["chosen"] == {"item_target": 256, "shape": "8 warps/CTA, 2 CTAs/SM, 96 registers"}
    assert tab["shapes"][2] == "2 warps/CTA, 9 CTAs/SM, 95 registers"
    assert tab["ms"] == [[100.0 + t * 10 + v for v in range(4)] for t in range(3)]


def test_merge_errors_takes_worst_and_sums_cells():
    b = _bench()
    m = b.merge_errors([{"cells": 10, "max_rel": 1e-7, "p99_rel": 5e-8}, None,
                        {"cells": 30, "max_rel": 4e-7, "p99_rel": 2e-8}])
    assert m["cells"] == 40 and m["snapshots"] == 2
    assert m["max_rel"] == 4e-7 and m["p99_rel"] == 5e-8
