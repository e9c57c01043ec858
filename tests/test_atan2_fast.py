"""The FP32 atan2 of the pair-integral kernel (octant reduction and the
library's own polynomial, coefficients read from its header) emulated in
numpy FP32 against FP64 arctan2: the error bound the kernel relies on."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def coefficients():
    src = open(os.path.join(ROOT, "paper_2404_17084_gb300", "csrc", "wedge.cuh")).read()
    body = src[src.index("float atan2_fast("):src.index("return copysignf")]
    first = re.search(r"float p = (-?[0-9.e-]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, u, (-?[0-9.e-]+)f\);", body)
    return [np.float32(first)] + [np.float32(c) for c in rest]


def atan2_emulated(y, x):
    f32 = np.float32
    y = y.astype(f32); x = x.astype(f32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(all="ignore"):
        t = np.where(mx > 0, (mn / mx).astype(f32), f32(0))
    u = (t * t).astype(f32)
    c = coefficients()
    p = np.full_like(u, c[0])
    for ci in c[1:]:
        p = (p * u + ci).astype(f32)   # two roundings: a looser bound than the device's fmaf
    r = (t * p).astype(f32)
    r = np.where(ay > ax, (f32(np.pi / 2) - r).astype(f32), r)
    r = np.where(np.signbit(x), (f32(np.pi) - r).astype(f32), r)
    return np.copysign(r, y)


def test_atan2_fast_error_bound():
    rng = np.random.default_rng(1)
    ang = rng.uniform(-np.pi, np.pi, 400000)
    rad = np.exp(rng.uniform(-20, 20, ang.size))
    y, x = (rad * np.sin(ang)).astype(np.float32), (rad * np.cos(ang)).astype(np.float32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(atan2_emulated(y, x).astype(np.float64) - ref)
    assert err.max() < 4e-7, err.max()


def test_atan2_fast_special_values():
    z = np.zeros(1, np.float32)
    assert atan2_emulated(z, z)[0] == 0.0
    assert np.isclose(atan2_emulated(z, -z)[0], np.pi)              # atan2(+0, -0) = pi
    assert np.isclose(atan2_emulated(-z, -z)[0], -np.pi)            # atan2(-0, -0) = -pi
    one = np.ones(1, np.float32)
    assert np.isclose(atan2_emulated(one, z)[0], np.pi / 2)
    assert np.isclose(atan2_emulated(-one, -one)[0], -3 * np.pi / 4)
