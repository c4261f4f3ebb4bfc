"""The polynomial behind the kernels' lens-angle atan2 (pt_device.cuh,
atan2_pos): its constants are the ones csrc/atan_poly.py fits, and the
kernel's evaluation order (Horner in FP32 with fused multiply-adds, then the
reflections pi/2 - t and pi - t) reproduces numpy's arctan2 over y >= 0 to
FP32 accuracy.  Host-side only: the constants are read from the source."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1504_07433_gb300", "csrc")


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "pt_device.cuh")).read()
    body = src[src.index("float atan2_pos("):]
    body = body[:body.index("float t = r * q;")]
    first = re.search(r"float q = ([-0-9.e+]+)f;", body).group(1)
    rest = re.findall(r"q = fmaf\(q, s, ([-0-9.e+]+)f\);", body)
    return np.array([float(first)] + [float(x) for x in rest], dtype=np.float32)   # r^16 ... r^0


def _fit_module():
    spec = importlib.util.spec_from_file_location("atan_poly", os.path.join(CSRC, "atan_poly.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _atan2_pos(y, x, c):
    """The kernel's steps in FP32 (the reciprocal taken correctly rounded)."""
    y = y.astype(np.float32)
    x = x.astype(np.float32)
    ax = np.abs(x)
    mx = np.maximum(y, ax)
    mn = np.minimum(y, ax)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(mx > 0, mn * (np.float32(1) / np.where(mx > 0, mx, 1)).astype(np.float32), 0).astype(np.float32)
    s = (r * r).astype(np.float32)
    q = np.full_like(s, c[0])
    for cj in c[1:]:
        q = (q.astype(np.float64) * s + cj).astype(np.float32)
    t = (r * q).astype(np.float32)
    t = np.where(y > ax, np.float32(np.pi / 2) - t, t).astype(np.float32)
    t = np.where(x < 0, np.float32(np.pi) - t, t).astype(np.float32)
    return t


def test_constants_match_the_fit():
    mod = _fit_module()
    c = mod.fit()
    assert np.array_equal(_kernel_coefficients(), c.astype(np.float32)[::-1])
    e64, e32 = mod.errors(c)
    assert e64 <= 2e-8 and e32 <= 1.5e-7


def test_atan2_pos_against_arctan2():
    c = _kernel_coefficients()
    rng = np.random.default_rng(3)
    ang = rng.uniform(0.0, np.pi, 200000)
    rad = 10.0 ** rng.uniform(-6, 1, ang.size)
    y = np.abs(rad * np.sin(ang))
    x = rad * np.cos(ang)
    # the lens geometry's exact cases: on the axes, both arguments zero
    y = np.concatenate([y, [0.0, 0.0, 1.0, 0.5, 0.0]])
    x = np.concatenate([x, [1.0, -1.0, 0.0, 0.5, 0.0]])
    y32, x32 = y.astype(np.float32), x.astype(np.float32)
    ref = np.arctan2(y32.astype(np.float64), x32.astype(np.float64))
    got = _atan2_pos(y32, x32, c).astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 4e-7              # ~1.5 ulp of pi
    small = ref < 0.1                                       # small angles keep relative accuracy
    assert np.max(np.abs(got[small] - ref[small]) / np.maximum(ref[small], 1e-30)) <= 1e-6
    assert got[-5:].tolist() == [0.0, np.float32(np.pi), np.float32(np.pi / 2), got[-2], 0.0]
    assert abs(got[-2] - np.pi / 4) <= 1e-7
