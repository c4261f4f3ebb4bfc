"""Coefficients of the polynomial behind atan2_pos in pt_device.cuh.

atan(r) = r P(r^2) on [0, 1], P of degree 8, fitted to atan(r)/r by
Lawson's iteratively reweighted least squares (weights multiplied by the
square root of the relative residual each pass, which drives the weighted
least-squares solution towards the minimax one) on Chebyshev nodes.

Run as a script it prints the coefficients (highest degree first, the order
of the Horner evaluation in the kernel) and the maximum absolute error of the
fit in FP64 and of the FP32 evaluation with fused multiply-adds.
"""
import numpy as np

DEGREE = 8


def fit(degree=DEGREE, n_nodes=6000, passes=500):
    x = 0.5 + 0.5 * np.cos(np.pi * (np.arange(n_nodes) + 0.5) / n_nodes)
    s = x * x
    A = np.stack([s ** j for j in range(degree + 1)], axis=1)
    f = np.arctan(x) / x
    w = np.ones(n_nodes)
    c = None
    for _ in range(passes):
        c, *_ = np.linalg.lstsq(A * w[:, None], f * w, rcond=None)
        r = np.abs(A @ c - f)
        w = w * np.sqrt(r / r.max() + 1e-4)
        w /= w.max()
    return c


def errors(c):
    x = np.linspace(0.0, 1.0, 400001)
    e64 = np.abs(np.polyval(c[::-1], x * x) * x - np.arctan(x)).max()
    c32 = c.astype(np.float32)
    x32 = x.astype(np.float32)
    s32 = x32 * x32
    q = np.full_like(s32, c32[-1])
    for j in range(len(c32) - 2, -1, -1):
        q = (q.astype(np.float64) * s32 + c32[j]).astype(np.float32)   # one rounding per step, as fmaf
    e32 = np.abs((q * x32).astype(np.float64) - np.arctan(x)).max()
    return e64, e32


if __name__ == "__main__":
    c = fit()
    e64, e32 = errors(c)
    print("coefficients, r^16 ... r^0:", ", ".join("%.9ef" % v for v in c.astype(np.float32)[::-1]))
    print("max |error|: FP64 %.2e, FP32 evaluation %.2e" % (e64, e32))
