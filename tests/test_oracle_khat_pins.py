"""Pins of the oracle's k^2 / k_hat^2 passband scaling (Sec. 3.5).

Equal radius ratios reduce it to the per-passband model; for a uniform disk
the depth of a point fully inside the transit is k^2 exactly, so there the
scaling is exact; elsewhere its error against per-passband radius ratios
falls in proportion to the spread of the k_b (first order: ingress, egress
and limb darkening make the depth depend on k beyond k^2).
"""
import numpy as np

import oracle
from paper_1504_07433_gb300 import workloads as W


def _wl(n_t=600):
    wl = W.long_cadence(n_v=3, n_t=n_t, n_ss=1, cadence=0.005)
    return wl


def test_equal_k_is_the_per_band_model():
    wl = _wl()
    k = np.repeat(wl["k"][:, None], 4, axis=1)
    ld = np.repeat(wl["ld"], 4, axis=1)
    fk, _ = oracle.lc_ma_khat(wl["t"], wl["orbit"], k, ld)
    fe, _ = oracle.lc_ma(wl["t"], wl["orbit"], k, ld)
    assert np.max(np.abs(fk - fe)) < 1e-15


def test_uniform_disk_inside_is_exact():
    wl = _wl(2000)
    rng = np.random.default_rng(2)
    k = wl["k"][:, None] * rng.uniform(0.9, 1.1, (3, 4))
    ld = np.zeros((3, 4, 2))
    fk, _ = oracle.lc_ma_khat(wl["t"], wl["orbit"], k, ld)
    fe, _ = oracle.lc_ma(wl["t"], wl["orbit"], k, ld)
    kh = np.repeat(k.mean(axis=1, keepdims=True), 4, axis=1)
    fh, _ = oracle.lc_ma(wl["t"], wl["orbit"], kh, ld)
    # fully inside for the passband's own k and for k_hat
    inside = (np.isclose(fe, 1 - k[:, :, None] ** 2, rtol=0, atol=1e-12)
              & np.isclose(fh, 1 - kh[:, :, None] ** 2, rtol=0, atol=1e-12))
    assert inside.sum() > 100
    assert np.max(np.abs(fk - fe)[inside]) < 1e-14


def test_error_falls_with_the_spread():
    wl = _wl()
    rng = np.random.default_rng(5)
    shape = rng.uniform(-1, 1, (3, 4))
    ld = np.repeat(wl["ld"], 4, axis=1)
    errs = []
    for spread in (0.04, 0.02, 0.01):
        k = wl["k"][:, None] * (1 + spread * shape)
        fk, _ = oracle.lc_ma_khat(wl["t"], wl["orbit"], k, ld)
        fe, _ = oracle.lc_ma(wl["t"], wl["orbit"], k, ld)
        errs.append(np.max(np.abs(fk - fe)))
    assert errs[0] > 0
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.6
