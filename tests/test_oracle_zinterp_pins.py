"""Pins of the oracle's Gimenez model interpolated in z (Sec. 3.3).

The interpolated model is pinned to what the method fixes: at the z nodes it
returns the series itself (alpha_n of Eq. gimenez); between nodes it is
linear; out of transit it is zero; its flux error against the series is of
the size the paper prints for its default grid (~25 ppm at most) and falls
as the grid is refined: first order overall (alpha_n has a kink at z = k)
and second order where alpha_n is smooth.
"""
import numpy as np

import oracle
from paper_1504_07433_gb300 import workloads as W

N, NJ = 8, 96


def _alpha(k, z):
    out = np.zeros(N + 1)
    oracle._lib().pto_gimenez_alpha(N, NJ, float(k), float(z), oracle._ptr(out))
    return out


def _nodes(k, n_in, n_edge):
    zb = max(1.0 - k, 0.0)
    return np.concatenate([np.arange(n_in) * zb / (n_in - 1), zb + np.arange(1, n_edge + 1) * (1 + k - zb) / n_edge])


def test_nodes_are_the_series():
    for k, n_in, n_edge in [(0.1, 7, 5), (0.3, 4, 9), (1.2, 2, 6)]:
        tab = oracle.gimenez_zi_table(N, NJ, k, n_in, n_edge)
        for i, z in enumerate(_nodes(k, n_in, n_edge)):
            assert np.allclose(tab[i], _alpha(k, z), rtol=0, atol=1e-15)
            if z < 1 + k:
                assert np.allclose(oracle.gimenez_zi_alpha(tab, k, z, n_in, n_edge), tab[i], rtol=0, atol=1e-14)


def test_linear_between_nodes_and_zero_outside():
    k, n_in, n_edge = 0.12, 9, 7
    tab = oracle.gimenez_zi_table(N, NJ, k, n_in, n_edge)
    zn = _nodes(k, n_in, n_edge)
    for i in (0, 4, n_in - 1, n_in + 2):
        z = 0.3 * zn[i] + 0.7 * zn[i + 1]
        assert np.allclose(oracle.gimenez_zi_alpha(tab, k, z, n_in, n_edge), 0.3 * tab[i] + 0.7 * tab[i + 1],
                           rtol=0, atol=1e-14)
    assert np.all(oracle.gimenez_zi_alpha(tab, k, 1 + k, n_in, n_edge) == 0.0)
    assert np.all(oracle.gimenez_zi_alpha(tab, k, 1.5, n_in, n_edge) == 0.0)


def _max_err(k, n_in, n_edge, z_lo=0.0, z_hi=None):
    z_hi = 1 + k if z_hi is None else z_hi
    u = np.zeros(N)
    u[:2] = W.quad_to_general(0.4, 0.25, 2)
    D = 1 - np.sum(np.arange(1, N + 1) * u / (np.arange(1, N + 1) + 2))
    C = np.concatenate([[1 - u.sum()], u]) / D
    tab = oracle.gimenez_zi_table(N, NJ, k, n_in, n_edge)
    return max(abs(np.dot(C, oracle.gimenez_zi_alpha(tab, k, z, n_in, n_edge) - _alpha(k, z)))
               for z in np.linspace(z_lo, z_hi, 1500, endpoint=False))


def test_error_scale_and_convergence():
    for k in (0.08, 0.15):
        e64 = _max_err(k, 64, 64)
        e128 = _max_err(k, 128, 128)
        assert 1e-6 < e64 < 3e-5          # the paper: ~25 ppm at its default grid
        # alpha_n has a kink at z = k (the planet's disk reaches the star's
        # centre), so refinement is first order overall ...
        assert e128 < e64 / 1.7
        # ... and second order where alpha_n is smooth
        s64 = _max_err(k, 64, 64, 0.3, 0.8)
        s128 = _max_err(k, 128, 128, 0.3, 0.8)
        assert s128 < s64 / 3.0           # (first order would give ~2)
