"""Pins of the oracle's interpolated Mandel-Agol terms (Sec. 2.2.3).

The interpolation has no closed form to compare with, so it is pinned to
what the method fixes:
  * at the grid nodes it returns the exact terms of the case table;
  * out of transit (z >= 1 + k) the terms are zero, as for the exact model;
  * its flux error against the exact model is of the size the paper prints
    for the default grid (n_k = 128, n_z = 256, a radius-ratio range of 0.02:
    ~4 ppm at most) and shrinks as the z grid is refined, while the k grid
    matters much less (the paper: even n_k = 8 stays near 8 ppm).
A wrong weight, a wrong cell index or a dropped Theta term fails one of these.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _max_flux_err(table, k_values, u1=0.4, u2=0.25, n_z=1500):
    worst = 0.0
    for k in k_values:
        for z in np.linspace(0.0, 1.0 + k, n_z, endpoint=False):
            worst = max(worst, abs(table.flux(k, z, u1, u2) - oracle.flux_quad(k, z, u1, u2)))
    return worst


def test_nodes_reproduce_exact_terms():
    T = oracle.MATable(0.08, 0.12, 5, 33)
    for i in range(T.n_k):
        k = 0.08 + i * 0.04 / 4
        for j in range(T.n_z):
            z = j * (1.0 + 0.12) / 32
            ref = np.array(oracle.ma_terms(k, z), dtype=float)
            if k > z:
                ref[1] += 2.0 / 3.0
            assert np.allclose(T.terms(k, z), ref, rtol=0, atol=1e-14), (k, z)


def test_out_of_transit_is_zero_and_k_is_clamped():
    T = oracle.MATable(0.08, 0.12, 9, 65)
    assert np.all(T.terms(0.1, 1.1) == 0.0)
    assert np.all(T.terms(0.1, 1.2) == 0.0)
    # k below / above the table reads the edge rows
    assert np.allclose(T.terms(0.05, 0.3), T.terms(0.08, 0.3), atol=0)
    assert np.allclose(T.terms(0.2, 0.3), T.terms(0.12, 0.3), atol=0)


def test_linear_between_nodes_along_z():
    T = oracle.MATable(0.1, 0.12, 3, 41)
    dz = 1.12 / 40
    a, b = T.terms(0.1, 10 * dz), T.terms(0.1, 11 * dz)
    assert np.allclose(T.terms(0.1, 10.25 * dz), 0.75 * a + 0.25 * b, rtol=0, atol=1e-15)


def test_error_matches_paper_scale_and_converges_in_z():
    ks = np.linspace(0.05, 0.07, 3)
    e_default = _max_flux_err(oracle.MATable(0.05, 0.07, 128, 256), ks)
    e_fine = _max_flux_err(oracle.MATable(0.05, 0.07, 128, 512), ks)
    e_coarse_k = _max_flux_err(oracle.MATable(0.05, 0.07, 8, 256), ks)
    # the paper prints ~4 ppm at its defaults (Sec. 2.2.3)
    assert 1e-6 < e_default < 1.5e-5
    # refining z helps (linear interpolation: between first and second order
    # at the contact points) ...
    assert e_fine < e_default / 2.5
    # ... while a much coarser k grid costs little
    assert e_coarse_k < 2.5 * e_default
