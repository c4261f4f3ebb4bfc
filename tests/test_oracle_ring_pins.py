"""Pins of the oracle's definition of the occulted flux (oracle.ring_alpha,
oracle.ring_flux): the ring integral that the Gimenez series converges to
(Sec. 2.1.1) and that measures the series' truncation error.

Referees, none of which shares code with it: scipy's adaptive quadrature of
the same ring integrand, the closed forms of a planet centred on the star
(z = 0) and wholly inside the disk, the lens-area closed form for the uniform
disk, and the Mandel-Agol case table (a separate computation in the oracle,
itself pinned against mpmath and 2-D brute force).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

PI = math.pi


def _arc(r, k, z):
    if r <= k - z:
        return 2 * PI
    if r >= z + k or r <= z - k:
        return 0.0
    return 2 * math.acos(min(1.0, max(-1.0, (r * r + z * z - k * k) / (2 * r * z))))


def _quad_alpha(n, k, z):
    pts = sorted(x for x in {abs(z - k), z + k} if 0 < x < 1)
    val, _ = integrate.quad(lambda r: (1 - r * r) ** (0.5 * n) * r * _arc(r, k, z), 0, 1, points=pts or None,
                            epsabs=1e-14, epsrel=1e-13, limit=500)
    return val / PI


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 8])
@pytest.mark.parametrize("k,z", [(0.1, 0.5), (0.1, 0.93), (0.1, 1.04), (0.2, 0.15), (0.05, 0.97), (0.5, 0.3),
                                 (0.3, 0.75), (1.2, 0.5), (0.1, 0.1)])
def test_ring_alpha_against_adaptive_quadrature(n, k, z):
    assert oracle.ring_alpha(n, k, z) == pytest.approx(_quad_alpha(n, k, z), rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("n", [0, 1, 2, 4, 7])
@pytest.mark.parametrize("k", [0.05, 0.2, 0.6])
def test_ring_alpha_centred_closed_form(n, k):
    # planet centred on the star: (1/pi) int_0^k mu^n 2 pi r dr = 2 (1 - (1 - k^2)^((n+2)/2)) / (n + 2)
    exact = 2.0 * (1.0 - (1.0 - k * k) ** (0.5 * (n + 2))) / (n + 2)
    assert oracle.ring_alpha(n, k, 0.0) == pytest.approx(exact, rel=1e-13)


def test_ring_alpha_uniform_disk_area():
    # n = 0: the covered area / pi -- k^2 inside, the lens area on the limb, 0 outside
    for k, z in [(0.1, 0.3), (0.1, 0.89), (0.25, 0.5)]:
        assert oracle.ring_alpha(0, k, z) == pytest.approx(k * k, rel=1e-13)
    for k, z in [(0.1, 0.95), (0.1, 1.05), (0.3, 0.9), (0.3, 1.2)]:
        k0 = math.acos((k * k + z * z - 1) / (2 * k * z))
        k1 = math.acos((1 - k * k + z * z) / (2 * z))
        lens = (k * k * k0 + k1 - 0.5 * math.sqrt(4 * z * z - (1 + z * z - k * k) ** 2)) / PI
        assert oracle.ring_alpha(0, k, z) == pytest.approx(lens, rel=1e-12)
    assert oracle.ring_alpha(3, 0.1, 1.1) == 0.0 and oracle.ring_alpha(0, 0.1, 1.2) == 0.0


def test_ring_flux_matches_case_table():
    # quadratic law: the definition against the Mandel-Agol case table
    for k in (0.05, 0.1, 0.2, 0.45):
        for z in np.linspace(0.0, 1.0 + k, 23)[:-1]:
            for u1, u2 in [(0.4, 0.2), (0.0, 0.0), (0.9, -0.3)]:
                f_def = oracle.ring_flux([u1 + 2 * u2, -u2], k, z)
                assert f_def == pytest.approx(oracle.flux_quad(k, z, u1, u2), abs=2e-13), (k, z, u1, u2)
    assert oracle.ring_flux([0.3, 0.1], 0.1, 1.1) == 1.0


def test_ring_flux_general_law_against_adaptive_quadrature():
    u = np.array([0.3, 0.2, -0.1, 0.05, 0.02])

    def intensity(r):
        mu = math.sqrt(max(0.0, 1 - r * r))
        return 1 - sum(u[n - 1] * (1 - mu ** n) for n in range(1, 6))

    for k, z in [(0.1, 0.6), (0.15, 0.9)]:
        pts = sorted(x for x in {abs(z - k), z + k} if 0 < x < 1)
        blocked, _ = integrate.quad(lambda r: intensity(r) * r * _arc(r, k, z), 0, 1, points=pts,
                                    epsabs=1e-14, epsrel=1e-13, limit=500)
        total, _ = integrate.quad(lambda r: intensity(r) * 2 * PI * r, 0, 1, epsabs=1e-14, epsrel=1e-13)
        assert oracle.ring_flux(u, k, z) == pytest.approx(1 - blocked / total, abs=1e-13)
