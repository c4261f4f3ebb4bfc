"""Pins of the oracle's analytic gradient against central finite differences
(h = 1e-6 relative) of the oracle's plain flux composition, and of the
overlap-integral derivatives against finite differences of the Mandel &
Agol terms.  A sign, index or dropped term in any chain-rule step fails one
of these."""
import math

import numpy as np
import pytest

import oracle

PI = math.pi


def _I(p, z):
    le, ld, ed = oracle.ma_terms(p, z)
    ldp = ld + (2.0 / 3.0 if p > z else 0.0)
    return np.array([PI * le, PI * ldp, PI * (le - ed)])


@pytest.mark.parametrize("p,z", [(0.1, 0.3), (0.1, 0.95), (0.1, 1.05), (0.3, 0.05), (0.3, 0.9), (0.7, 0.4),
                                 (0.05, 0.02), (0.2, 0.79), (0.15, 1.1), (1.3, 0.6)])
def test_overlap_derivs_vs_fd(p, z):
    d = oracle.overlap_derivs(p, z)
    h = 1e-7
    fp = (_I(p + h, z) - _I(p - h, z)) / (2 * h)
    fz = (_I(p, z + h) - _I(p, z - h)) / (2 * h)
    ref = np.array([fp[0], fz[0], fp[1], fz[1], fp[2], fz[2]])
    assert np.allclose(d, ref, rtol=1e-6, atol=1e-7), (d, ref)


def test_overlap_derivs_symmetry_and_zero():
    # z = 0: nothing changes to first order when the planet moves off centre
    d = oracle.overlap_derivs(0.1, 0.0)
    assert abs(d[1]) < 1e-15 and abs(d[3]) < 1e-15 and abs(d[5]) < 1e-15
    assert np.all(oracle.overlap_derivs(0.1, 1.2) == 0.0)
    # dI_1/dp for a planet fully inside is the circumference 2 pi p
    assert oracle.overlap_derivs(0.1, 0.5)[0] == pytest.approx(2 * PI * 0.1, rel=1e-15)


def _contact_distance(th, t):
    inc = oracle.inc_from_b(th[3], th[2], th[4], th[5])
    z, _ = oracle.z_ecc(t, th[0], th[1], th[2], inc, th[4], th[5])
    k = th[6]
    return min(abs(z - (1 + k)), abs(z - (1 - k)), abs(z - k), z)


THETAS = [
    [0.0, 3.0, 12.0, 0.3, 0.15, 1.1, 0.1, 0.4, 0.2],
    [0.7, 2.2, 8.0, 0.6, 0.05, 4.0, 0.15, 0.6, 0.1],
    [-0.3, 5.1, 20.0, 0.1, 0.3, 2.5, 0.08, 0.2, 0.5],
    [0.0, 3.0, 10.0, 0.2618, 0.0, 0.5 * PI, 0.1, 0.4, 0.2],
]


@pytest.mark.parametrize("th", THETAS)
def test_flux_grad_vs_central_differences(th):
    th = np.array(th)
    rng = np.random.default_rng(7)
    ts = th[0] + rng.uniform(-0.2, 0.2, 40)
    checked = 0
    for t in ts:
        if _contact_distance(th, t) < 1e-4:
            continue
        f, g = oracle.flux_grad(t, th)
        assert f == pytest.approx(oracle.flux_theta(t, th), abs=1e-14)
        fd = np.zeros(9)
        for i in range(9):
            h = 1e-6 * max(1.0, abs(th[i]))
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            fd[i] = (oracle.flux_theta(t, tp) - oracle.flux_theta(t, tm)) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-8), (t, g, fd)
        checked += f < 1.0
    assert checked >= 5


def test_flux_grad_supersampled_and_ssr():
    th = np.array(THETAS[0])
    t = np.linspace(-0.12, 0.12, 61)
    rng = np.random.default_rng(3)
    y = 1.0 - 0.005 * (np.abs(t) < 0.04) + rng.normal(0, 1e-4, t.size)
    wt = rng.uniform(0.5, 2.0, t.size)
    ths = np.stack([th, np.array(THETAS[1])])
    ths[1, 0] = 0.01
    ssr, grad = oracle.ssr_grad(t, ths, y, wt, n_ss=3, t_exp=0.02)
    for v in range(2):
        for i in range(9):
            h = 1e-6 * max(1.0, abs(ths[v, i]))
            tp, tm = ths[v].copy(), ths[v].copy()
            tp[i] += h
            tm[i] -= h
            sp = sum(wt[j] * (y[j] - oracle.flux_theta(t[j], tp, 3, 0.02)) ** 2 for j in range(t.size))
            sm = sum(wt[j] * (y[j] - oracle.flux_theta(t[j], tm, 3, 0.02)) ** 2 for j in range(t.size))
            assert grad[v, i] == pytest.approx((sp - sm) / (2 * h), rel=1e-4, abs=1e-9), (v, i)
        s0 = sum(wt[j] * (y[j] - oracle.flux_theta(t[j], ths[v], 3, 0.02)) ** 2 for j in range(t.size))
        assert ssr[v] == pytest.approx(s0, rel=1e-13)


def test_out_of_transit_gradient_is_zero():
    th = np.array(THETAS[0])
    f, g = oracle.flux_grad(1.0, th)
    assert f == 1.0 and np.all(g == 0.0)
