"""Pins of the FP64 oracle against things other than itself.

Every check here compares the oracle with an independent referee: mpmath's
elliptic and hypergeometric functions, a 1-D ring-integral definition of the
occulted flux, brute-force 2-D integration, closed forms, and invariants of
the geometry.  A dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate

import oracle

PI = math.pi


# ------------------------------------------------------------------ referees
def intensity(r, u1, u2):
    mu = math.sqrt(max(0.0, 1.0 - r * r))
    return 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2


def arc_angle(r, p, z):
    """Angle subtended at the star centre by the part of the ring of radius r
    that lies inside the planet disk (radius p, centre at distance z)."""
    if r <= p - z:
        return 2.0 * PI
    if r >= z + p or r <= z - p:
        return 0.0
    c = (r * r + z * z - p * p) / (2.0 * r * z)
    return 2.0 * math.acos(min(1.0, max(-1.0, c)))


def ring_blocked(p, z, weight):
    """int_0^1 weight(r) r theta(r) dr with breakpoints at the kinks."""
    pts = sorted({abs(z - p), min(z + p, 1.0)} - {0.0, 1.0})
    pts = [x for x in pts if 0.0 < x < 1.0]
    val, err = integrate.quad(lambda r: weight(r) * r * arc_angle(r, p, z), 0.0, 1.0, points=pts or None,
                              epsabs=1e-14, epsrel=1e-13, limit=400)
    return val


def ring_flux_quad(p, z, u1, u2):
    """Definition: f = 1 - (1/F_tot) int int_overlap I dA, F_tot = pi (1 - u1/3 - u2/6)."""
    return 1.0 - ring_blocked(p, z, lambda r: intensity(r, u1, u2)) / (PI * (1.0 - u1 / 3.0 - u2 / 6.0))


def ring_alpha(n, p, z):
    """alpha_n = (1/pi) int int_overlap mu^n dA."""
    return ring_blocked(p, z, lambda r: max(0.0, 1.0 - r * r) ** (0.5 * n)) / PI


# ------------------------------------------------------------------ Carlson / elliptic
@pytest.mark.parametrize("x,y,z", [(0.0, 0.3, 1.0), (0.2, 0.7, 1.3), (1e-6, 1.0, 2.0), (0.5, 0.5, 0.5)])
def test_carlson_rf_rd(x, y, z):
    assert oracle.rf(x, y, z) == pytest.approx(float(mp.elliprf(x, y, z)), rel=1e-14)
    assert oracle.rd(x, y, z) == pytest.approx(float(mp.elliprd(x, y, z)), rel=1e-14)


@pytest.mark.parametrize("x,y,z,p", [(0.0, 0.3, 1.0, 2.0), (0.2, 0.7, 1.3, 0.1), (0.0, 1e-4, 1.0, 1e6),
                                     (0.0, 50.0, 1.0, 1e-8)])
def test_carlson_rj(x, y, z, p):
    assert oracle.rj(x, y, z, p) == pytest.approx(float(mp.elliprj(x, y, z, p)), rel=1e-13)


@pytest.mark.parametrize("x,y", [(0.3, 0.9), (0.9, 0.3), (0.0, 2.0), (1.0, 1.0)])
def test_carlson_rc(x, y):
    assert oracle.rc(x, y) == pytest.approx(float(mp.elliprc(x, y)), rel=1e-14)


@pytest.mark.parametrize("m", [0.0, 0.1, 0.5, 0.9, 0.999999])
def test_complete_k_e(m):
    assert oracle.ellk(m) == pytest.approx(float(mp.ellipk(m)), rel=1e-14)
    assert oracle.elle(m) == pytest.approx(float(mp.ellipe(m)), rel=1e-14)


def test_elliptic_special_values():
    assert oracle.ellk(0.0) == pytest.approx(PI / 2, rel=1e-15)
    assert oracle.elle(0.0) == pytest.approx(PI / 2, rel=1e-15)
    # Pi(0|m) = K(m)
    for m in (0.1, 0.6):
        assert oracle.ellpi(0.0, m) == pytest.approx(oracle.ellk(m), rel=1e-14)


@pytest.mark.parametrize("n,m", [(-2.5, 0.36), (-1e12, 0.09), (-3.0, 0.998001), (0.5, 0.04), (-0.01, 0.5),
                                 (-1e-6, 0.2)])
def test_complete_pi(n, m):
    # mpmath's ellippi(n, m) uses the same (1 - n sin^2) convention
    assert oracle.ellpi(n, m) == pytest.approx(float(mp.ellippi(n, m)), rel=1e-13)


# ------------------------------------------------------------------ Mandel-Agol
def test_lambda_e_closed_forms():
    for p in (0.05, 0.1, 0.3):
        assert oracle.lambda_e(p, 1.0 + p) == 0.0
        assert oracle.lambda_e(p, 2.0) == 0.0
        assert oracle.lambda_e(p, 0.5 * (1 - p)) == pytest.approx(p * p, rel=1e-15)
    # lens area against the ring integral of a uniform disk
    for p, z in [(0.1, 0.95), (0.3, 1.1), (0.7, 0.5), (1.5, 1.0)]:
        assert oracle.lambda_e(p, z) == pytest.approx(ring_blocked(p, z, lambda r: 1.0) / PI, abs=1e-13)


def test_out_of_transit_is_exactly_one():
    for p in (0.05, 0.2, 0.5):
        for z in (1.0 + p, 1.0 + p + 1e-12, 3.0, oracle.Z_BEHIND):
            assert oracle.flux_quad(p, z, 0.4, 0.2) == 1.0


def test_uniform_disk_closed_form():
    for p in (0.05, 0.1, 0.2):
        for z in (0.0, 0.3, 0.5 * (1 - p)):
            assert oracle.flux_quad(p, z, 0.0, 0.0) == pytest.approx(1.0 - p * p, abs=1e-15)
        for z in (1.0 - 0.5 * p, 1.0, 1.0 + 0.5 * p):
            assert oracle.flux_quad(p, z, 0.0, 0.0) == pytest.approx(1.0 - oracle.lambda_e(p, z), abs=1e-15)


def _z0_closed_form(k, u1, u2):
    """f(z=0) = 1 - [2 pi int_0^k I(r) r dr] / F_tot with r dr = -mu dmu: the
    integrand is a polynomial in mu, integrated from mu_k = sqrt(1-k^2) to 1."""
    mk = math.sqrt(1.0 - k * k)

    def prim(m):
        c0 = 1.0 - u1 - u2            # coefficient of mu^1 in I(mu) * mu
        c1 = u1 + 2.0 * u2            # coefficient of mu^2
        c2 = -u2                      # coefficient of mu^3
        return c0 * m ** 2 / 2 + c1 * m ** 3 / 3 + c2 * m ** 4 / 4

    blocked = 2.0 * PI * (prim(1.0) - prim(mk))
    return 1.0 - blocked / (PI * (1.0 - u1 / 3.0 - u2 / 6.0))


@pytest.mark.parametrize("k", [0.05, 0.1, 0.3, 0.7])
@pytest.mark.parametrize("u1,u2", [(0.4, 0.2), (0.1, 0.6), (0.9, -0.3)])
def test_z_zero_closed_form(k, u1, u2):
    assert oracle.flux_quad(k, 0.0, u1, u2) == pytest.approx(_z0_closed_form(k, u1, u2), abs=1e-14)


GRID = [(p, z) for p in (0.05, 0.1, 0.3, 0.7, 1.3)
        for z in (0.02, 0.3, 0.6, 0.8, 0.95, 1.0, 1.1, 1.25, 1.6, 2.2) if z < 1 + p]


@pytest.mark.parametrize("p,z", GRID)
def test_flux_quad_vs_ring_integral(p, z):
    u1, u2 = 0.4, 0.2
    assert oracle.flux_quad(p, z, u1, u2) == pytest.approx(ring_flux_quad(p, z, u1, u2), abs=2e-12)


@pytest.mark.parametrize("p,z,label", [
    (0.1, 0.0, "case 10 lambda_6"), (0.3, 0.3, "case 5 lambda_4"), (0.7, 0.7, "case 7 lambda_3"),
    (0.1, 0.9, "case 4 lambda_5"), (0.7, 0.3, "lambda_5, p > 1/2"), (0.5, 0.5, "case 6"),
    (2.0, 0.5, "case 11 star covered"), (0.3, 0.7, "case 4, p = 0.3")])
def test_flux_quad_special_cases(p, z, label):
    if p >= 1 and z <= p - 1:
        assert oracle.flux_quad(p, z, 0.4, 0.2) == pytest.approx(0.0, abs=1e-15)
        return
    assert oracle.flux_quad(p, z, 0.4, 0.2) == pytest.approx(ring_flux_quad(p, z, 0.4, 0.2), abs=1e-11), label


@pytest.mark.parametrize("p,zs", [(0.1, 0.1), (0.3, 0.3), (0.1, 0.9), (0.3, 0.7), (0.7, 0.7), (0.7, 0.3)])
def test_flux_quad_continuous_through_special_points(p, zs):
    """The general formulas just off a special point agree with the special
    formula on it (and with the ring integral): no dropped Theta term."""
    f0 = oracle.flux_quad(p, zs, 0.4, 0.2)
    for dz in (-1e-9, 1e-9):
        f = oracle.flux_quad(p, zs + dz, 0.4, 0.2)
        assert abs(f - f0) < 1e-8
        assert f == pytest.approx(ring_flux_quad(p, zs + dz, 0.4, 0.2), abs=1e-9)


def _brute_force_2d(p, z, u1, u2, n=1500):
    """Midpoint sum over the planet disk in polar coordinates about its own
    centre, keeping points inside the star."""
    rho = (np.arange(n) + 0.5) / n * p
    phi = (np.arange(2 * n) + 0.5) / (2 * n) * 2 * PI
    R, F = np.meshgrid(rho, phi, indexing="ij")
    x = z + R * np.cos(F)
    y = R * np.sin(F)
    r2 = x * x + y * y
    inside = r2 < 1.0
    mu = np.sqrt(np.clip(1.0 - r2, 0.0, None))
    I = (1.0 - u1 * (1 - mu) - u2 * (1 - mu) ** 2) * inside
    blocked = np.sum(I * R) * (p / n) * (2 * PI / (2 * n))
    return 1.0 - blocked / (PI * (1 - u1 / 3 - u2 / 6))


@pytest.mark.parametrize("p,z", [(0.1, 0.4), (0.1, 0.97), (0.2, 1.1), (0.3, 0.15)])
def test_flux_quad_vs_brute_force_2d(p, z):
    assert oracle.flux_quad(p, z, 0.5, 0.1) == pytest.approx(_brute_force_2d(p, z, 0.5, 0.1), abs=3e-6)


def test_flux_monotone_in_z_for_monotone_ld():
    p = 0.12
    zs = np.linspace(0.0, 1.0 + p, 400)
    f = oracle.flux_quad_vec(p, zs, 0.4, 0.2)
    assert np.all(np.diff(f) >= -1e-14)


# ------------------------------------------------------------------ Gimenez
@pytest.mark.parametrize("p,q,x", [(3.0, 2.0, 0.91), (3.0, 1.0, 0.3), (7.0, 6.0, 0.85), (7.0, 1.0, 0.99),
                                   (3.5, 2.5, 0.5)])
def test_jacobi_g_is_2f1(p, q, x):
    g = oracle.jacobi_g(30, p, q, x)
    ref = np.array([float(mp.hyp2f1(-j, p + j, q, x)) for j in range(30)])
    assert np.max(np.abs(g - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [0, 1, 2, 5, 8])
def test_gimenez_a_table(n):
    nu = mp.mpf(n + 2) / 2
    for j in (0, 1, 7, 40):
        ref = (-1) ** j * (2 * j + nu + 2) * mp.gamma(nu + j + 1) / (nu * mp.gamma(nu + 1) * mp.gamma(j + 2))
        assert oracle.gimenez_a(n, j) == pytest.approx(float(ref), rel=1e-12)


@pytest.mark.parametrize("n", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("z", [0.0, 0.5, 0.95, 1.05])
def test_gimenez_alpha_converges_to_ring_integral(n, z):
    k = 0.1
    exact = ring_alpha(n, k, z)
    a300 = oracle.gimenez_alpha(8, 300, k, z)[n]
    tol = {0: 2e-6, 1: 3e-7}.get(n, 5e-8)
    assert abs(a300 - exact) < tol
    # the error shrinks with the truncation depth (Fig. 1 behaviour)
    a20 = oracle.gimenez_alpha(8, 20, k, z)[n]
    assert abs(a300 - exact) <= abs(a20 - exact) + 1e-12


def test_gimenez_alpha_zero_out_of_transit():
    assert np.all(oracle.gimenez_alpha(8, 50, 0.1, 1.1) == 0.0)
    assert np.all(oracle.gimenez_alpha(8, 50, 0.1, 5.0) == 0.0)


def test_gimenez_matches_ma_for_quadratic_ld():
    """Both models describe the same physics: with u_1 = a + 2b, u_2 = -b
    (Sec. 2.1.2) the Gimenez flux agrees with MA to the truncation error."""
    a, b = 0.4, 0.2
    u = [a + 2 * b, -b]
    for k in (0.05, 0.1, 0.2):
        for z in (0.1, 0.5, 0.9, 1.0, 1.0 + 0.5 * k):
            fg = oracle.flux_gimenez(k, z, u, 400)
            fm = oracle.flux_quad(k, z, a, b)
            assert abs(fg - fm) < 3e-6, (k, z, fg, fm)


def test_gimenez_c_coefficients_against_direct_integral():
    """A 4-term general law through C_n against the ring integral of the same
    intensity profile (pins C_0, C_n and the normalisation of Sec. 2.1.3)."""
    u = np.array([0.3, 0.2, -0.1, 0.05])
    k, z = 0.1, 0.6

    def I(r):
        mu = math.sqrt(max(0.0, 1 - r * r))
        return 1.0 - sum(u[n - 1] * (1 - mu ** n) for n in range(1, 5))

    ftot = PI * (1 - sum(n * u[n - 1] / (n + 2) for n in range(1, 5)))
    exact = 1.0 - ring_blocked(k, z, I) / ftot
    assert oracle.flux_gimenez(k, z, u, 300) == pytest.approx(exact, abs=3e-6)


# ------------------------------------------------------------------ orbits
def test_ecc_zero_equals_circular():
    a, inc, P, t0 = 10.0, math.radians(88.5), 3.0, 0.7
    for t in np.linspace(-1.4, 1.4, 41) + t0:
        zc = oracle.z_circ(t, t0, P, a, inc)
        ze, st = oracle.z_ecc(t, t0, P, a, inc, 0.0, 0.5 * PI)
        assert st == 0
        if zc >= oracle.Z_BEHIND:
            assert ze >= oracle.Z_BEHIND
        else:
            assert ze == pytest.approx(zc, rel=1e-12, abs=1e-12)


def test_circular_symmetry_and_period():
    a, inc, P, t0 = 10.0, math.radians(88.5), 3.0, 0.2
    for dt in (0.0, 0.01, 0.05, 0.1, 0.4):
        zp = oracle.z_circ(t0 + dt, t0, P, a, inc)
        zm = oracle.z_circ(t0 - dt, t0, P, a, inc)
        assert zp == pytest.approx(zm, rel=1e-12)
        assert oracle.z_circ(t0 + dt + 7 * P, t0, P, a, inc) == pytest.approx(zp, rel=1e-10)


@pytest.mark.parametrize("e,w", [(0.0, 1.0), (0.1, 0.3), (0.3, 2.5), (0.3, 4.0), (0.6, 5.5)])
def test_z_at_conjunction_is_impact_parameter(e, w):
    a, b = 12.0, 0.4
    inc = oracle.inc_from_b(b, a, e, w)
    z, st = oracle.z_ecc(0.0, 0.0, 3.0, a, inc, e, w)
    assert st == 0 and z == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("e", [0.0, 0.1, 0.5, 0.9, 0.97])
def test_kepler_residual(e):
    for M in np.linspace(-PI, PI, 37):
        E, it = oracle.kepler_newton(M, e)
        assert it > 0
        assert abs(E - e * math.sin(E) - M) < 1e-13


def test_ecc_minimum_near_t0_and_behind_masked():
    a, e, w = 8.0, 0.3, 1.2
    inc = oracle.inc_from_b(0.2, a, e, w)
    P = 3.0
    # half an orbit away the planet is behind the star
    z, _ = oracle.z_ecc(0.5 * P, 0.0, P, a, inc, e, w)
    assert z >= oracle.Z_BEHIND
    ts = np.linspace(-0.05, 0.05, 201)
    zs = np.array([oracle.z_ecc(t, 0.0, P, a, inc, e, w)[0] for t in ts])
    assert abs(ts[np.argmin(zs)]) < 0.01


# ------------------------------------------------------------------ batched drivers
def test_supersampling_is_mean_of_shifted_points():
    t = np.array([-0.05, -0.01, 0.0, 0.02])
    orb = dict(t0=[0.0], P=[3.0], a=[10.0], inc=[math.radians(88.5)])
    f1, _ = oracle.lc_ma(t, orb, [0.1], [[[0.4, 0.2]]], n_ss=5, t_exp=0.02)
    for i, ti in enumerate(t):
        vals = [oracle.flux_quad(0.1, oracle.z_circ(ti + 0.02 * ((s + 0.5) / 5 - 0.5), 0.0, 3.0, 10.0,
                                                    math.radians(88.5)), 0.4, 0.2) for s in range(5)]
        assert f1[0, 0, i] == pytest.approx(np.mean(vals), abs=1e-15)
    f_plain, _ = oracle.lc_ma(t, orb, [0.1], [[[0.4, 0.2]]], n_ss=1, t_exp=0.02)
    for i, ti in enumerate(t):
        assert f_plain[0, 0, i] == oracle.flux_quad(0.1, oracle.z_circ(ti, 0.0, 3.0, 10.0, math.radians(88.5)),
                                                    0.4, 0.2)


def test_batched_layout_and_ssr():
    rng = np.random.default_rng(3)
    t = np.linspace(-0.1, 0.1, 17)
    n_v, n_b = 3, 2
    orb = dict(t0=rng.uniform(-0.01, 0.01, n_v), P=np.full(n_v, 3.0), a=rng.uniform(8, 12, n_v),
               inc=np.full(n_v, math.radians(89.0)))
    k = rng.uniform(0.08, 0.12, (n_v, n_b))
    ld = rng.uniform(0.1, 0.3, (n_v, n_b, 2))
    f, _ = oracle.lc_ma(t, orb, k, ld)
    for v in range(n_v):
        for b in range(n_b):
            for i in (0, 8, 16):
                z = oracle.z_circ(t[i], orb["t0"][v], 3.0, orb["a"][v], orb["inc"][v])
                assert f[v, b, i] == oracle.flux_quad(k[v, b], z, ld[v, b, 0], ld[v, b, 1])
    y = rng.normal(1.0, 1e-3, (n_b, t.size))
    wt = rng.uniform(0.5, 2.0, (n_b, t.size))
    s = oracle.ssr(f, y, wt)
    assert np.allclose(s, np.sum(wt[None] * (y[None] - f) ** 2, axis=2), rtol=1e-14, atol=0)
