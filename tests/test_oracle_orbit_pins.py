"""Pins of the oracle's orbits (Sec. 1: circular orbits and eccentric orbits
solved by Newton's method; the paper prints no orbit formula) away from
conjunction.

Referee: the planet's sky position from an independent 3-D construction.  The
Keplerian ellipse is placed in its orbital plane with periapsis on the x axis,
(a (cos E - e), a sqrt(1 - e^2) sin E, 0) with E from Kepler's equation solved
by bracketing root-finding (scipy brentq), then rotated by R_z(Omega) R_x(i)
R_z(w); the observer looks along the line of sight +Z, so the planet is in
front of the star when its Z > 0 and z is its distance from the star in the
sky plane.  The time of inferior conjunction t0 is found by root-finding too:
the mean anomaly where the planet crosses the plane through the line of sight
and the sky-plane axis perpendicular to the line of nodes, on the observer's
side.  None of this shares a formula with the oracle's half-angle anomaly
maps, its conjunction anchor or its projection.

Also: z_circ(t0 +- P/4) -> a; a face-on orbit has z = r, so z = a (1 - e) at
periapsis; the impact parameter of oracle.inc_from_b is the referee's sky
distance at conjunction.  The last test plants mistakes in a copy of the
oracle (an omega sign, a swapped projection, a wrong radius, ...) and checks
that these pins catch every one.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle

PI = math.pi
HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "pt_oracle.c")


# ------------------------------------------------------------------ referee
def kepler_E(M, e):
    if e == 0.0:
        return M
    return brentq(lambda E: E - e * math.sin(E) - M, M - e - 1e-9, M + e + 1e-9, xtol=1e-15, rtol=1e-15,
                  maxiter=200)


def sky(M, a, e, inc, w, Om=0.7):
    """(sky distance, line-of-sight coordinate Z, in-plane X1) at mean anomaly M."""
    E = kepler_E(M, e)
    x = a * (math.cos(E) - e)
    y = a * math.sqrt(1.0 - e * e) * math.sin(E)
    x1 = x * math.cos(w) - y * math.sin(w)          # R_z(w)
    y1 = x * math.sin(w) + y * math.cos(w)
    X, Y, Z = x1, y1 * math.cos(inc), y1 * math.sin(inc)   # R_x(i)
    Xs = X * math.cos(Om) - Y * math.sin(Om)        # R_z(Omega): a rotation within the sky plane
    Ys = X * math.sin(Om) + Y * math.cos(Om)
    return math.hypot(Xs, Ys), Z, x1, y1


def conjunction_M(a, e, w):
    """Mean anomaly of inferior conjunction: x1 = 0 with y1 > 0 (the planet on
    the observer's side of the star), by a sign scan and brentq."""
    grid = np.linspace(0.0, 2 * PI, 721)
    vals = [sky(M, a, e, 0.5, w)[2:] for M in grid]
    for i in range(len(grid) - 1):
        (x0, y0), (x1, _) = vals[i], vals[i + 1]
        if x0 == 0.0 and y0 > 0:
            return grid[i]
        if x0 * x1 < 0 and y0 > 0:
            return brentq(lambda M: sky(M, a, e, 0.5, w)[2], grid[i], grid[i + 1], xtol=1e-15, rtol=1e-15)
    raise AssertionError("no conjunction found")


# ------------------------------------------------------------------ the pins as functions of the oracle
class _Lib:
    """z_ecc / z_circ / inc_from_b of an oracle library (the real one or a
    planted copy)."""

    def __init__(self, cdll):
        D, I = ctypes.c_double, ctypes.c_int
        self.lib = cdll
        cdll.pto_z_ecc.restype = D
        cdll.pto_z_ecc.argtypes = [D, D, D, D, D, D, D, I, D, ctypes.POINTER(I)]
        cdll.pto_z_circ.restype = D
        cdll.pto_z_circ.argtypes = [D, D, D, D, D]
        cdll.pto_inc_from_b.restype = D
        cdll.pto_inc_from_b.argtypes = [D, D, D, D]

    def z_ecc(self, t, t0, P, a, inc, e, w):
        st = ctypes.c_int()
        return self.lib.pto_z_ecc(t, t0, P, a, inc, e, w, 60, 1e-15, ctypes.byref(st))

    def z_circ(self, t, t0, P, a, inc):
        return self.lib.pto_z_circ(t, t0, P, a, inc)

    def inc_from_b(self, b, a, e, w):
        return self.lib.pto_inc_from_b(b, a, e, w)


ORBITS = [(a, e, w, inc) for a in (5.0, 15.0) for e in (0.0, 0.1, 0.3, 0.6) for w in (0.3, 1.9, 4.0, 5.5)
          for inc in (math.radians(88.0), math.radians(60.0), 0.0)]


def rotation_failures(L, a, e, w, inc, n_m=60):
    """Mismatches between the oracle's z_ecc and the 3-D referee at n_m mean
    anomalies over a whole orbit plus a few near conjunction."""
    P, t0 = 3.0, 0.4
    Mc = conjunction_M(a, e, w)
    offs = list(2 * PI * (np.arange(n_m) / n_m - 0.5)) + [-0.05, -0.01, 0.002, 0.02]
    bad = []
    for dM in offs:
        t = t0 + dM * P / (2 * PI)
        zr, Z, _, _ = sky(Mc + dM, a, e, inc, w)
        zo = L.z_ecc(t, t0, P, a, inc, e, w)
        if abs(Z) < 1e-9 * a:
            continue
        if Z > 0:
            if not abs(zo - zr) <= 1e-11 * a:
                bad.append((dM, zo, zr))
        elif zo < oracle.Z_BEHIND:
            bad.append((dM, zo, "behind"))
    return bad


def circular_failures(L, a, inc):
    P, t0 = 2.5, -0.3
    bad = []
    for dM in 2 * PI * (np.arange(48) / 48 - 0.5) + 1e-3:
        t = t0 + dM * P / (2 * PI)
        zr, Z, _, _ = sky(dM, a, 0.0, inc, 0.5 * PI)   # circular: conjunction at M = 0 when w = pi/2
        zo = L.z_circ(t, t0, P, a, inc)
        if abs(Z) < 1e-9 * a:
            continue
        if (Z > 0 and not abs(zo - zr) <= 1e-11 * a) or (Z < 0 and zo < oracle.Z_BEHIND):
            bad.append((dM, zo, zr))
    # a quarter period from conjunction the planet is at the full radius a
    for s in (1.0, -1.0):
        zq = L.z_circ(t0 + s * P / 4 * (1 - 1e-9), t0, P, a, inc)
        if not abs(zq - a) <= 1e-6 * a:
            bad.append(("quarter", s, zq))
    return bad


def periapsis_failures(L):
    """Face-on orbits (i = 0): z = r, and at periapsis r = a (1 - e)."""
    bad = []
    for e in (0.1, 0.3, 0.6):
        for w in (0.5, 1.2, 2.0):        # periapsis on the observer's side (sin w > 0)
            a, P, t0 = 7.0, 3.0, 0.25
            Mc = conjunction_M(a, e, w)
            t = t0 - Mc * P / (2 * PI)       # M = 0
            t -= P * round((t - t0) / P)
            z = L.z_ecc(t, t0, P, a, 0.0, e, w)
            if not abs(z - a * (1 - e)) <= 1e-12 * a:
                bad.append((e, w, z, a * (1 - e)))
    return bad


def impact_failures(L):
    """inc_from_b(b, ...) must give the inclination whose sky distance at
    conjunction (the referee's) is b."""
    bad = []
    for a, e, w, b in [(12.0, 0.0, 1.0, 0.4), (12.0, 0.3, 2.5, 0.4), (8.0, 0.6, 5.5, 0.7), (20.0, 0.2, 4.0, 0.1)]:
        inc = L.inc_from_b(b, a, e, w)
        zc = sky(conjunction_M(a, e, w), a, e, inc, w)[0]
        if not abs(zc - b) <= 1e-10:
            bad.append((a, e, w, b, zc))
    return bad


def all_failures(L):
    bad = []
    for a, e, w, inc in ORBITS[::3]:
        bad += rotation_failures(L, a, e, w, inc, n_m=24)
    for a, inc in [(5.0, math.radians(85.0)), (12.0, math.radians(30.0))]:
        bad += circular_failures(L, a, inc)
    return bad + periapsis_failures(L) + impact_failures(L)


REAL = _Lib(oracle._lib())


# ------------------------------------------------------------------ tests of the oracle
@pytest.mark.parametrize("a,e,w,inc", ORBITS)
def test_z_ecc_against_3d_rotation(a, e, w, inc):
    assert rotation_failures(REAL, a, e, w, inc) == []


@pytest.mark.parametrize("a,inc", [(5.0, math.radians(85.0)), (10.0, math.radians(88.5)), (12.0, math.radians(30.0)),
                                   (30.0, 0.0)])
def test_z_circ_against_3d_rotation_and_quarter_period(a, inc):
    assert circular_failures(REAL, a, inc) == []


def test_face_on_periapsis_distance():
    assert periapsis_failures(REAL) == []


def test_impact_parameter_at_conjunction():
    assert impact_failures(REAL) == []


# ------------------------------------------------------------------ planted mistakes
PLANTS = {
    "omega sign at conjunction": ("double ftr = 0.5 * PTO_PI - w;", "double ftr = 0.5 * PTO_PI + w;", "pto_z_ecc"),
    "sin/cos swapped in the sky projection": ("return r * sqrt(c * c + s * s * ci * ci);",
                                              "return r * sqrt(s * s + c * c * ci * ci);", "pto_z_ecc"),
    "wrong sign in r(E)": ("double r = a * (1.0 - e * cos(E));", "double r = a * (1.0 + e * cos(E));", "pto_z_ecc"),
    "true anomaly factors swapped": ("sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E)",
                                     "sqrt(1.0 - e) * sin(0.5 * E), sqrt(1.0 + e) * cos(0.5 * E)", "pto_z_ecc"),
    "wrong sign in M at conjunction": ("double Mtr = Etr - e * sin(Etr);", "double Mtr = Etr + e * sin(Etr);",
                                       "pto_z_ecc"),
    "behind-the-star mask inverted": ("if (s <= 0.0) return PTO_Z_BEHIND;", "if (s >= 0.0) return PTO_Z_BEHIND;",
                                      "pto_z_ecc"),
    "omega sign in b -> i": ("(1.0 + e * sin(w)) / (1.0 - e * e)", "(1.0 - e * sin(w)) / (1.0 - e * e)",
                             "pto_inc_from_b"),
    "circular projection swapped": ("return a * sqrt(sp * sp + ci * ci * cp * cp);",
                                    "return a * sqrt(cp * cp + ci * ci * sp * sp);", "pto_z_circ"),
}


def _planted_library(tmp_path, name):
    old, new, func = PLANTS[name]
    src = open(SRC).read()
    start = src.index("double %s(" % func)
    pos = src.index(old, start)
    mutated = src[:pos] + new + src[pos + len(old):]
    c = tmp_path / "planted.c"
    so = tmp_path / "planted.so"
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"], check=True)
    return _Lib(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_orbit_mistake_is_caught(tmp_path, name):
    assert len(all_failures(_planted_library(tmp_path, name))) > 0


def test_pins_pass_on_the_unplanted_copy(tmp_path):
    # the same build route as the planted copies, without a change
    so = tmp_path / "clean.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", SRC, "-o", str(so), "-lm"], check=True)
    assert all_failures(_Lib(ctypes.CDLL(str(so)))) == []
