"""Seeded synthetic workloads (inputs only).

This module draws the inputs every test, the smoke check and the benchmark
use: time grids, orbit parameters from the priors the workloads name, radius
ratios and limb-darkening coefficients.  It holds none of the transit model's
arithmetic and is imported by both the CUDA-path tests and the oracle tests;
neither the oracle nor the CUDA library imports the other.

Two parameter maps are part of input generation:
  * q1, q2 ~ U[0,1] to quadratic (u1, u2) (Kipping 2013, MNRAS 435, 2152):
    u1 = 2 sqrt(q1) q2,  u2 = sqrt(q1) (1 - 2 q2);
  * impact parameter b to inclination (Winn 2010, Exoplanets, eq. 7):
    b = a cos i (1 - e^2) / (1 + e sin w).

Workload recipes (seed 1504 + index):
  plain        1,000 times evenly over t0 +- 0.1 d, P = 3 d, a = 10, i = 88.5 deg,
               k = 0.1, (u1, u2) = (0.4, 0.2), circular, 1 vector, 1 passband.
  long_cadence 50,000 times every 0.02 d over 1,000 d, 29.4-min exposures
               supersampled x10, 256 vectors with k~U[.05,.2], b~U[0,.9],
               a~U[5,30], e~U[0,.3], w~U[0,2pi), q1,q2~U[0,1], P = 3 d,
               t0~U[0,3); one passband.  Gimenez variant: 8 general-law
               coefficients (u1, u2 from the quadratic law via Sec. 2.1.2,
               u3..u8 ~ U[-0.02, 0.02]).
  batched      32 transits of uneven length (500..5,000 points), each window
               centred on epoch j and T14/0.35 wide (35 % in transit, the
               paper's performance mix), 1,024 walkers jittered around the plain
               orbit, 64 passbands with k~U[.09,.11] and q1,q2~U[0,1] per
               (walker, passband); y = 1 + N(0, 1e-3^2) per passband.
  adjoint      4,096 eccentric vectors (priors as long_cadence) near a seeded
               true vector, 10,000 times evenly over t0 +- 0.15 d.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1504
T_EXP_LONG = 29.4 / (24.0 * 60.0)   # Kepler long-cadence exposure, days


def q_to_u(q1, q2):
    q1 = np.asarray(q1, dtype=np.float64)
    q2 = np.asarray(q2, dtype=np.float64)
    sq = np.sqrt(q1)
    return 2.0 * sq * q2, sq * (1.0 - 2.0 * q2)


def inc_from_b(b, a, e=0.0, w=0.5 * math.pi):
    b, a, e, w = (np.asarray(x, dtype=np.float64) for x in (b, a, e, w))
    return np.arccos(b / a * (1.0 + e * np.sin(w)) / (1.0 - e * e))


def quad_to_general(u1, u2, n_terms=2):
    """Quadratic (a, b) to general-law coefficients u_1 = a + 2b, u_2 = -b
    (Sec. 2.1.2), padded with zeros to n_terms."""
    u1 = np.asarray(u1, dtype=np.float64)
    u2 = np.asarray(u2, dtype=np.float64)
    out = np.zeros(u1.shape + (n_terms,))
    out[..., 0] = u1 + 2.0 * u2
    out[..., 1] = -u2
    return out


def plain(n_t=1000):
    t0 = 0.0
    t = np.linspace(t0 - 0.1, t0 + 0.1, n_t)
    orbit = dict(t0=np.array([t0]), P=np.array([3.0]), a=np.array([10.0]),
                 inc=np.array([math.radians(88.5)]), e=None, w=None)
    return dict(name="plain MA quadratic, circular, 1 vector, 1 passband, %d times" % n_t,
                t=t, orbit=orbit, k=np.array([0.1]), ld=np.array([[[0.4, 0.2]]]), n_ss=1, t_exp=0.0)


def long_cadence(n_v=256, n_t=50000, n_ss=10, seed=SEED + 1, n_gim=8, cadence=0.02):
    rng = np.random.default_rng(seed)
    t = np.arange(n_t, dtype=np.float64) * cadence
    k = rng.uniform(0.05, 0.2, n_v)
    b = rng.uniform(0.0, 0.9, n_v)
    a = rng.uniform(5.0, 30.0, n_v)
    e = rng.uniform(0.0, 0.3, n_v)
    w = rng.uniform(0.0, 2.0 * math.pi, n_v)
    q1 = rng.uniform(0.0, 1.0, n_v)
    q2 = rng.uniform(0.0, 1.0, n_v)
    P = np.full(n_v, 3.0)
    t0 = rng.uniform(0.0, 3.0, n_v)
    inc = inc_from_b(b, a, e, w)
    u1, u2 = q_to_u(q1, q2)
    ld = np.stack([u1, u2], axis=-1)[:, None, :]
    gen = quad_to_general(u1, u2, n_gim)
    if n_gim > 2:
        gen[:, 2:] = rng.uniform(-0.02, 0.02, (n_v, n_gim - 2))
    orbit = dict(t0=t0, P=P, a=a, inc=inc, e=e, w=w, b=b)
    return dict(name="long cadence: %d times over %.0f d, 29.4-min exposures x%d, %d eccentric vectors"
                % (n_t, n_t * cadence, n_ss, n_v),
                t=t, orbit=orbit, k=k, ld=ld, ld_gim=gen[:, None, :], n_ss=n_ss, t_exp=T_EXP_LONG)


def batched(n_walkers=1024, n_pb=64, n_lc=32, seed=SEED + 2, len_lo=500, len_hi=5000):
    """Spectrophotometric batch: n_lc light curves of uneven length around
    successive transits of one circular orbit, n_walkers parameter vectors,
    n_pb passbands each with its own k and LD pair."""
    rng = np.random.default_rng(seed)
    P, a, inc0, t00 = 3.0, 10.0, math.radians(88.5), 0.0
    b0 = a * math.cos(inc0)
    # T14 of the plain orbit with k = 0.11 (an upper bound for the passbands)
    t14 = P / math.pi * math.asin(math.sqrt((1.11) ** 2 - b0 ** 2) / (a * math.sin(inc0)))
    width = t14 / 0.35
    lengths = rng.integers(len_lo, len_hi + 1, n_lc)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    t = np.concatenate([t00 + j * P + np.linspace(-0.5 * width, 0.5 * width, int(L))
                        for j, L in enumerate(lengths)])
    t0 = t00 + rng.normal(0.0, 2e-4, n_walkers)
    Pw = P + rng.normal(0.0, 1e-6, n_walkers)
    aw = a + rng.normal(0.0, 0.05, n_walkers)
    bw = np.clip(b0 + rng.normal(0.0, 0.01, n_walkers), 0.0, None)
    incw = inc_from_b(bw, aw)
    k = rng.uniform(0.09, 0.11, (n_walkers, n_pb))
    q1 = rng.uniform(0.0, 1.0, (n_walkers, n_pb))
    q2 = rng.uniform(0.0, 1.0, (n_walkers, n_pb))
    u1, u2 = q_to_u(q1, q2)
    ld = np.stack([u1, u2], axis=-1)
    y = 1.0 + rng.normal(0.0, 1e-3, (n_pb, t.size))
    orbit = dict(t0=t0, P=Pw, a=aw, inc=incw, e=None, w=None, b=bw)
    return dict(name="batched spectrophotometry: %d walkers x %d passbands x %d light curves (%d points)"
                % (n_walkers, n_pb, n_lc, t.size),
                t=t, lc_offsets=offsets, orbit=orbit, k=k, ld=ld, y=y, n_ss=1, t_exp=0.0)


def adjoint(n_v=4096, n_t=10000, seed=SEED + 3, spread=1.0):
    """Eccentric vectors scattered around a seeded true vector; times evenly
    over t0 +- 0.15 d.  `spread` scales the scatter."""
    rng = np.random.default_rng(seed)
    true = dict(t0=0.0, P=3.0, a=12.0, b=0.3, e=0.15, w=1.1, k=0.1, u1=0.4, u2=0.2)
    t = np.linspace(-0.15, 0.15, n_t)
    s = spread
    th = dict(
        t0=true["t0"] + s * rng.normal(0, 2e-3, n_v),
        P=true["P"] + s * rng.normal(0, 1e-4, n_v),
        a=true["a"] * (1 + s * rng.normal(0, 0.03, n_v)),
        b=np.clip(true["b"] + s * rng.normal(0, 0.05, n_v), 0.0, 0.8),
        e=np.clip(true["e"] + s * rng.normal(0, 0.03, n_v), 0.0, 0.3),
        w=true["w"] + s * rng.normal(0, 0.1, n_v),
        k=true["k"] * (1 + s * rng.normal(0, 0.03, n_v)),
        u1=np.clip(true["u1"] + s * rng.normal(0, 0.05, n_v), 0.0, 1.0),
        u2=np.clip(true["u2"] + s * rng.normal(0, 0.05, n_v), -0.2, 0.6),
    )
    return dict(name="adjoint: %d eccentric vectors x %d times" % (n_v, n_t), t=t, theta=th, true=true,
                noise=1e-4, rng=rng)


def surrogate_points(n, seed=SEED + 4, k_lo=0.01, k_hi=0.3):
    """(k, z) over the ingress/egress band z in [|1-k|, 1+k]."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(k_lo, k_hi, n)
    s = rng.uniform(0.0, 1.0, n)
    z = np.abs(1.0 - k) + s * 2.0 * np.minimum(k, 1.0)
    return k, z, s
