"""Truncation error of the Gimenez series (Sec. 2.1.1, the quantity of Fig. 1).

tests/golden/gimenez_truncation.json is written by
tests/golden/make_gimenez_truncation.py from the oracle alone: the series at
N_J terms against the occulted flux from its definition (a ring integral,
pinned in test_oracle_ring_pins.py).  These tests recompute entries of it,
check what the paper states about the curve, and fix the default series depth
of the long-cadence workload: the smallest N_J whose largest error over that
workload's priors stays within 1e-5 less the FP32 budget of 1e-6.
"""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "gimenez_truncation.json")))
PRINTED = json.load(open(os.path.join(HERE, "golden", "paper_printed.json")))

import importlib.util  # noqa: E402

_spec = importlib.util.spec_from_file_location("make_gimenez_truncation",
                                               os.path.join(HERE, "golden", "make_gimenez_truncation.py"))
MK = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(MK)


def _row(rows, k, nj):
    return next(r for r in rows if r["k"] == k and r["n_j"] == nj)


@pytest.mark.parametrize("k,nj", [(0.1, 40), (0.2, 128), (0.05, 192)])
def test_curve_entries_recomputed(k, nj):
    zs = MK.curve_z(k)
    u = np.array([0.8, -0.2])
    d = np.abs(np.array([oracle.flux_gimenez(k, z, u, nj) - oracle.ring_flux(u, k, z) for z in zs]))
    r = _row(GOLD["curve"], k, nj)
    assert d.max() == pytest.approx(r["max_abs"], rel=1e-6)
    assert d.mean() == pytest.approx(r["mean_abs"], rel=1e-6)


def test_prior_worst_case_recomputed_at_default_depth():
    k, nj = 0.2, GOLD["default_n_j"]
    zs = MK.prior_z(k)
    C = MK.c_coefficients(MK.prior_ld_sets())
    ring = np.array([[oracle.ring_alpha(n, k, z) for n in range(MK.N_LD + 1)] for z in zs])
    ser = np.array([oracle.gimenez_alpha(MK.N_LD, nj, k, z) for z in zs])
    worst = float(np.abs(C @ (ser - ring).T).max())
    assert worst == pytest.approx(_row(GOLD["priors"], k, nj)["max_abs"], rel=1e-6)


def test_default_depth_is_the_smallest_within_budget():
    worst = {int(k): v for k, v in GOLD["priors_worst"].items()}
    d = GOLD["default_n_j"]
    assert worst[d] <= GOLD["budget"] <= 1e-5 - 1e-6
    assert all(worst[nj] > GOLD["budget"] for nj in worst if nj < d)
    # the error grows with k over the prior (k <= 0.2 is the worst case)
    at_d = [_row(GOLD["priors"], k, d)["max_abs"] for k in MK.PRIOR_K]
    assert at_d == sorted(at_d)


def test_curve_converges_and_paper_claims():
    for k in MK.CURVE_K:
        mx = [_row(GOLD["curve"], k, nj)["max_abs"] for nj in MK.CURVE_NJ]
        mn = [_row(GOLD["curve"], k, nj)["mean_abs"] for nj in MK.CURVE_NJ]
        assert mx[-1] < mx[0] / 30 and mn[-1] < mn[0] / 100
        assert all(a <= b for a, b in zip(mn, mx))
    # Sec. 2.1.1: about 40 terms suffice for ground-based precision
    g = PRINTED["gimenez_nj_ground"]
    for k in MK.CURVE_K:
        assert _row(GOLD["curve"], k, g["n_j"])["max_abs"] < g["ground_precision_ppm"] * 1e-6
