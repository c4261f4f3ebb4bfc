"""Writes gimenez_truncation.json: the truncation error of the Gimenez series.

The series of Eq. (gimenez) keeps N_J Jacobi terms (Sec. 2.1.1).  Its error
against the exact flux is the quantity of the paper's Fig. 1 (maximum and
mean absolute deviation over z in [0, 1 + k] as a function of N_J, two limb
darkening coefficients); the figure's values are not in the text, so they are
computed here.  Both sides come from the oracle only: the series
(oracle.flux_gimenez / oracle.gimenez_alpha) and the definition of the
occulted flux as a ring integral (oracle.ring_flux / oracle.ring_alpha).

Three parts:
  curve           Fig. 1's quantity for the quadratic law (u1, u2) = (0.4, 0.2)
                  at k = 0.05, 0.1, 0.2 on 400 evenly spaced z in [0, 1 + k).
  priors          the largest |delta f| over the long-cadence workload's
                  priors (k up to 0.2; q1, q2 in [0, 1] mapped to (u1, u2);
                  u3..u8 in [-0.02, 0.02]) for a range of N_J.  f is linear in
                  the alpha_n, so delta f = sum_n C_n delta alpha_n with the C_n
                  of Sec. 2.1.3; the maximum is taken over a 5 x 5 grid of
                  (q1, q2) times every sign pattern of u3..u8 = +-0.02, on z
                  grids refined around the kinks z = k and z = 1 - k.
  default_n_j     the smallest N_J of that range whose maximum stays below
                  1e-5 minus the 1e-6 budget of the FP32 evaluation.

Run from the repository root: python tests/golden/make_gimenez_truncation.py
"""
import itertools
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gimenez_truncation.json")

N_LD = 8
CURVE_K = (0.05, 0.1, 0.2)
CURVE_NJ = (8, 16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256)
PRIOR_K = (0.05, 0.1, 0.15, 0.2)
PRIOR_NJ = (128, 160, 176, 192, 208, 256)
BUDGET = 1e-5 - 1e-6


def curve_z(k):
    return np.linspace(0.0, 1.0 + k, 401)[:-1]


def prior_z(k):
    return np.unique(np.concatenate([np.linspace(0.0, 1.0 + k, 301)[:-1],
                                     1.0 - k + np.linspace(-0.004, 0.004, 161),
                                     k + np.linspace(-0.004, 0.004, 41)]))


def q_to_general(q1, q2):
    """q1, q2 -> quadratic (u1, u2) (Kipping 2013) -> general-law u_1 = u1 + 2 u2,
    u_2 = -u2 (Sec. 2.1.2)."""
    u1 = 2.0 * np.sqrt(q1) * q2
    u2 = np.sqrt(q1) * (1.0 - 2.0 * q2)
    return np.array([u1 + 2.0 * u2, -u2])


def prior_ld_sets():
    out = []
    for q1 in np.linspace(0.0, 1.0, 5):
        for q2 in np.linspace(0.0, 1.0, 5):
            base = np.zeros(N_LD)
            base[:2] = q_to_general(q1, q2)
            for signs in itertools.product((-1.0, 1.0), repeat=N_LD - 2):
                u = base.copy()
                u[2:] = 0.02 * np.array(signs)
                out.append(u)
    return np.array(out)


def c_coefficients(U):
    """C_0 = (1 - sum u_n)/D, C_n = u_n/D, D = 1 - sum n u_n/(n + 2) (Sec. 2.1.3)."""
    n = np.arange(1, U.shape[1] + 1)
    D = 1.0 - np.sum(n * U / (n + 2.0), axis=1)
    C = np.empty((U.shape[0], U.shape[1] + 1))
    C[:, 0] = (1.0 - U.sum(axis=1)) / D
    C[:, 1:] = U / D[:, None]
    return C


def main():
    u_curve = np.array([0.4 + 2 * 0.2, -0.2])   # quadratic (u1, u2) = (0.4, 0.2), Sec. 2.1.2
    curve = []
    for k in CURVE_K:
        zs = curve_z(k)
        ref = np.array([oracle.ring_flux(u_curve, k, z) for z in zs])
        for nj in CURVE_NJ:
            d = np.abs(np.array([oracle.flux_gimenez(k, z, u_curve, nj) for z in zs]) - ref)
            curve.append(dict(k=k, n_j=nj, max_abs=float(d.max()), mean_abs=float(d.mean()),
                              z_of_max=float(zs[int(np.argmax(d))])))
    C = c_coefficients(prior_ld_sets())
    priors = []
    for k in PRIOR_K:
        zs = prior_z(k)
        ring = np.array([[oracle.ring_alpha(n, k, z) for n in range(N_LD + 1)] for z in zs])
        for nj in PRIOR_NJ:
            ser = np.array([oracle.gimenez_alpha(N_LD, nj, k, z) for z in zs])
            df = np.abs(C @ (ser - ring).T)
            i, j = np.unravel_index(int(np.argmax(df)), df.shape)
            priors.append(dict(k=k, n_j=nj, max_abs=float(df.max()), z_of_max=float(zs[j]),
                               worst_c=[float(x) for x in C[i]]))
    worst = {nj: max(r["max_abs"] for r in priors if r["n_j"] == nj) for nj in PRIOR_NJ}
    default = min(nj for nj in PRIOR_NJ if worst[nj] <= BUDGET)
    doc = dict(
        citation="Sec. 2.1.1 (Eq. gimenez; Fig. 1: maximum and mean absolute deviation from the exact "
                 "solution over z in [0, 1 + k] against the number of Jacobi terms N_J)",
        how="oracle.flux_gimenez / oracle.gimenez_alpha (the series, N_J terms) against oracle.ring_flux / "
            "oracle.ring_alpha (the occulted flux from its definition, tanh-sinh ring integral)",
        curve_ld="quadratic (u1, u2) = (0.4, 0.2) as general-law (u_1, u_2) = (0.8, -0.2)",
        curve=curve,
        priors_desc="k in {0.05, 0.1, 0.15, 0.2}; q1, q2 on a 5 x 5 grid over [0, 1]; u3..u8 = +-0.02 (all "
                    "sign patterns); z on 300 even points over [0, 1 + k) plus 161 within 0.004 of 1 - k and 41 "
                    "within 0.004 of k",
        priors=priors,
        priors_worst={str(k): v for k, v in worst.items()},
        budget=BUDGET,
        default_n_j=default)
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("default n_j", default, {k: "%.3e" % v for k, v in worst.items()})


if __name__ == "__main__":
    main()
