"""GPU parity of the interpolated Mandel-Agol path (Sec. 2.2.3:
pt_ma_table_create, pt_ma_terms_interp, pt_ma_quad_interp) against the FP64
oracle's own table and interpolation, through the C ABI.

Tolerances: the table nodes are the exact FP32 terms (~2e-7 from FP64) at
FP32-rounded node positions, and the interpolation runs in FP32, so each term
agrees with the oracle's interpolation to 1e-6 and the flux to 1e-6 (the
exact path's bound).  The interpolation error itself (against the exact
model) is a property of the method, checked at the paper's scale.
"""
import numpy as np
import pytest

import oracle
from paper_1504_07433_gb300 import workloads as W
from tests.helpers import f32, gpu_inputs, oracle_orbit

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


def _terms(pt, torch, table, k, z):
    kd = torch.as_tensor(np.asarray(k, np.float32), device="cuda")
    zd = torch.as_tensor(np.asarray(z, np.float32), device="cuda")
    return np.stack([x.cpu().numpy().astype(np.float64) for x in pt.ma_terms_interp(table, kd, zd)], axis=1)


def test_nodes_and_random_points_vs_oracle(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    k_lo, k_hi, n_k, n_z = 0.05, 0.2, 32, 256
    tab = pt.MATable(k_lo, k_hi, n_k, n_z)
    ref = oracle.MATable(k_lo, k_hi, n_k, n_z)
    rng = np.random.default_rng(7)
    # every node of three k rows, at the FP32-rounded node positions
    ii = np.array([0, 13, n_k - 1])
    jj = np.arange(n_z)
    k = np.repeat(k_lo + ii * (k_hi - k_lo) / (n_k - 1), n_z).astype(np.float32)
    z = np.tile(jj * (1.0 + k_hi) / (n_z - 1), ii.size).astype(np.float32)
    got = _terms(pt, torch, tab, k, z)
    exp = ref.terms_vec(k.astype(np.float64), z.astype(np.float64))
    assert np.max(np.abs(got - exp)) <= TOL
    # random points across the table, including k outside it (clamped), the
    # contacts z = 1 - k, z = k, and out of transit
    n = 4000
    k = rng.uniform(0.03, 0.22, n).astype(np.float32)
    z = (rng.uniform(0.0, 1.3, n) * (1 + k)).astype(np.float32)
    z[:50] = (1 - k[:50])
    z[50:100] = k[50:100]
    z[100:110] = 1e30
    got = _terms(pt, torch, tab, k, z)
    exp = ref.terms_vec(k.astype(np.float64), z.astype(np.float64))
    assert np.max(np.abs(got - exp)) <= TOL
    out = z.astype(np.float64) >= 1 + k.astype(np.float64)
    assert np.all(got[out] == 0.0)
    # flux from the terms for physical laws
    q1, q2 = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    u1, u2 = W.q_to_u(q1, q2)
    c = u1 + 2 * u2
    D = 1 - u1 / 3 - u2 / 6
    fg = ((1 - c) * got[:, 0] + c * got[:, 1] + u2 * got[:, 2]) / D
    fe = ((1 - c) * exp[:, 0] + c * exp[:, 1] + u2 * exp[:, 2]) / D
    assert np.max(np.abs(fg - fe)) <= TOL


def test_interpolation_error_at_paper_scale(torch_cuda):
    """Default grid (n_k = 128, n_z = 256) over a 0.02 range of k: a few ppm
    against the exact model (the paper prints ~4 ppm)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    tab = pt.MATable(0.05, 0.07, 128, 256)
    k = np.repeat(np.linspace(0.05, 0.07, 5), 3000).astype(np.float32)
    z = np.concatenate([np.linspace(0, 1 + kk, 3000, endpoint=False) for kk in np.linspace(0.05, 0.07, 5)])
    z = z.astype(np.float32)
    got = _terms(pt, torch, tab, k, z)
    u1, u2 = 0.4, 0.25
    c = u1 + 2 * u2
    fg = 1 - ((1 - c) * got[:, 0] + c * got[:, 1] + u2 * got[:, 2]) / (1 - u1 / 3 - u2 / 6)
    fe = oracle.flux_quad_vec(k.astype(np.float64), z.astype(np.float64), u1, u2)
    err = np.max(np.abs(fg - fe))
    assert 5e-7 < err < 1.5e-5


@pytest.mark.parametrize("n_t,n_v,n_ss,kpb", [(1500, 5, 10, False), (700, 3, 1, False), (333, 2, 3, True)])
def test_lc_interp_vs_oracle(torch_cuda, n_t, n_v, n_ss, kpb):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=n_v, n_t=n_t, n_ss=n_ss, cadence=0.01)
    n_b = 3 if kpb else 1
    if kpb:
        rng = np.random.default_rng(3)
        wl["k"] = wl["k"][:, None] * rng.uniform(0.95, 1.05, (n_v, n_b))
        wl["ld"] = np.repeat(wl["ld"], n_b, axis=1)
    t, orb, k, ld = gpu_inputs(wl)
    tab = pt.MATable(0.04, 0.22, 64, 256)
    ref = oracle.MATable(0.04, 0.22, 64, 256)
    flux, _ = pt.ma_quad_interp(tab, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"])
    f = flux.cpu().numpy().astype(np.float64)
    exp = oracle.lc_ma_interp(ref, wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]),
                              n_ss=n_ss, t_exp=wl["t_exp"])[0]
    assert (exp < 1).sum() > 0
    assert np.max(np.abs(f - exp)) <= TOL
    # and the residual sums through the same path
    y = torch.as_tensor(np.random.default_rng(1).normal(1.0, 1e-3, (n_b, n_t)).astype(np.float32), device="cuda")
    _, ssr = pt.ma_quad_interp(tab, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"], y=y, want_flux=False,
                               want_ssr=True)
    yy = y.cpu().numpy().astype(np.float64)
    assert np.allclose(ssr.cpu().numpy(), np.sum((yy[None] - f) ** 2, axis=2), rtol=2e-5)


def test_table_edges_and_errors(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    # the smallest table: bilinear over one cell
    tab = pt.MATable(0.1, 0.11, 2, 2)
    ref = oracle.MATable(0.1, 0.11, 2, 2)
    k = np.array([0.1, 0.105, 0.11, 0.105], np.float32)
    z = np.array([0.2, 0.5, 1.0, 1.2], np.float32)
    got = _terms(pt, torch, tab, k, z)
    assert np.max(np.abs(got - ref.terms_vec(k.astype(np.float64), z.astype(np.float64)))) <= TOL
    # empty input
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    le, ld, ed = pt.ma_terms_interp(tab, e, e)
    assert le.numel() == 0
    # invalid tables are refused on the host
    for args in [(0.1, 0.1, 8, 8), (0.2, 0.1, 8, 8), (0.1, 0.2, 1, 8), (0.1, 0.2, 8, 1), (0.0, 0.2, 8, 8)]:
        with pytest.raises(pt.PTError):
            pt.MATable(*args)
