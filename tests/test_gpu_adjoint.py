"""GPU adjoint (pt_ma_quad_bwd and the autograd wrapper) against the FP64
oracle gradient, through the C ABI.

Tolerance (derived from the FP32 error of the two factors of every term
2 wt (f - y) df/dtheta): an absolute flux error eps_f = 1e-6 in f - y (the
exact path's flux tolerance) and a relative error eps_g in df/dtheta give
  |d grad_i| <= 2 sum_t wt |df/dtheta_i| (eps_f + eps_g |f - y|),
plus 1e-5 of sum_t |2 wt (f-y) df/dtheta_i| for the FP32 accumulation.
eps_g = 1e-5 for every component (t0, P, a, b, e, w, k, u1, u2): FP32
elliptic integrals and the chain rule through Kepler's equation.  Measured on
these configurations the largest error is 0.11 of this bound (w) and below
0.06 for every other component; the t0 gradient is a small difference of
ingress and egress terms, so its error is judged against the size of its
terms, not against the gradient itself.
"""
import numpy as np
import pytest

import oracle
from paper_1504_07433_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS_F = 1e-6
EPS_G = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


def _theta_rows(th, idx):
    names = ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")
    cols = []
    for nm in names:
        x = np.asarray(th[nm])[idx]
        cols.append(x.astype(np.float64) if nm in ("t0", "P") else x.astype(np.float32).astype(np.float64))
    return np.stack(cols, axis=1)


def _data(wl, n_ss, t_exp):
    rng = np.random.default_rng(99)
    true = wl["true"]
    th = np.array([true[nm] for nm in ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")])
    y = np.array([oracle.flux_theta(t, th, n_ss, t_exp) for t in wl["t"]])
    return (y + rng.normal(0, wl["noise"], y.size)).astype(np.float32)


def _bound(t, rows, y, wt, n_ss, t_exp):
    """Per-(vector, component) tolerance from the error model above."""
    out = np.zeros((rows.shape[0], 9))
    for v in range(rows.shape[0]):
        s1 = np.zeros(9)
        s2 = np.zeros(9)
        for j, tj in enumerate(t):
            f, g = oracle.flux_grad(tj, rows[v], n_ss, t_exp)
            w = 1.0 if wt is None else wt[j]
            r = abs(f - y[j])
            s1 += 2 * w * np.abs(g) * (EPS_F + EPS_G * r)
            s2 += 2 * w * r * np.abs(g)
        out[v] = s1 + 1e-5 * s2
    return out


@pytest.mark.parametrize("n_v,n_t,n_ss,spread", [(24, 1500, 1, 1.0), (9, 800, 3, 2.0), (5, 301, 1, 0.2)])
def test_adjoint_vs_oracle_gradient(torch_cuda, n_v, n_t, n_ss, spread):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.adjoint(n_v=n_v, n_t=n_t, spread=spread)
    t_exp = 0.01 if n_ss > 1 else 0.0
    y = _data(wl, n_ss, t_exp)
    rng = np.random.default_rng(5)
    wt = rng.uniform(0.5, 2.0, n_t).astype(np.float32)
    th_dev = pt.theta_to_device(wl["theta"])
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device="cuda")
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    ssr, grad, flux = pt.ma_quad_bwd(t, th_dev, torch.as_tensor(y, device="cuda"), torch.as_tensor(wt, device="cuda"),
                                     n_ss=n_ss, t_exp=t_exp, want_flux=True, n_bad=bad)
    assert int(bad.item()) == 0
    rows = _theta_rows(wl["theta"], slice(0, n_v))
    yd = y.astype(np.float64)
    wd = wt.astype(np.float64)
    ssr_r, grad_r = oracle.ssr_grad(wl["t"], rows, yd, wd, n_ss=n_ss, t_exp=t_exp)
    f_ref = np.array([[oracle.flux_theta(tj, rows[v], n_ss, t_exp) for tj in wl["t"]] for v in range(n_v)])
    f_gpu = flux.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(f_gpu - f_ref)) <= EPS_F
    assert (f_ref < 1).sum() > 0
    s = ssr.cpu().numpy().astype(np.float64)
    assert np.allclose(s, ssr_r, rtol=2e-4, atol=1e-9)
    g = grad.cpu().numpy().astype(np.float64)
    tol = _bound(wl["t"], rows, yd, wd, n_ss, t_exp)
    err = np.abs(g - grad_r)
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    assert np.all(err <= tol), (worst, g[worst], grad_r[worst], tol[worst])


def test_autograd_function_matches_adjoint(torch_cuda):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.adjoint(n_v=7, n_t=900)
    y = torch.as_tensor(_data(wl, 1, 0.0), device="cuda")
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device="cuda")
    th = pt.theta_to_device(wl["theta"])
    leaves = {nm: th[nm].clone().requires_grad_(True) for nm in th}
    ssr = pt.transit_ssr(t, y, leaves)
    weights = torch.arange(1, 8, dtype=torch.float32, device="cuda")
    (ssr * weights).sum().backward()
    ssr2, grad, _ = pt.ma_quad_bwd(t, th, y)
    assert torch.equal(ssr.detach(), ssr2)
    for i, nm in enumerate(pt.THETA_NAMES):
        ref = (weights * grad[:, i]).to(leaves[nm].grad.dtype)
        assert torch.allclose(leaves[nm].grad, ref, rtol=1e-6, atol=0), nm


def test_adjoint_full_size_sampled(torch_cuda):
    """4,096 eccentric vectors x 10,000 points (the adjoint workload) in the
    benchmark's launch configuration; 6 sampled vectors against the oracle."""
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.adjoint()
    y = _data(wl, 1, 0.0)
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device="cuda")
    th = pt.theta_to_device(wl["theta"])
    ssr, grad, _ = pt.ma_quad_bwd(t, th, torch.as_tensor(y, device="cuda"))
    g = grad.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(g))
    rng = np.random.default_rng(4)
    idx = rng.choice(4096, 6, replace=False)
    rows = _theta_rows(wl["theta"], idx)
    ssr_r, grad_r = oracle.ssr_grad(wl["t"], rows, y.astype(np.float64))
    tol = _bound(wl["t"], rows, y.astype(np.float64), None, 1, 0.0)
    assert np.all(np.abs(g[idx] - grad_r) <= tol)
    assert np.allclose(ssr.cpu().numpy()[idx], ssr_r, rtol=2e-4)


def test_adjoint_tile_skipping_epochs_and_order(torch_cuda):
    """Tiles of 64 times that meet no transit window are skipped (flux 1,
    residual sum from the tile's FP64 sum of wt (y - 1)^2).  Times over ten
    orbits, and the same times shuffled so that every tile spans them all (no
    tile can be skipped): flux bitwise the same point by point, residual sums
    and gradients of both orders against the oracle."""
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    n_v, n_t = 6, 3000
    wl = W.adjoint(n_v=n_v, n_t=n_t)
    rng = np.random.default_rng(21)
    t_sorted = np.sort(rng.uniform(-10.0, 20.0, n_t))
    perm = rng.permutation(n_t)
    true = wl["true"]
    th_true = np.array([true[nm] for nm in ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")])
    y = np.array([oracle.flux_theta(tj, th_true, 1, 0.0) for tj in t_sorted])
    y = (y + rng.normal(0, 1e-4, n_t)).astype(np.float32)
    wt = rng.uniform(0.5, 2.0, n_t).astype(np.float32)
    th = pt.theta_to_device(wl["theta"])
    rows = _theta_rows(wl["theta"], slice(0, n_v))
    out = {}
    for name, order in (("sorted", np.arange(n_t)), ("shuffled", perm)):
        t = torch.as_tensor(t_sorted[order], dtype=torch.float64, device="cuda")
        ssr, grad, flux = pt.ma_quad_bwd(t, th, torch.as_tensor(y[order], device="cuda"),
                                         torch.as_tensor(wt[order], device="cuda"), want_flux=True)
        f = np.empty((n_v, n_t), np.float32)
        f[:, order] = flux.cpu().numpy()
        out[name] = (ssr.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64), f)
    assert np.array_equal(out["sorted"][2], out["shuffled"][2])
    assert (out["sorted"][2] < 1).sum() > 0
    ssr_r, grad_r = oracle.ssr_grad(t_sorted, rows, y.astype(np.float64), wt.astype(np.float64))
    tol = _bound(t_sorted, rows, y.astype(np.float64), wt.astype(np.float64), 1, 0.0)
    for name in out:
        s, g, _ = out[name]
        assert np.allclose(s, ssr_r, rtol=2e-4, atol=1e-9), name
        assert np.all(np.abs(g - grad_r) <= tol), name
