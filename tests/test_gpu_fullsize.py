"""Parity at full size, in the launch configuration the benchmark times.

Long-cadence workload (50,000 exposures x 10 supersamples x 256 eccentric
vectors):
  * Mandel-Agol: every one of the 1.28e7 flux points against the oracle at
    1e-6, and the in-transit mask: a point the GPU puts in transit (flux < 1)
    that the oracle has fully out of transit (flux exactly 1) must graze
    contact, its smallest FP64 z within 1e-5 of 1 + k;
  * Gimenez (N = 8, the default depth): the first 64 vectors in full against
    the oracle at 1e-6, and on all 256 vectors flux exactly 1 wherever the
    oracle's Mandel-Agol flux is exactly 1 (no supersample within reach of
    the planet) except at grazing points as above.
Batched spectrophotometry (1,024 walkers x 64 passbands x 32 light curves):
64 sampled (walker, passband) residual sums of the fused-SSR plan, and the
full 64-passband flux cube of two walkers from the flux-cube plan.
Adjoint (4,096 vectors x 10,000 points): 64 vectors against the oracle
gradient.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1504_07433_gb300 import workloads as W
from tests.helpers import f32, gpu_inputs, oracle_orbit

pytestmark = pytest.mark.gpu

TOL = 1e-6
HERE = os.path.dirname(os.path.abspath(__file__))
N_J = json.load(open(os.path.join(HERE, "golden", "gimenez_truncation.json")))["default_n_j"]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


@pytest.fixture(scope="module")
def long_cadence():
    wl = W.long_cadence()
    f_ma, nbad = oracle.lc_ma(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]), n_ss=wl["n_ss"],
                              t_exp=wl["t_exp"])
    assert nbad == 0
    return wl, f_ma[:, 0]


def _grazing(wl, v, idx):
    """Smallest FP64 z over the supersamples of exposures idx of vector v,
    minus 1 + k."""
    o = oracle_orbit(wl["orbit"])
    k = float(np.float32(wl["k"][v]))
    out = []
    for i in idx:
        zs = [oracle.z_ecc(wl["t"][i] + wl["t_exp"] * ((s + 0.5) / wl["n_ss"] - 0.5), o["t0"][v], o["P"][v],
                           o["a"][v], o["inc"][v], o["e"][v], o["w"][v])[0] for s in range(wl["n_ss"])]
        out.append(min(zs) - (1.0 + k))
    return np.array(out)


def _check_mask(wl, f_gpu, f_ref_ma):
    """GPU in transit where the oracle is exactly out: only at grazing contact."""
    sus = np.argwhere((f_gpu < 1.0) & (f_ref_ma == 1.0))
    assert sus.shape[0] < 1000, sus.shape
    for v in np.unique(sus[:, 0]):
        gap = _grazing(wl, v, sus[sus[:, 0] == v, 1])
        assert np.all(gap < 1e-5), (v, gap.max())


def test_ma_full_long_cadence_every_point(torch_cuda, long_cadence):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl, ref = long_cadence
    t, orb, k, ld = gpu_inputs(wl)
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    flux, _ = pt.ma_quad(t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], n_bad=bad)
    f = flux.cpu().numpy()[:, 0].astype(np.float64)
    assert int(bad.item()) == 0
    err = np.abs(f - ref)
    assert err.max() <= TOL, np.unravel_index(np.argmax(err), err.shape)
    assert (ref < 1).sum() > 100000
    _check_mask(wl, f, ref)


def test_gimenez_full_long_cadence_64_vectors_in_full(torch_cuda, long_cadence):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl, ref_ma = long_cadence
    t, orb, k, _ = gpu_inputs(wl)
    ldg = torch.as_tensor(np.asarray(wl["ld_gim"], np.float32), device="cuda")
    plan = pt.GimenezPlan(8, N_J)
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    flux, _ = pt.gimenez(plan, t, orb, k, ldg, n_ss=wl["n_ss"], t_exp=wl["t_exp"], n_bad=bad)
    f = flux.cpu().numpy()[:, 0].astype(np.float64)
    assert int(bad.item()) == 0
    n = 64
    sub = {kk: (None if vv is None else vv[:n]) for kk, vv in oracle_orbit(wl["orbit"]).items()}
    ref, nb = oracle.lc_gimenez(wl["t"], sub, f32(wl["k"][:n]), f32(wl["ld_gim"][:n]), N_J, n_ss=wl["n_ss"],
                                t_exp=wl["t_exp"])
    err = np.abs(f[:n] - ref[:, 0])
    assert nb == 0 and err.max() <= TOL, np.unravel_index(np.argmax(err), err.shape)
    _check_mask(wl, f, ref_ma)


def test_batched_full_size_64_ssrs_and_two_full_cubes(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.batched()
    t, orb, k, ld = gpu_inputs(wl)
    y = torch.as_tensor(wl["y"], dtype=torch.float32, device="cuda")
    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, y=y, want_flux=False, want_ssr=True)
    _, ssr = plan.run()
    torch.cuda.synchronize()
    s = ssr.cpu().numpy().astype(np.float64)
    plan.close()
    assert np.all(np.isfinite(s))
    rng = np.random.default_rng(41)
    pairs = [(int(v), int(b)) for v, b in zip(rng.choice(1024, 64, replace=False), rng.integers(0, 64, 64))]
    orb_o = oracle_orbit(wl["orbit"])
    yy = np.asarray(wl["y"], np.float32).astype(np.float64)
    vs = np.array([p[0] for p in pairs])
    bs = np.array([p[1] for p in pairs])
    ref = oracle.lc_ma(wl["t"], {kk: (None if vv is None else vv[vs]) for kk, vv in orb_o.items()},
                       f32(wl["k"])[vs, bs][:, None], f32(wl["ld"])[vs, bs][:, None, :])[0][:, 0]
    ssr_ref = np.sum((yy[bs] - ref) ** 2, axis=1)
    bound = np.sum(2 * np.abs(yy[bs] - ref) * TOL + TOL ** 2, axis=1) + 2e-5 * ssr_ref
    assert np.all(np.abs(s[vs, bs] - ssr_ref) <= bound)
    # flux-cube plan at full size (about 23 GB), two walkers' cubes in full
    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, want_flux=True, want_ssr=False)
    flux, _ = plan.run()
    torch.cuda.synchronize()
    for v in (0, int(rng.integers(1, 1024))):
        ref = oracle.lc_ma(wl["t"], {kk: (None if vv is None else vv[[v]]) for kk, vv in orb_o.items()},
                           f32(wl["k"])[[v]], f32(wl["ld"])[[v]])[0][0]
        f = flux[v].cpu().numpy().astype(np.float64)
        assert (ref < 1).mean() > 0.2
        assert np.max(np.abs(f - ref)) <= TOL, v
    plan.close()
    del flux
    torch.cuda.empty_cache()


def test_adjoint_full_size_64_vectors(torch_cuda):
    import paper_1504_07433_gb300 as pt
    from tests.test_gpu_adjoint import _bound, _data, _theta_rows
    torch = torch_cuda
    wl = W.adjoint()
    y = _data(wl, 1, 0.0)
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device="cuda")
    th = pt.theta_to_device(wl["theta"])
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    ssr, grad, _ = pt.ma_quad_bwd(t, th, torch.as_tensor(y, device="cuda"), n_bad=bad)
    g = grad.cpu().numpy().astype(np.float64)
    assert int(bad.item()) == 0 and np.all(np.isfinite(g))
    idx = np.random.default_rng(4).choice(4096, 64, replace=False)
    rows = _theta_rows(wl["theta"], idx)
    ssr_r, grad_r = oracle.ssr_grad(wl["t"], rows, y.astype(np.float64))
    tol = _bound(wl["t"], rows, y.astype(np.float64), None, 1, 0.0)
    err = np.abs(g[idx] - grad_r)
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    assert np.all(err <= tol), (worst, g[idx][worst], grad_r[worst], tol[worst])
    assert np.allclose(ssr.cpu().numpy()[idx], ssr_r, rtol=2e-4)
