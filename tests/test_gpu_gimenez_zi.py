"""GPU parity of the Gimenez model interpolated in z (Sec. 3.3,
pt_gimenez_zi) against the FP64 oracle's own z tables, through the C ABI.

Tolerance 1e-6 in flux: the z nodes carry the FP32 series (~1e-7, as for
pt_gimenez) at FP32 node positions, and the interpolation is FP32.  The
interpolation error against the series itself is a property of the method,
checked at the paper's scale.
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


@pytest.mark.parametrize("n_t,n_v,n_ss,n_in,n_edge,N", [(1500, 5, 10, 64, 64, 8), (700, 3, 1, 16, 9, 8),
                                                         (401, 2, 3, 2, 1, 4), (900, 3, 25, 100, 40, 3)])
def test_gimenez_zi_vs_oracle(torch_cuda, n_t, n_v, n_ss, n_in, n_edge, N):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=n_v, n_t=n_t, n_ss=n_ss, cadence=0.01, n_gim=max(N, 2))
    wl["ld"] = wl["ld_gim"][:, :, :N]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(N, 64)
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    flux, _ = pt.gimenez_zi(plan, t, orb, k, ld, n_in=n_in, n_edge=n_edge, n_ss=n_ss, t_exp=wl["t_exp"], n_bad=bad)
    f = flux.cpu().numpy().astype(np.float64)
    ref = oracle.lc_gimenez_zi(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]), 64, n_in, n_edge,
                               n_ss=n_ss, t_exp=wl["t_exp"])[0]
    assert int(bad.item()) == 0
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(f - ref)) <= TOL


def test_gimenez_zi_multiband_ssr_and_error_scale(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=4, n_t=1200, n_ss=5, cadence=0.01)
    rng = np.random.default_rng(11)
    n_b = 3
    wl["k"] = wl["k"][:, None] * rng.uniform(0.95, 1.05, (4, n_b))
    wl["ld"] = np.repeat(wl["ld_gim"], n_b, axis=1)
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 96)
    flux, _ = pt.gimenez_zi(plan, t, orb, k, ld, n_ss=5, t_exp=wl["t_exp"])
    f = flux.cpu().numpy().astype(np.float64)
    ref = oracle.lc_gimenez_zi(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]), 96, 64, 64,
                               n_ss=5, t_exp=wl["t_exp"])[0]
    assert np.max(np.abs(f - ref)) <= TOL
    # residuals through the same path
    y = torch.as_tensor(rng.normal(1.0, 1e-3, (n_b, 1200)).astype(np.float32), device="cuda")
    _, ssr = pt.gimenez_zi(plan, t, orb, k, ld, n_ss=5, t_exp=wl["t_exp"], y=y, want_flux=False, want_ssr=True)
    yy = y.cpu().numpy().astype(np.float64)
    assert np.allclose(ssr.cpu().numpy(), np.sum((yy[None] - f) ** 2, axis=2), rtol=2e-5)
    # against the series itself: the paper's ~25 ppm scale at the default grid
    fs, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=5, t_exp=wl["t_exp"])
    err = np.max(np.abs(f - fs.cpu().numpy()))
    assert err < 3e-5


def test_gimenez_zi_argument_errors(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=1, n_t=10, n_ss=1, cadence=0.01)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 32)
    for n_in, n_edge in [(1, 4), (4, 0), (2000, 2000)]:
        with pytest.raises(pt.PTError):
            pt.gimenez_zi(plan, t, orb, k, ld, n_in=n_in, n_edge=n_edge)
