"""No kernel reads work-buffer bytes that the call did not write first: the
list paths (Mandel-Agol, Gimenez, Gimenez interpolated in z) and the adjoint,
run once with a work buffer of zero bytes and once with one of 0xff bytes
(NaN as floats, -1 as integers), give bitwise the same results.  This covers
the Chebyshev coefficient rows' padding orders as well as every list,
counter, prefix and table region."""
import numpy as np
import pytest

from paper_1504_07433_gb300 import workloads as W
from tests.helpers import gpu_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


def _filled(torch, n, byte):
    return torch.full((max(int(n), 256),), byte, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("N,n_j", [(8, 64), (7, 33), (2, 40)])
def test_list_paths_read_only_what_they_write(torch_cuda, N, n_j):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.long_cadence(n_v=20, n_t=2000, n_gim=N)
    t, orb, k, ld = gpu_inputs(wl)
    ldg = torch.as_tensor(np.asarray(wl["ld_gim"], np.float32), device="cuda")
    n_v, n_t = k.numel(), t.numel()
    y = torch.ones((1, n_t), dtype=torch.float32, device="cuda")
    plan = pt.GimenezPlan(N, n_j)
    out = {}
    for byte in (0, 255):
        wm = _filled(torch, pt.ma_quad_work_bytes(n_t, n_v, 1), byte)
        wg = _filled(torch, plan.work_bytes(n_t, n_v, 1), byte)
        nz = pt.load_library().pt_gimenez_zi_work_bytes(plan.handle, 64, 64, n_t, n_v, 1, 0)
        fm, sm = pt.ma_quad(t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], y=y, want_ssr=True, work=wm)
        fg, sg = pt.gimenez(plan, t, orb, k, ldg, n_ss=wl["n_ss"], t_exp=wl["t_exp"], y=y, want_ssr=True, work=wg)
        wz = _filled(torch, nz, byte)
        fz, _ = pt.gimenez_zi(plan, t, orb, k, ldg, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=wz)
        torch.cuda.synchronize()
        out[byte] = [x.clone() for x in (fm, sm, fg, sg, fz)]
    for a, b in zip(out[0], out[255]):
        assert torch.equal(a, b)
    assert torch.isfinite(out[255][2]).all() and (out[255][2] < 1).any()
    plan.close()


def test_adjoint_reads_only_what_it_writes(torch_cuda):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.adjoint(n_v=16, n_t=1500)
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device="cuda")
    th = pt.theta_to_device(wl["theta"])
    y = torch.ones(t.numel(), dtype=torch.float32, device="cuda")
    lib = pt.load_library()
    out = {}
    for byte in (0, 255):
        work = _filled(torch, lib.pt_ma_quad_bwd_work_bytes(t.numel()), byte)
        ssr, grad, flux = pt.ma_quad_bwd(t, th, y, want_flux=True, work=work)
        torch.cuda.synchronize()
        out[byte] = (ssr.clone(), grad.clone(), flux.clone())
    for a, b in zip(out[0], out[255]):
        assert torch.equal(a, b)
    assert torch.isfinite(out[255][1]).all()
