"""The Gimenez list paths hand out work items in a cost order (geometries
sorted by the estimated in-transit share of their listed pairs; the
Mandel-Agol path keeps the index order).  The order decides only which CTA
evaluates which pair, never the arithmetic of a pair, so a call with many
geometries (per-passband radius ratios) must give bitwise the flux of the
same geometries evaluated passband by passband.  The sizes take the three
ordering paths: a rank count (up to 1,024 geometries), a bitonic sort (up to
4,096) and the index order (above).
"""
import numpy as np
import pytest

from paper_1504_07433_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    pt.load_library()
    return torch


@pytest.mark.parametrize("n_v,n_b", [(8, 4), (40, 32), (140, 32)])
def test_item_order_bitwise_per_band(torch_cuda, n_v, n_b):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    wl = W.long_cadence(n_v=n_v, n_t=400, n_ss=4, cadence=0.01)
    rng = np.random.default_rng(n_v * 100 + n_b)
    k = (wl["k"][:, None] * (1.0 + rng.uniform(-0.05, 0.05, (n_v, n_b)))).astype(np.float32)
    ld = np.repeat(np.asarray(wl["ld"], np.float32), n_b, axis=1)
    ldg = np.repeat(np.asarray(wl["ld_gim"], np.float32), n_b, axis=1)
    dev = "cuda"
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device=dev)
    orb = pt.orbit_to_device(wl["orbit"], dev)
    plan = pt.GimenezPlan(8, 48)
    kt = torch.as_tensor(k, device=dev)
    fm, _ = pt.ma_quad(t, orb, kt, torch.as_tensor(ld, device=dev), n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    fg, _ = pt.gimenez(plan, t, orb, kt, torch.as_tensor(ldg, device=dev), n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    fm = fm.cpu().numpy()
    fg = fg.cpu().numpy()
    assert (fm < 1).sum() > 0 and (fg < 1).sum() > 0
    for b in range(n_b):
        kb = torch.as_tensor(np.ascontiguousarray(k[:, b]), device=dev)
        mb, _ = pt.ma_quad(t, orb, kb, torch.as_tensor(ld[:, b:b + 1].copy(), device=dev), n_ss=wl["n_ss"],
                           t_exp=wl["t_exp"])
        gb, _ = pt.gimenez(plan, t, orb, kb, torch.as_tensor(ldg[:, b:b + 1].copy(), device=dev), n_ss=wl["n_ss"],
                           t_exp=wl["t_exp"])
        assert np.array_equal(fm[:, b], mb.cpu().numpy()[:, 0]), b
        assert np.array_equal(fg[:, b], gb.cpu().numpy()[:, 0]), b
