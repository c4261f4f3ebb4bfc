"""GPU parity of the Gimenez path (pt_gimenez_alpha, pt_gimenez) against the
FP64 oracle at the same series depth n_j, through the C ABI.

Tolerance: 1e-6 absolute flux (the exact-path bound), alpha_n to 5e-7.
The truncation error against the exact flux is a separate, reported
property (Fig. 1 behaviour), checked here only as MA-Gimenez agreement.
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


@pytest.mark.parametrize("n_j", [16, 64, 160])
def test_gimenez_alpha_vs_oracle(torch_cuda, n_j):
    torch = torch_cuda
    import paper_1504_07433_gb300 as pt
    plan = pt.GimenezPlan(8, n_j)
    rng = np.random.default_rng(n_j)
    k = rng.uniform(0.01, 0.3, 400).astype(np.float32)
    z = (rng.uniform(0, 1.05, k.size) * (1 + k)).astype(np.float32)
    z[:8] = 0.0
    z[8:16] = (1 - k[8:16])
    a = pt.gimenez_alpha(plan, torch.as_tensor(k, device="cuda"), torch.as_tensor(z, device="cuda")).cpu().numpy()
    ref = np.array([oracle.gimenez_alpha(8, n_j, float(kk), float(zz)) for kk, zz in zip(k, z)])
    assert np.max(np.abs(a - ref)) <= 5e-7
    # physical 8-term laws: a quadratic law in general form plus small higher terms
    q1, q2 = rng.uniform(0, 1, k.size), rng.uniform(0, 1, k.size)
    u = np.zeros((k.size, 8))
    u[:, :2] = W.quad_to_general(*W.q_to_u(q1, q2), 2)
    u[:, 2:] = rng.uniform(-0.02, 0.02, (k.size, 6))
    D = 1 - np.sum(np.arange(1, 9) * u / (np.arange(1, 9) + 2), axis=1)
    C = np.concatenate([(1 - u.sum(1))[:, None], u], axis=1) / D[:, None]
    assert np.max(np.abs(np.sum(C * (a - ref), axis=1))) <= TOL


def _oracle_lc(wl, n_j):
    return oracle.lc_gimenez(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld_gim"]), n_j,
                             n_ss=wl["n_ss"], t_exp=wl["t_exp"])[0]


@pytest.mark.parametrize("n_t,n_v,n_ss,n_j", [(1500, 5, 10, 128), (700, 3, 1, 64), (301, 2, 3, 40)])
def test_gimenez_lc_vs_oracle(torch_cuda, n_t, n_v, n_ss, n_j):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=n_v, n_t=n_t, n_ss=n_ss, cadence=0.01)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, n_j)
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"], n_bad=bad)
    f = flux.cpu().numpy().astype(np.float64)
    ref = _oracle_lc(wl, n_j)
    assert int(bad.item()) == 0
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(f - ref)) <= TOL



@pytest.mark.parametrize("N,n_ss", [(1, 4), (3, 7), (16, 2), (8, 20), (4, 25)])
def test_gimenez_lc_series_orders(torch_cuda, N, n_ss):
    """Odd and even N, the largest N, supersample counts that leave the last
    round of the evaluation partly filled, and supersample lists longer than
    one batch of 16 (n_ss = 20, 25)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=3, n_t=900, n_ss=n_ss, cadence=0.01)
    rng = np.random.default_rng(100 + N)
    u = np.zeros((3, 1, N))
    u[..., 0] = rng.uniform(0.3, 0.6, (3, 1))
    if N > 1:
        u[..., 1] = rng.uniform(0.0, 0.2, (3, 1))
    if N > 2:
        u[..., 2:] = rng.uniform(-0.02, 0.02, (3, 1, N - 2))
    wl["ld"] = wl["ld_gim"] = u
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(N, 64)
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"])
    f = flux.cpu().numpy().astype(np.float64)
    ref = _oracle_lc(wl, 64)
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(f - ref)) <= TOL

@pytest.mark.parametrize("N,n_j,n_ss,n_t", [(16, 512, 40, 900), (1, 2, 3, 900)])
def test_gimenez_extreme_plans(torch_cuda, N, n_j, n_ss, n_t):
    """The largest plan (N = 16, n_j = 512: coefficient rows and round buffers
    past the default 48 KB of shared memory) with three supersample batches,
    and the smallest series (n_j = 2: no recurrence step at all)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=2, n_t=n_t, n_ss=n_ss, cadence=0.01)
    rng = np.random.default_rng(7 + N)
    u = np.zeros((2, 1, N))
    u[..., 0] = rng.uniform(0.3, 0.6, (2, 1))
    if N > 1:
        u[..., 1] = rng.uniform(0.0, 0.2, (2, 1))
    if N > 2:
        u[..., 2:] = rng.uniform(-0.01, 0.01, (2, 1, N - 2))
    wl["ld"] = wl["ld_gim"] = u
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(N, n_j)
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"])
    f = flux.cpu().numpy().astype(np.float64)
    ref = _oracle_lc(wl, n_j)
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(f - ref)) <= TOL


def test_gimenez_ssr_and_multiband(torch_cuda):
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.batched(n_walkers=3, n_pb=4, n_lc=2, len_lo=200, len_hi=400)
    rng = np.random.default_rng(2)
    u = np.concatenate([W.quad_to_general(wl["ld"][..., 0], wl["ld"][..., 1], 2),
                        rng.uniform(-0.02, 0.02, wl["ld"].shape[:2] + (2,))], axis=-1)
    wl["ld"] = u
    wl["k"] = wl["k"][:, 0]
    plan = pt.GimenezPlan(4, 96)
    t, orb, k, ld = gpu_inputs(wl)
    y = torch.as_tensor(wl["y"], dtype=torch.float32, device="cuda")
    flux, ssr = pt.gimenez(plan, t, orb, k, ld, y=y, want_ssr=True)
    f = flux.cpu().numpy().astype(np.float64)
    ref = oracle.lc_gimenez(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(u), 96)[0]
    assert np.max(np.abs(f - ref)) <= TOL
    yy = np.asarray(wl["y"], np.float32).astype(np.float64)
    assert np.allclose(ssr.cpu().numpy(), np.sum((yy[None] - f) ** 2, axis=2), rtol=2e-5)


def test_gimenez_agrees_with_ma_for_quadratic_ld(torch_cuda):
    """Same physics: with u_1 = a + 2b, u_2 = -b (Sec. 2.1.2) the two GPU
    models agree to the series truncation error (n_j = 300 here)."""
    import paper_1504_07433_gb300 as pt
    wl = W.long_cadence(n_v=8, n_t=3000, n_ss=1, cadence=0.005)
    t, orb, k, ld = gpu_inputs(wl)
    fm, _ = pt.ma_quad(t, orb, k, ld)
    import torch
    ldg = torch.as_tensor(W.quad_to_general(wl["ld"][..., 0], wl["ld"][..., 1], 2), dtype=torch.float32,
                          device="cuda")
    fg, _ = pt.gimenez(pt.GimenezPlan(2, 300), t, orb, k, ldg)
    assert torch.max(torch.abs(fm - fg)).item() < 5e-6


def test_gimenez_full_long_cadence_sampled(torch_cuda):
    """Full 50,000 x 256 x 10 workload with N = 8, n_j = 128 in the
    benchmark's launch configuration; sampled outputs against the oracle."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence()
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 128)
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    f = flux.cpu().numpy()
    assert np.all(f <= 1.0 + 1e-6) and np.all(f > 0.9)
    rng = np.random.default_rng(22)
    for v in rng.choice(256, 12, replace=False):
        row = f[v, 0]
        intr = np.nonzero(row < 1.0)[0]
        pick = np.concatenate([rng.choice(intr, min(40, intr.size), replace=False),
                               rng.choice(row.size, 10, replace=False)])
        sub = dict(t=wl["t"][pick], orbit={kk: (None if vv is None else np.asarray(vv)[[v]])
                                          for kk, vv in wl["orbit"].items()},
                   k=wl["k"][[v]], ld_gim=wl["ld_gim"][[v]], n_ss=wl["n_ss"], t_exp=wl["t_exp"])
        ref = _oracle_lc(sub, 128)
        assert np.max(np.abs(row[pick].astype(np.float64) - ref[0, 0])) <= TOL, v


@pytest.mark.parametrize("order", ["shuffled", "partly_reversed"])
def test_time_order_does_not_matter(torch_cuda, order):
    """The window kernel searches sorted tiles by epoch and tests every pair
    of unsorted ones; both give the oracle's light curves (MA and Gimenez)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=4, n_t=2000, n_ss=3, cadence=0.01)
    rng = np.random.default_rng(21)
    if order == "shuffled":
        perm = rng.permutation(wl["t"].size)
    else:   # sorted tiles, one reversed stretch, and a tile mixing both
        perm = np.arange(wl["t"].size)
        perm[700:1300] = perm[700:1300][::-1]
    wl["t"] = wl["t"][perm]
    wl_g = dict(wl, ld=wl["ld_gim"])
    t, orb, k, ld = gpu_inputs(wl)
    ldg = torch.as_tensor(np.asarray(wl["ld_gim"], np.float32), device="cuda")
    fm, _ = pt.ma_quad(t, orb, k, ld, n_ss=3, t_exp=wl["t_exp"])
    plan = pt.GimenezPlan(8, 64)
    fg, _ = pt.gimenez(plan, t, orb, k, ldg, n_ss=3, t_exp=wl["t_exp"])
    ref_m = oracle.lc_ma(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]), n_ss=3,
                         t_exp=wl["t_exp"])[0]
    ref_g = _oracle_lc(wl_g, 64)
    assert (ref_m < 1).sum() > 0
    assert np.max(np.abs(fm.cpu().numpy() - ref_m)) <= TOL
    assert np.max(np.abs(fg.cpu().numpy() - ref_g)) <= TOL


@pytest.mark.parametrize("k_scale", [0.3, 0.45])
def test_gimenez_large_radius_ratio(torch_cuda, k_scale):
    """Radius ratios beyond the long-cadence prior (where the series values
    and their Chebyshev coefficients are largest relative to the result)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=4, n_t=1200, n_ss=5, cadence=0.01)
    wl["k"] = np.full(4, k_scale) * np.array([0.9, 0.95, 1.0, 1.05])
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 128)
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=5, t_exp=wl["t_exp"])
    ref = _oracle_lc(wl, 128)
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(flux.cpu().numpy() - ref)) <= TOL


@pytest.mark.parametrize("N,n_j", [(8, 97), (8, 98), (5, 33)])
def test_gimenez_series_depths(torch_cuda, N, n_j):
    """Series depths that are odd (the middle Chebyshev node pairs with
    itself in the transform) or not a multiple of four (scalar copies of the
    cosine table)."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=3, n_t=1000, n_ss=4, cadence=0.01, n_gim=N)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(N, n_j)
    flux, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=4, t_exp=wl["t_exp"])
    ref = _oracle_lc(wl, n_j)
    assert (ref < 1).sum() > 0
    assert np.max(np.abs(flux.cpu().numpy() - ref)) <= TOL


def test_evaluation_timing_events(torch_cuda):
    """pt_gim_plan_time_evaluation records the caller's events around the
    series-evaluation kernel only: inside the call's own time, results
    unchanged, and switched off again by passing no events."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=16, n_t=20000)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 128)
    f0, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.time_evaluation(e0, e1)
    c0.record()
    f1, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    c1.record()
    torch.cuda.synchronize()
    kernel_ms, call_ms = e0.elapsed_time(e1), c0.elapsed_time(c1)
    assert 0.0 < kernel_ms < call_ms
    assert torch.equal(f0, f1)
    plan.time_evaluation()
    f2, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    assert torch.equal(f0, f2)
    with pytest.raises(pt.PTError):
        plan.time_evaluation(e0, None)


def test_graph_capture_and_workspace_reuse(torch_cuda):
    """A call captured into a CUDA graph and replayed, and back-to-back calls
    with two radius-ratio sets that reuse one workspace on a non-default
    stream, give the flux of a plain call, which matches the oracle."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=6, n_t=3000)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 96)
    n_v, n_t = k.numel(), t.numel()
    work = torch.empty(plan.work_bytes(n_t, n_v, 1), dtype=torch.uint8, device="cuda")
    f0, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work)
    torch.cuda.synchronize()
    ref = _oracle_lc(wl, 96)
    assert np.max(np.abs(f0.cpu().numpy() - ref)) <= TOL
    # two radius-ratio sets through one workspace, back to back on another stream
    k2 = (k * 1.05).contiguous()
    s = torch.cuda.Stream()
    fa = torch.empty_like(f0)
    fb = torch.empty_like(f0)
    with torch.cuda.stream(s):
        for _ in range(3):
            pt.gimenez(plan, t, orb, k2, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=fa)
            pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=fb)
    torch.cuda.synchronize()
    assert torch.equal(fb, f0)
    fa_ref, _ = pt.gimenez(plan, t, orb, k2, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
    torch.cuda.synchronize()
    assert torch.equal(fa, fa_ref)
    # captured into a graph and replayed
    fg = torch.empty_like(f0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=fg)
    torch.cuda.synchronize()
    fg.zero_()
    with torch.cuda.graph(g, stream=s):
        pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=fg)
    fg.zero_()
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(fg, f0)
    plan.close()


def test_plan_shared_by_host_threads(torch_cuda):
    """Two host threads share one plan, each with its own stream and work
    buffer and its own radius ratios, calls interleaved: the plan forks the
    table and coefficient work of every call onto its own stream, and each
    call still gives bitwise the flux of a call made alone."""
    import threading
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=12, n_t=4000)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 64)
    n_v, n_t = k.numel(), t.numel()
    ks = [k, (k * 1.07).contiguous()]
    refs = []
    for kk in ks:
        f, _ = pt.gimenez(plan, t, orb, kk, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"])
        torch.cuda.synchronize()
        refs.append(f.clone())
    outs = [[None] * 6 for _ in ks]
    errors = []

    def worker(i):
        try:
            s = torch.cuda.Stream()
            work = torch.empty(plan.work_bytes(n_t, n_v, 1), dtype=torch.uint8, device="cuda")
            with torch.cuda.stream(s):
                for r in range(6):
                    f = torch.empty_like(refs[i])
                    pt.gimenez(plan, t, orb, ks[i], ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=f)
                    outs[i][r] = f
            s.synchronize()
        except Exception as e:   # reported below: a thread's failure must fail the test
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(ks))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for i in range(len(ks)):
        for f in outs[i]:
            assert torch.equal(f, refs[i])
    plan.close()


def test_misaligned_workspace_rejected(torch_cuda):
    """A work buffer that does not start on a 16-byte boundary is refused
    (PT_ERR_WORKSPACE) before any kernel is launched."""
    import paper_1504_07433_gb300 as pt
    torch = torch_cuda
    wl = W.long_cadence(n_v=2, n_t=500)
    wl["ld"] = wl["ld_gim"]
    t, orb, k, ld = gpu_inputs(wl)
    plan = pt.GimenezPlan(8, 64)
    need = plan.work_bytes(t.numel(), 2, 1)
    raw = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(pt.PTError):
        pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=raw[4:])
    f, _ = pt.gimenez(plan, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=raw[16:])
    torch.cuda.synchronize()
    assert torch.isfinite(f).all()
    plan.close()
