"""Surrogate network: GPU training kernels against the FP64 oracle network,
the BF16 tensor-core serving path against the FP32 network, and the served
surrogate (with its exact fallback) against the FP64 oracle flux."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300.surrogate as S
    S.lib()
    return torch, S


def _rand_params(S, seed, scale=1.0):
    p = S.init_params(seed).cpu().numpy().astype(np.float64) * scale
    rng = np.random.default_rng(seed + 100)
    p[S._OFF["b1"]:S._OFF["W2"]] = rng.normal(0, 0.1, 128)
    p[S._OFF["b2"]:S._OFF["W3"]] = rng.normal(0, 0.1, 128)
    p[S._OFF["b3"]:S._OFF["W4"]] = rng.normal(0, 0.1, 128)
    p[S._OFF["b4"]:] = rng.normal(0, 0.1, 2)
    return p.astype(np.float32)


def test_mlp_forward_and_loss_grad_vs_oracle(env):
    torch, S = env
    p32 = _rand_params(S, 3)
    rng = np.random.default_rng(4)
    n = 700                                   # ragged against the 64-row tiles and the 512-row split
    X = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    T = rng.normal(0, 1, (n, 2)).astype(np.float32)
    pd = p32.astype(np.float64)
    Xd, Td = X.astype(np.float64), T.astype(np.float64)
    Pt = torch.as_tensor(p32, device="cuda")
    Xt, Tt = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    Y = S.forward_f32(Pt, Xt).cpu().numpy()
    Yr = oracle.mlp_forward(pd, Xd)
    assert np.max(np.abs(Y - Yr)) <= 1e-5 * max(1.0, np.max(np.abs(Yr)))
    tr = S.Trainer(Pt.clone(), batch=1024)
    loss, g = tr.loss_grad(Xt, Tt)
    loss_r, g_r = oracle.mlp_loss_grad(pd, Xd, Td)
    assert float(loss.item()) == pytest.approx(loss_r, rel=1e-5)
    g = g.cpu().numpy().astype(np.float64)
    err = np.abs(g - g_r)
    assert np.all(err <= 1e-4 * np.max(np.abs(g_r)) + 1e-3 * np.abs(g_r)), np.argmax(err)


def test_adam_step(env):
    torch, S = env
    rng = np.random.default_rng(5)
    p = rng.normal(0, 1, S.N_PARAMS).astype(np.float32)
    g = rng.normal(0, 1, S.N_PARAMS).astype(np.float32)
    tr = S.Trainer(torch.as_tensor(p, device="cuda"), batch=64)
    tr.g.copy_(torch.as_tensor(g))
    tr.step_no = 0
    L = S.lib()
    for step in (1, 2):
        tr.step_no += 1
        from paper_1504_07433_gb300 import _ptr, _stream
        L.pt_mlp_adam(_ptr(tr.p), _ptr(tr.g), _ptr(tr.m), _ptr(tr.v), tr.step_no, 1e-3, 0.9, 0.999, 1e-8, _stream())
    m = np.zeros_like(p, dtype=np.float64)
    v = np.zeros_like(m)
    q = p.astype(np.float64)
    for step in (1, 2):
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g.astype(np.float64) ** 2
        q -= 1e-3 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    assert np.allclose(tr.p.cpu().numpy(), q, rtol=1e-5, atol=1e-6)


def test_datagen_targets_are_exact_terms(env):
    torch, S = env
    X, T, kz = S.datagen(5000, seed=11, with_kz=True)
    kz = kz.cpu().numpy().astype(np.float64)
    X, T = X.cpu().numpy(), T.cpu().numpy()
    k, z = kz[:, 0], kz[:, 1]
    assert np.all((k >= S.K_LO) & (k <= S.K_HI))
    s = (1 - np.cos((X[:, 1] + 1) * np.pi / 2)) / 2       # inverse of the band coordinate
    assert np.allclose(z, np.abs(1 - k) + 2 * k * s, atol=2e-6)
    ref = np.array([oracle.ma_terms(kk, zz) for kk, zz in zip(k, z)])
    ld = ref[:, 1] + np.where(k > z, 2 / 3, 0.0)
    ed = ref[:, 2]
    n = S.NORM
    t0 = (ld / k ** 2 - n[2]) / n[3]
    t1 = (ed / k ** 2 - n[4]) / n[5]
    tol = 2e-6 / (k ** 2 * min(n[3], n[5]))      # the exact FP32 kernel's 1e-6 flux-level error, normalised
    assert np.all(np.abs(T[:, 0] - t0) <= tol) and np.all(np.abs(T[:, 1] - t1) <= tol)
    # a disjoint offset gives a different, reproducible stream
    X2, _, _ = S.datagen(5000, seed=11, offset=5000)
    X3, _, _ = S.datagen(5000, seed=11, offset=5000)
    assert torch.equal(X2, X3) and not np.allclose(X2.cpu().numpy(), X)


def test_tensor_core_network_matches_fp32(env):
    """tcgen05 BF16 layers against the FP32 network run with the same BF16
    operand rounding: agreement to the rounding noise, not to garbage."""
    torch, S = env
    p = torch.as_tensor(_rand_params(S, 9), device="cuda")
    rng = np.random.default_rng(10)
    X = torch.as_tensor(rng.uniform(-1, 1, (1000, 2)).astype(np.float32), device="cuda")   # 8 tiles, ragged
    model = S.SurrogateModel(p)
    Y_tc = model.network(X)
    torch.cuda.synchronize()
    assert not model.timed_out()
    Y_ref = S.forward_f32(p, X, qat=True)
    Y_f32 = S.forward_f32(p, X, qat=False)
    d_tc = torch.max(torch.abs(Y_tc - Y_ref)).item()
    d_q = torch.max(torch.abs(Y_f32 - Y_ref)).item()
    scale = torch.max(torch.abs(Y_ref)).item()
    assert scale > 0.05
    # the tensor-core result differs from the rounded FP32 network by at most
    # the size of the rounding effect itself (same operands, other summation
    # order, tanh-based SiLU before rounding)
    assert d_tc <= max(2.0 * d_q, 1e-3 * scale), (d_tc, d_q, scale)


def test_surrogate_trained_small_with_fallback(env):
    """A short training run, the error-bound table, and the served terms:
    every point's flux error against the FP64 oracle stays within 1e-5 for
    quadratic laws with q1, q2 in [0, 1] (network where the table allows it,
    exact kernel elsewhere)."""
    torch, S = env
    X, T, _ = S.datagen(2_000_000, seed=21)
    tr = S.Trainer(S.init_params(0), batch=16384)
    tr.fit(X, T, epochs=8, lr0=3e-3, lr1=3e-5, qat_epochs=2)
    table, cm = S.build_table(tr.p, nk=32, ns=32, n_val=1_000_000)
    model = S.SurrogateModel(tr.p, table)
    k, z = S.validation_points(20000, seed=99)
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    le, ld, ed = model.terms(k, z, nfb)
    torch.cuda.synchronize()
    assert not model.timed_out()
    kk, zz = k.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64)
    le, ld, ed = (x.cpu().numpy().astype(np.float64) for x in (le, ld, ed))
    worst = 0.0
    for q1, q2 in [(0.1, 0.1), (0.5, 0.5), (1.0, 0.0), (1.0, 1.0), (0.3, 0.9)]:
        u1, u2 = 2 * np.sqrt(q1) * q2, np.sqrt(q1) * (1 - 2 * q2)
        c = u1 + 2 * u2
        D = 1 - u1 / 3 - u2 / 6
        f = 1 - ((1 - c) * le + c * ld + u2 * ed) / D
        ref = oracle.flux_quad_vec(kk, zz, u1, u2)
        worst = max(worst, float(np.max(np.abs(f - ref))))
    used = 1.0 - int(nfb.item()) / kk.size
    print("small surrogate: network share %.3f, cells exact %.3f, worst flux error %.2e"
          % (used, table.mean(), worst))
    assert worst <= 1e-5
    assert table.mean() < 1.0     # the network serves part of the band
