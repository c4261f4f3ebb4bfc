"""pt_ma_quad_noalloc: the allocation-free variant of pt_ma_quad.

Callers that cannot allocate device memory (their device memory belongs to
a fixed pool of their own, or their sampling loop must not stall on an
allocation) use this entry point; it takes its scratch from a static device
array inside the library.  These tests call it through the C ABI and check
it against pt_ma_quad (caller-provided work buffer) on two different calls
in a row, so that anything a call failed to overwrite in the shared scratch
would show up in the second one, and both calls against the FP64 oracle
directly (its tile kernel is reached by no other exact-model entry point).

This file is collected last on purpose; it also runs alone in a fresh
process (the first call on the device performs the scratch look-up).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1504_07433_gb300 import workloads as W
from tests.helpers import f32, gpu_inputs, oracle_orbit

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the exact-path flux tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1504_07433_gb300 as pt
    lib = pt.load_library()
    fn = lib.pt_ma_quad_noalloc
    fn.restype = ctypes.c_int
    P = ctypes.c_void_p
    fn.argtypes = [P, ctypes.c_int, ctypes.POINTER(pt.Orbit), P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_int, P, P, P, P, P, P]
    return torch, pt, fn


def _call_noalloc(torch, pt, fn, t, orb, k, ld, n_ss, t_exp, y=None, wt=None, want_ssr=False):
    o = pt.Orbit(*(ctypes.c_void_p(orb[key].data_ptr()) if orb.get(key) is not None else None
                   for key in ("t0", "P", "a", "inc", "e", "w")), orb["t0"].numel())
    n_v, n_b, n_t = orb["t0"].numel(), ld.shape[1], t.numel()
    flux = torch.empty((n_v, n_b, n_t), dtype=torch.float32, device="cuda")
    ssr = torch.empty((n_v, n_b), dtype=torch.float32, device="cuda") if want_ssr else None
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    ptr = lambda x: None if x is None else ctypes.c_void_p(x.data_ptr())
    st = fn(ptr(t), n_t, ctypes.byref(o), ptr(k), 1 if k.dim() == 2 else 0, ptr(ld), n_b, n_ss, float(t_exp), 16,
            ptr(y), ptr(wt), ptr(flux), ptr(ssr), ptr(bad), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, pt.load_library().pt_last_error_string()
    torch.cuda.synchronize()
    assert int(bad.item()) == 0
    return flux, ssr


def test_noalloc_matches_work_buffer_entry_point_twice(env):
    torch, pt, fn = env
    # call 1: eccentric, supersampled, 2 passbands with SSR
    wl = W.long_cadence(n_v=40, n_t=6000, n_ss=10, cadence=0.01)
    wl["ld"] = np.concatenate([wl["ld"], wl["ld"][:, :, ::-1]], axis=1)
    t, orb, k, ld = gpu_inputs(wl)
    y = torch.ones((2, t.numel()), dtype=torch.float32, device="cuda")
    f_na, s_na = _call_noalloc(torch, pt, fn, t, orb, k, ld, 10, wl["t_exp"], y=y, want_ssr=True)
    f_ref, s_ref = pt.ma_quad(t, orb, k, ld, n_ss=10, t_exp=wl["t_exp"], y=y, want_ssr=True)
    assert (f_ref < 1).sum().item() > 0
    assert torch.max(torch.abs(f_na - f_ref)).item() <= TOL
    # the residual sums agree to what the flux tolerance implies:
    # |sum (y - f1)^2 - sum (y - f2)^2| <= sum (2 |y - f| TOL + TOL^2)
    bound = (2.0 * TOL * torch.abs(y[None] - f_ref).double().sum(dim=2) + t.numel() * TOL ** 2)
    assert torch.all(torch.abs(s_na.double() - s_ref.double()) <= bound)
    ref = oracle.lc_ma(wl["t"], oracle_orbit(wl["orbit"]), f32(wl["k"]), f32(wl["ld"]), n_ss=10,
                       t_exp=wl["t_exp"])[0]
    assert np.max(np.abs(f_na.cpu().numpy().astype(np.float64) - ref)) <= TOL
    # call 2, straight after: a different, smaller circular problem with per-band k
    wl2 = W.batched(n_walkers=7, n_pb=3, n_lc=2, len_lo=300, len_hi=600)
    t2, orb2, k2, ld2 = gpu_inputs(wl2)
    f_na2, _ = _call_noalloc(torch, pt, fn, t2, orb2, k2, ld2, 1, 0.0)
    f_ref2, _ = pt.ma_quad(t2, orb2, k2, ld2)
    assert (f_ref2 < 1).sum().item() > 0
    assert torch.max(torch.abs(f_na2 - f_ref2)).item() <= TOL
    ref2 = oracle.lc_ma(wl2["t"], oracle_orbit(wl2["orbit"]), f32(wl2["k"]), f32(wl2["ld"]))[0]
    assert np.max(np.abs(f_na2.cpu().numpy().astype(np.float64) - ref2)) <= TOL


def test_noalloc_rejects_problems_beyond_its_scratch(env):
    torch, pt, fn = env
    lib = pt.load_library()
    n_t = 2_000_000   # 16 MB of time split alone, beyond the 4 MiB scratch
    o = pt.Orbit(8, 8, 8, 8, None, None, 4)
    st = fn(ctypes.c_void_p(8), n_t, ctypes.byref(o), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1, 1, 0.0, 16,
            None, None, ctypes.c_void_p(8), None, None, None)
    assert st == 5   # PT_ERR_WORKSPACE, detected on the host before any launch
    assert b"static scratch" in lib.pt_last_error_string()
