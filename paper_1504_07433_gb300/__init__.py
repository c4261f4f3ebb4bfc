"""GB300 (sm_103a) transit-model hot path: thin Python binding of ``include/pt.h``.

Every function here marshals arguments (torch CUDA tensors -> device
pointers, the current CUDA stream) and calls the C ABI of
``libpt_gb300.so``; all arithmetic runs in the library's CUDA kernels.  There
is no CPU fallback: if the library is missing or no GPU is visible the calls
raise.

Model: Parviainen (2015), PyTransit -- quadratic Mandel-Agol (Sec. 2.2) and
Gimenez (Sec. 2.1) transit fluxes over times x parameter vectors x passbands,
with exposure supersampling (Sec. 3.2), circular/eccentric orbits (Sec. 1) and
an optional on-device likelihood reduction (Sec. 3.4).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build_mod

__all__ = ["load_library", "Orbit", "Theta", "orbit_to_device", "z_circ", "z_ecc", "ma_terms", "ma_quad",
           "domain_check", "status_read",
           "MATable", "ma_terms_interp", "ma_quad_interp", "gimenez_zi",
           "ma_quad_work_bytes", "GimenezPlan", "gimenez", "gimenez_alpha", "ma_quad_bwd", "transit_ssr",
           "PTError", "Z_BEHIND"]

Z_BEHIND = 1.0e30

_c_void_p = ctypes.c_void_p
_c_int = ctypes.c_int
_c_size = ctypes.c_size_t
_c_double = ctypes.c_double


class PTError(RuntimeError):
    pass


class Orbit(ctypes.Structure):
    """Mirror of ``pt_orbit`` (device pointers)."""
    _fields_ = [("t0", _c_void_p), ("P", _c_void_p), ("a", _c_void_p), ("inc", _c_void_p),
                ("e", _c_void_p), ("w", _c_void_p), ("n_v", _c_int)]


class Theta(ctypes.Structure):
    """Mirror of ``pt_theta`` (device pointers)."""
    _fields_ = [("t0", _c_void_p), ("P", _c_void_p), ("a", _c_void_p), ("b", _c_void_p), ("e", _c_void_p),
                ("w", _c_void_p), ("k", _c_void_p), ("u1", _c_void_p), ("u2", _c_void_p), ("n_v", _c_int)]


THETA_NAMES = ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")

_LIB = None


def load_library(build_if_missing: bool = False):
    """Load libpt_gb300.so (raises if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build_mod.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build_mod.build()
        else:
            raise PTError("libpt_gb300.so is not built; run __graft_entry__.build() or "
                          "python -m paper_1504_07433_gb300.build")
    lib = ctypes.CDLL(path)
    P = _c_void_p
    sig = {
        "pt_version": (_c_int, []),
        "pt_status_string": (ctypes.c_char_p, [_c_int]),
        "pt_last_error_string": (ctypes.c_char_p, []),
        "pt_z_circ": (_c_int, [P, _c_int, ctypes.POINTER(Orbit), _c_int, _c_double, P, P]),
        "pt_z_ecc": (_c_int, [P, _c_int, ctypes.POINTER(Orbit), _c_int, _c_double, _c_int, _c_double, P, P, P]),
        "pt_ma_terms": (_c_int, [P, P, _c_size, P, P, P, P]),
        "pt_domain_check": (_c_int, [ctypes.POINTER(Orbit), P, _c_int, P, P]),
        "pt_status_read": (_c_int, [P, P, P]),
        "pt_ma_quad_work_bytes": (_c_size, [_c_int, _c_int, _c_int, _c_int]),
        "pt_ma_quad": (_c_int, [P, _c_int, ctypes.POINTER(Orbit), P, _c_int, P, _c_int, _c_int, _c_double, _c_int,
                                P, P, P, P, P, _c_size, P, P]),
        "pt_ma_table_create": (_c_int, [ctypes.c_float, ctypes.c_float, _c_int, _c_int, ctypes.POINTER(_c_void_p)]),
        "pt_ma_table_destroy": (_c_int, [P]),
        "pt_ma_terms_interp": (_c_int, [P, P, P, _c_size, P, P, P, P]),
        "pt_ma_quad_interp": (_c_int, [P, P, _c_int, ctypes.POINTER(Orbit), P, _c_int, P, _c_int, _c_int,
                                       _c_double, _c_int, P, P, P, P, P, _c_size, P, P]),
        "pt_gim_plan_create": (_c_int, [_c_int, _c_int, ctypes.POINTER(_c_void_p)]),
        "pt_gim_plan_destroy": (_c_int, [P]),
        "pt_gim_plan_time_evaluation": (_c_int, [P, P, P]),
        "pt_gimenez_alpha": (_c_int, [P, P, P, _c_size, P, P]),
        "pt_gimenez_work_bytes": (_c_size, [P, _c_int, _c_int, _c_int, _c_int]),
        "pt_gimenez": (_c_int, [P, P, _c_int, ctypes.POINTER(Orbit), P, _c_int, P, _c_int, _c_int, _c_double,
                                _c_int, P, P, P, P, P, _c_size, P, P]),
        "pt_gimenez_zi_work_bytes": (_c_size, [P, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int]),
        "pt_gimenez_zi": (_c_int, [P, _c_int, _c_int, P, _c_int, ctypes.POINTER(Orbit), P, _c_int, P, _c_int,
                                   _c_int, _c_double, _c_int, P, P, P, P, P, _c_size, P, P]),
        "pt_ma_quad_bwd_work_bytes": (_c_size, [_c_int]),
        "pt_ma_quad_bwd": (_c_int, [P, _c_int, ctypes.POINTER(Theta), _c_int, _c_double, _c_int, P, P, P, P, P, P,
                                    _c_size, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, what):
    if status != 0:
        lib = load_library()
        raise PTError("%s failed: %s (%s)" % (what, lib.pt_status_string(status).decode(),
                                              lib.pt_last_error_string().decode()))


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return _c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    if x is None:
        return None
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise PTError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise PTError("expected a contiguous tensor")
    return _c_void_p(x.data_ptr())


def _dev(x, dtype, device):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(x, dtype=dtype, device=device).contiguous()


def orbit_to_device(orbit, device="cuda"):
    """Copy an orbit dict (t0, P, a, inc[, e, w]) to device tensors with the
    ABI's dtypes (t0, P FP64; the rest FP32)."""
    torch = _torch()
    out = dict(t0=_dev(orbit["t0"], torch.float64, device), P=_dev(orbit["P"], torch.float64, device),
               a=_dev(orbit["a"], torch.float32, device), inc=_dev(orbit["inc"], torch.float32, device))
    if orbit.get("e") is not None:
        out["e"] = _dev(orbit["e"], torch.float32, device)
        out["w"] = _dev(orbit["w"], torch.float32, device)
    else:
        out["e"] = None
        out["w"] = None
    return out


def _orbit_struct(orb):
    n_v = int(orb["t0"].numel())
    return Orbit(_ptr(orb["t0"]), _ptr(orb["P"]), _ptr(orb["a"]), _ptr(orb["inc"]),
                 _ptr(orb.get("e")), _ptr(orb.get("w")), n_v), n_v


def z_circ(t, orb, n_ss=1, t_exp=0.0):
    """z[v, i*n_ss + s] for a circular orbit (pt_z_circ)."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    z = torch.empty((n_v, t.numel() * n_ss), dtype=torch.float32, device=t.device)
    _check(lib.pt_z_circ(_ptr(t), t.numel(), ctypes.byref(o), n_ss, float(t_exp), _ptr(z), _stream()),
           "pt_z_circ")
    return z


def z_ecc(t, orb, n_ss=1, t_exp=0.0, max_iter=50, tol=1e-12):
    """z[v, i*n_ss + s] for an eccentric orbit with FP64 Newton (pt_z_ecc);
    returns (z, n_bad) with n_bad a device int tensor."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    z = torch.empty((n_v, t.numel() * n_ss), dtype=torch.float32, device=t.device)
    bad = torch.zeros(1, dtype=torch.int32, device=t.device)
    _check(lib.pt_z_ecc(_ptr(t), t.numel(), ctypes.byref(o), n_ss, float(t_exp), int(max_iter), float(tol),
                        _ptr(z), _ptr(bad), _stream()), "pt_z_ecc")
    return z, bad


def ma_terms(k, z):
    """(lambda_e, lambda_d + 2/3 Theta(k-z), eta_d) for (k, z) pairs (pt_ma_terms)."""
    torch = _torch()
    lib = load_library()
    k = k.contiguous()
    z = z.contiguous()
    le = torch.empty_like(z)
    ld = torch.empty_like(z)
    ed = torch.empty_like(z)
    _check(lib.pt_ma_terms(_ptr(k), _ptr(z), z.numel(), _ptr(le), _ptr(ld), _ptr(ed), _stream()), "pt_ma_terms")
    return le, ld, ed


def domain_check(orb, k, n_out=None):
    """pt_domain_check: count the parameter sets outside the model's domain
    into a device int (returned; pass n_out to accumulate into your own).
    k is [n_v] or [n_v, n_b]."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    if n_out is None:
        n_out = torch.zeros(1, dtype=torch.int32, device=orb["t0"].device)
    per_v = 1 if k.dim() == 1 else int(k.shape[1])
    _check(lib.pt_domain_check(ctypes.byref(o), _ptr(k.contiguous()), per_v, _ptr(n_out), _stream()),
           "pt_domain_check")
    return n_out


def status_read(n_bad=None, n_domain=None):
    """pt_status_read: synchronise the current stream and turn the device
    counters into a status; returns (status, message)."""
    lib = load_library()
    st = int(lib.pt_status_read(_ptr(n_bad), _ptr(n_domain), _stream()))
    return st, (lib.pt_last_error_string().decode() if st else "")


def ma_quad_work_bytes(n_t, n_v, n_b, k_per_band=False):
    return int(load_library().pt_ma_quad_work_bytes(n_t, n_v, n_b, int(bool(k_per_band))))


def _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, device, flux, ssr):
    torch = _torch()
    if want_flux and flux is None:
        flux = torch.empty((n_v, n_b, n_t), dtype=torch.float32, device=device)
    if want_ssr and ssr is None:
        ssr = torch.empty((n_v, n_b), dtype=torch.float32, device=device)
    return (flux if want_flux else None), (ssr if want_ssr else None)


def ma_quad(t, orb, k, ld, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None, want_flux=True, want_ssr=False,
            work=None, flux=None, ssr=None, n_bad=None):
    """Quadratic Mandel-Agol light curves (pt_ma_quad).

    t [n_t] float64; orb from orbit_to_device; k [n_v] or [n_v, n_b] float32;
    ld [n_v, n_b, 2] float32 (u1, u2).  Returns (flux [n_v, n_b, n_t] or None,
    ssr [n_v, n_b] or None)."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    n_b = int(ld.shape[1])
    kpb = 1 if k.dim() == 2 else 0
    n_t = t.numel()
    fl, ss = _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, t.device, flux, ssr)
    need = int(lib.pt_ma_quad_work_bytes(n_t, n_v, n_b, kpb))
    if work is None or work.numel() < need:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _check(lib.pt_ma_quad(_ptr(t), n_t, ctypes.byref(o), _ptr(k), kpb, _ptr(ld), n_b, int(n_ss), float(t_exp),
                          int(max_iter), _ptr(y), _ptr(wt), _ptr(fl), _ptr(ss), _ptr(work), work.numel(),
                          _ptr(n_bad), _stream()), "pt_ma_quad")
    return fl, ss


class MATable:
    """Interpolation table of the Mandel-Agol terms (Sec. 2.2.3;
    pt_ma_table_create): n_k radius ratios over [k_lo, k_hi] x n_z separations
    over [0, 1 + k_hi], read by bilinear interpolation."""

    def __init__(self, k_lo, k_hi, n_k=128, n_z=256):
        lib = load_library()
        h = _c_void_p()
        _check(lib.pt_ma_table_create(float(k_lo), float(k_hi), int(n_k), int(n_z), ctypes.byref(h)),
               "pt_ma_table_create")
        self.handle = h
        self.k_lo, self.k_hi, self.n_k, self.n_z = float(k_lo), float(k_hi), int(n_k), int(n_z)

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().pt_ma_table_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ma_terms_interp(table, k, z):
    """Interpolated (lambda_e, lambda_d + 2/3 Theta(k-z), eta_d) for (k, z)
    pairs (pt_ma_terms_interp)."""
    torch = _torch()
    lib = load_library()
    k = k.contiguous()
    z = z.contiguous()
    le = torch.empty_like(z)
    ld = torch.empty_like(z)
    ed = torch.empty_like(z)
    _check(lib.pt_ma_terms_interp(table.handle, _ptr(k), _ptr(z), z.numel(), _ptr(le), _ptr(ld), _ptr(ed),
                                  _stream()), "pt_ma_terms_interp")
    return le, ld, ed


def ma_quad_interp(table, t, orb, k, ld, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None, want_flux=True,
                   want_ssr=False, work=None, flux=None, ssr=None, n_bad=None):
    """ma_quad with the terms read from an MATable (pt_ma_quad_interp)."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    n_b = int(ld.shape[1])
    kpb = 1 if k.dim() == 2 else 0
    n_t = t.numel()
    fl, ss = _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, t.device, flux, ssr)
    need = int(lib.pt_ma_quad_work_bytes(n_t, n_v, n_b, kpb))
    if work is None or work.numel() < need:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _check(lib.pt_ma_quad_interp(table.handle, _ptr(t), n_t, ctypes.byref(o), _ptr(k), kpb, _ptr(ld), n_b,
                                 int(n_ss), float(t_exp), int(max_iter), _ptr(y), _ptr(wt), _ptr(fl), _ptr(ss),
                                 _ptr(work), work.numel(), _ptr(n_bad), _stream()), "pt_ma_quad_interp")
    return fl, ss


class GimenezPlan:
    """Tables of Sec. 2.1.4 (A_{n,j} and the Jacobi recursion) for N
    general-law coefficients and series depth n_j (pt_gim_plan_create)."""

    def __init__(self, N, n_j):
        lib = load_library()
        h = _c_void_p()
        _check(lib.pt_gim_plan_create(int(N), int(n_j), ctypes.byref(h)), "pt_gim_plan_create")
        self.handle = h
        self.N = int(N)
        self.n_j = int(n_j)

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().pt_gim_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def work_bytes(self, n_t, n_v, n_b, k_per_band=False):
        return int(load_library().pt_gimenez_work_bytes(self.handle, n_t, n_v, n_b, int(bool(k_per_band))))

    def time_evaluation(self, start=None, end=None):
        """Record the torch.cuda.Event pair start/end around the series
        evaluation kernel of later gimenez() calls with this plan
        (pt_gim_plan_time_evaluation); no arguments stops it."""
        h0 = h1 = None
        if start is not None or end is not None:
            if start is None or end is None:
                raise PTError("time_evaluation needs both events or neither")
            for e in (start, end):
                if not e.cuda_event:   # the CUDA event is created on its first record
                    e.record()
            h0, h1 = _c_void_p(start.cuda_event), _c_void_p(end.cuda_event)
        _check(load_library().pt_gim_plan_time_evaluation(self.handle, h0, h1), "pt_gim_plan_time_evaluation")
        self._timing_events = (start, end)   # kept alive while the plan records them


def gimenez_alpha(plan, k, z):
    """alpha_0..alpha_N for (k, z) pairs (pt_gimenez_alpha): [n, N+1]."""
    torch = _torch()
    lib = load_library()
    k = k.contiguous()
    z = z.contiguous()
    out = torch.empty((z.numel(), plan.N + 1), dtype=torch.float32, device=z.device)
    _check(lib.pt_gimenez_alpha(plan.handle, _ptr(k), _ptr(z), z.numel(), _ptr(out), _stream()),
           "pt_gimenez_alpha")
    return out


def gimenez(plan, t, orb, k, ld, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None, want_flux=True,
            want_ssr=False, work=None, flux=None, ssr=None, n_bad=None):
    """Gimenez light curves (pt_gimenez); ld [n_v, n_b, N] holds u_1..u_N."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    n_b = int(ld.shape[1])
    if int(ld.shape[2]) != plan.N:
        raise PTError("ld has %d coefficients, plan expects %d" % (int(ld.shape[2]), plan.N))
    kpb = 1 if k.dim() == 2 else 0
    n_t = t.numel()
    fl, ss = _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, t.device, flux, ssr)
    need = plan.work_bytes(n_t, n_v, n_b, kpb)
    if work is None or work.numel() < need:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _check(lib.pt_gimenez(plan.handle, _ptr(t), n_t, ctypes.byref(o), _ptr(k), kpb, _ptr(ld), n_b, int(n_ss),
                          float(t_exp), int(max_iter), _ptr(y), _ptr(wt), _ptr(fl), _ptr(ss), _ptr(work),
                          work.numel(), _ptr(n_bad), _stream()), "pt_gimenez")
    return fl, ss


def gimenez_zi(plan, t, orb, k, ld, n_in=64, n_edge=64, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None,
               want_flux=True, want_ssr=False, work=None, flux=None, ssr=None, n_bad=None):
    """Gimenez light curves interpolated in z (pt_gimenez_zi, Sec. 3.3):
    alpha_n on n_in nodes over [0, 1 - k] and n_edge over (1 - k, 1 + k]."""
    torch = _torch()
    lib = load_library()
    o, n_v = _orbit_struct(orb)
    n_b = int(ld.shape[1])
    if int(ld.shape[2]) != plan.N:
        raise PTError("ld has %d coefficients, plan expects %d" % (int(ld.shape[2]), plan.N))
    kpb = 1 if k.dim() == 2 else 0
    n_t = t.numel()
    fl, ss = _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, t.device, flux, ssr)
    need = int(lib.pt_gimenez_zi_work_bytes(plan.handle, int(n_in), int(n_edge), n_t, n_v, n_b, kpb))
    if work is None or work.numel() < need:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _check(lib.pt_gimenez_zi(plan.handle, int(n_in), int(n_edge), _ptr(t), n_t, ctypes.byref(o), _ptr(k), kpb,
                             _ptr(ld), n_b, int(n_ss), float(t_exp), int(max_iter), _ptr(y), _ptr(wt), _ptr(fl),
                             _ptr(ss), _ptr(work), work.numel(), _ptr(n_bad), _stream()), "pt_gimenez_zi")
    return fl, ss


def ma_quad_noalloc(t, orb, k, ld, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None, want_flux=True,
                    want_ssr=False, flux=None, ssr=None, n_bad=None):
    """pt_ma_quad_noalloc: pt_ma_quad with the library's static device scratch
    instead of a work buffer, for callers that cannot allocate device memory
    (the outputs are still the caller's; pass flux/ssr to avoid allocating
    them here).  Rejects problems whose scratch exceeds
    PT_MA_NOALLOC_SCRATCH_BYTES; overlapping calls on the GPU race."""
    lib = load_library()
    fn = lib.pt_ma_quad_noalloc
    fn.restype = _c_int
    P = _c_void_p
    fn.argtypes = [P, _c_int, ctypes.POINTER(Orbit), P, _c_int, P, _c_int, _c_int, _c_double, _c_int,
                   P, P, P, P, P, P]
    o, n_v = _orbit_struct(orb)
    n_b = int(ld.shape[1])
    kpb = 1 if k.dim() == 2 else 0
    n_t = t.numel()
    fl, ss = _lc_outputs(n_v, n_b, n_t, want_flux, want_ssr, t.device, flux, ssr)
    _check(fn(_ptr(t), n_t, ctypes.byref(o), _ptr(k), kpb, _ptr(ld), n_b, int(n_ss), float(t_exp), int(max_iter),
              _ptr(y), _ptr(wt), _ptr(fl), _ptr(ss), _ptr(n_bad), _stream()), "pt_ma_quad_noalloc")
    return fl, ss


def theta_to_device(theta, device="cuda"):
    """Parameter dict (t0, P, a, b, e, w, k, u1, u2) to device tensors (t0, P FP64; rest FP32)."""
    torch = _torch()
    out = {}
    for name in THETA_NAMES:
        x = theta.get(name)
        if x is None:
            out[name] = None
            continue
        out[name] = _dev(x, torch.float64 if name in ("t0", "P") else torch.float32, device)
    return out


def ma_quad_bwd(t, theta, y, wt=None, n_ss=1, t_exp=0.0, max_iter=16, want_flux=False, work=None, n_bad=None):
    """pt_ma_quad_bwd: (ssr [n_v], grad [n_v, 9], flux [n_v, n_t] or None) for the
    parameter tensors in theta (see theta_to_device)."""
    torch = _torch()
    lib = load_library()
    n_v = int(theta["t0"].numel())
    th = Theta(*(_ptr(theta.get(nm)) for nm in THETA_NAMES), n_v)
    n_t = t.numel()
    grad = torch.empty((n_v, 9), dtype=torch.float32, device=t.device)
    ssr = torch.empty(n_v, dtype=torch.float32, device=t.device)
    flux = torch.empty((n_v, n_t), dtype=torch.float32, device=t.device) if want_flux else None
    need = int(lib.pt_ma_quad_bwd_work_bytes(n_t))
    if work is None or work.numel() < need:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=t.device)
    _check(lib.pt_ma_quad_bwd(_ptr(t), n_t, ctypes.byref(th), int(n_ss), float(t_exp), int(max_iter), _ptr(y),
                              _ptr(wt), _ptr(grad), _ptr(ssr), _ptr(flux), _ptr(work), work.numel(), _ptr(n_bad),
                              _stream()), "pt_ma_quad_bwd")
    return ssr, grad, flux


def _make_ssr_function():
    torch = _torch()

    class _TransitSSR(torch.autograd.Function):
        """SSR of the quadratic MA light curve with the hand-written adjoint as
        its backward; the forward call already produces the gradient, which is
        the only thing kept for backward."""

        @staticmethod
        def forward(ctx, t, y, wt, n_ss, t_exp, t0, P, a, b, e, w, k, u1, u2):
            th = dict(t0=t0.detach().contiguous(), P=P.detach().contiguous(), a=a.detach().contiguous(),
                      b=b.detach().contiguous(), e=None if e is None else e.detach().contiguous(),
                      w=None if w is None else w.detach().contiguous(), k=k.detach().contiguous(),
                      u1=u1.detach().contiguous(), u2=u2.detach().contiguous())
            ssr, grad, _ = ma_quad_bwd(t, th, y, wt, n_ss=n_ss, t_exp=t_exp)
            ctx.save_for_backward(grad)
            ctx.has_e = e is not None
            return ssr

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            g = gout[:, None].to(grad.dtype) * grad
            cols = [g[:, i] for i in range(9)]
            cols[0] = cols[0].double()
            cols[1] = cols[1].double()
            if not ctx.has_e:
                cols[4] = None
                cols[5] = None
            return (None, None, None, None, None, *cols)

    return _TransitSSR


_SSR_FN = None


def transit_ssr(t, y, theta, wt=None, n_ss=1, t_exp=0.0):
    """Differentiable SSR [n_v] (torch.autograd): d/d theta comes from pt_ma_quad_bwd."""
    global _SSR_FN
    if _SSR_FN is None:
        _SSR_FN = _make_ssr_function()
    return _SSR_FN.apply(t, y, wt, int(n_ss), float(t_exp), *(theta.get(nm) for nm in THETA_NAMES))


class BatchDesc(ctypes.Structure):
    """Mirror of ``pt_batch_desc``."""
    _fields_ = [("t", _c_void_p), ("n_t", _c_int), ("lc_offsets", ctypes.POINTER(_c_int)), ("n_lc", _c_int),
                ("orb", Orbit), ("k", _c_void_p), ("ld", _c_void_p), ("n_b", _c_int), ("n_ss", _c_int),
                ("t_exp", _c_double), ("max_iter", _c_int), ("y", _c_void_p), ("wt", _c_void_p),
                ("flux", _c_void_p), ("ssr", _c_void_p), ("n_bad", _c_void_p), ("k_mode", _c_int),
                ("table", _c_void_p)]


class BatchPlan:
    """Persistent, graph-captured evaluation of n_v walkers x n_b passbands
    over light curves of uneven length (pt_batch_plan_create / pt_batch_run).

    The plan binds the given tensors (their storage, not their values):
    update walker parameters or data in place between run() calls.
    k [n_v, n_b], ld [n_v, n_b, 2], y/wt [n_b, n_t]; flux/ssr are outputs
    ([n_v, n_b, n_t] / [n_v, n_b]); pass want_flux / want_ssr to allocate them.
    k_mode 1 evaluates the model once per walker with the mean k of its
    passbands and scales each passband's depth by k_b^2 / k_hat^2 (Sec. 3.5);
    k_mode 2 reads the Mandel-Agol terms from ``table`` (an MATable, kept
    alive by the plan) by bilinear interpolation (Sec. 2.2.3).
    """

    def __init__(self, t, lc_offsets, orb, k, ld, n_ss=1, t_exp=0.0, max_iter=16, y=None, wt=None,
                 want_flux=True, want_ssr=False, autotune=True, n_bad=None, k_mode=0, table=None):
        torch = _torch()
        lib = load_library()
        for name, res, args in [("pt_batch_plan_create", _c_int, [ctypes.POINTER(BatchDesc), _c_int,
                                                                 ctypes.POINTER(_c_void_p)]),
                                ("pt_batch_run", _c_int, [_c_void_p, _c_void_p]),
                                ("pt_batch_plan_info", _c_int, [_c_void_p, ctypes.POINTER(_c_int),
                                                                ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                                                ctypes.POINTER(ctypes.c_float)]),
                                ("pt_batch_plan_destroy", _c_int, [_c_void_p])]:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        o, n_v = _orbit_struct(orb)
        n_b = int(k.shape[1])
        n_t = t.numel()
        self.flux = torch.empty((n_v, n_b, n_t), dtype=torch.float32, device=t.device) if want_flux else None
        self.ssr = torch.empty((n_v, n_b), dtype=torch.float32, device=t.device) if want_ssr else None
        offs = [int(x) for x in lc_offsets]
        self._offs = (_c_int * len(offs))(*offs)
        self._keep = (t, orb, k, ld, y, wt, n_bad, table)
        d = BatchDesc(_ptr(t), n_t, self._offs, len(offs) - 1, o, _ptr(k), _ptr(ld), n_b, int(n_ss), float(t_exp),
                      int(max_iter), _ptr(y), _ptr(wt), _ptr(self.flux), _ptr(self.ssr), _ptr(n_bad), int(k_mode),
                      table.handle.value if table is not None else None)
        h = _c_void_p()
        _check(lib.pt_batch_plan_create(ctypes.byref(d), int(bool(autotune)), ctypes.byref(h)),
               "pt_batch_plan_create")
        self.handle = h

    def run(self):
        _check(load_library().pt_batch_run(self.handle, _stream()), "pt_batch_run")
        return self.flux, self.ssr

    def info(self):
        tile, cps, items = _c_int(), _c_int(), _c_int()
        ms = ctypes.c_float()
        load_library().pt_batch_plan_info(self.handle, ctypes.byref(tile), ctypes.byref(cps), ctypes.byref(items),
                                          ctypes.byref(ms))
        return dict(tile=tile.value, ctas_per_sm=cps.value, items=items.value, tuned_ms=ms.value)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().pt_batch_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
