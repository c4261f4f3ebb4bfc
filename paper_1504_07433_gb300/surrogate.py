"""Surrogate network for the ingress/egress Mandel-Agol terms: training on the
GPU with the library's own kernels, error-bound table, and serving.

The network (2 -> 128 -> 128 -> 128 -> 2, SiLU) maps normalised (k, s) to
normalised (lambda_d / k^2, eta_d / k^2) over the band z = |1-k| + 2 min(k,1) s.
Training data are (k, s) samples from a counter-based generator whose targets
come from the exact FP32 kernel (pt_sur_datagen); loss, gradients and the
Adam step are the library's kernels (pt_mlp_loss_grad, pt_mlp_adam); the last
epochs run quantisation-aware (BF16 rounding of the tensor-core operands in
the forward pass).  The error-bound table marks every (k, s) cell whose
worst validation error bound exceeds the threshold; those cells are served
by the exact kernel.  This module only sequences kernel calls.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _check, _c_int, _c_void_p, _ptr, _stream, _torch, load_library

N_PARAMS = 33666
HIDDEN = 128
K_LO, K_HI = 0.01, 0.3
# normalisation: k -> (k - 0.155)/0.145;  (ld/k^2 - 0.18)/0.165;  (ed/k^2 - 0.41)/0.25
NORM = (0.155, 0.145, 0.18, 0.165, 0.41, 0.25)
_OFF = {"W1": 0, "b1": 256, "W2": 384, "b2": 384 + 16384, "W3": 512 + 16384, "b3": 512 + 32768,
        "W4": 640 + 32768, "b4": 896 + 32768}


def _sig(lib):
    P = _c_void_p
    S = ctypes.c_size_t
    F = ctypes.c_float
    for name, res, args in [
        ("pt_mlp_work_bytes", S, [_c_int]),
        ("pt_sur_datagen", _c_int, [ctypes.c_ulonglong, S, S, F, F, P, P, P, P, P]),
        ("pt_mlp_forward", _c_int, [P, P, _c_int, _c_int, P, P, S, P]),
        ("pt_mlp_loss_grad", _c_int, [P, P, P, _c_int, _c_int, P, P, P, S, P]),
        ("pt_mlp_adam", _c_int, [P, P, P, P, _c_int, F, F, F, F, P]),
        ("pt_sur_model_create", _c_int, [P, ctypes.POINTER(F), F, F, ctypes.POINTER(ctypes.c_ubyte), _c_int, _c_int,
                                         ctypes.POINTER(_c_void_p)]),
        ("pt_sur_model_destroy", _c_int, [P]),
        ("pt_ma_surrogate", _c_int, [P, P, P, S, P, P, P, P, P, S, P]),
        ("pt_sur_work_bytes", S, [S]),
        ("pt_sur_mlp_eval", _c_int, [P, P, S, P, P]),
        ("pt_sur_cell_errors", _c_int, [P, P, P, P, P, P, S, F, F, _c_int, _c_int, P, P]),
        ("pt_sur_model_error", _c_int, [P, ctypes.POINTER(_c_int)]),
        ("pt_ma_terms", _c_int, [P, P, S, P, P, P, P]),
    ]:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def lib():
    return _sig(load_library())


def init_params(seed=0, device="cuda"):
    """He-style initial weights (numpy, seeded), zero biases."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS, np.float32)
    p[_OFF["W1"]:_OFF["b1"]] = rng.normal(0, math.sqrt(2.0 / 2), 256)
    p[_OFF["W2"]:_OFF["b2"]] = rng.normal(0, math.sqrt(2.0 / HIDDEN), HIDDEN * HIDDEN)
    p[_OFF["W3"]:_OFF["b3"]] = rng.normal(0, math.sqrt(2.0 / HIDDEN), HIDDEN * HIDDEN)
    p[_OFF["W4"]:_OFF["b4"]] = rng.normal(0, math.sqrt(1.0 / HIDDEN), 256)
    return torch.as_tensor(p, device=device)


def datagen(n, seed=1504, offset=0, device="cuda", with_kz=False):
    """(X [n,2], T [n,2], kz [n,2] or None) from pt_sur_datagen."""
    torch = _torch()
    L = lib()
    norm = torch.as_tensor(NORM, dtype=torch.float32, device=device)
    X = torch.empty((n, 2), dtype=torch.float32, device=device)
    T = torch.empty((n, 2), dtype=torch.float32, device=device)
    kz = torch.empty((n, 2), dtype=torch.float32, device=device) if with_kz else None
    _check(L.pt_sur_datagen(seed, offset, n, K_LO, K_HI, _ptr(norm), _ptr(X), _ptr(T), _ptr(kz), _stream()),
           "pt_sur_datagen")
    return X, T, kz


class Trainer:
    """Adam on the mean squared error; the last `qat_epochs` epochs round the
    tensor-core operands to BF16 in the forward pass."""

    def __init__(self, params, batch=16384, device="cuda"):
        torch = _torch()
        self.L = lib()
        self.p = params
        self.batch = batch
        self.g = torch.zeros_like(params)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        nb = int(self.L.pt_mlp_work_bytes(batch))
        self.work = torch.empty(nb, dtype=torch.uint8, device=device)
        self.step_no = 0

    def loss_grad(self, X, T, qat=False):
        n = X.shape[0]
        if n > self.batch:
            raise ValueError("batch larger than the trainer's work buffer")
        _check(self.L.pt_mlp_loss_grad(_ptr(self.p), _ptr(X), _ptr(T), n, int(bool(qat)), _ptr(self.g),
                                       _ptr(self.loss), _ptr(self.work), self.work.numel(), _stream()),
               "pt_mlp_loss_grad")
        return self.loss, self.g

    def step(self, X, T, lr, qat=False):
        self.loss_grad(X, T, qat)
        self.step_no += 1
        _check(self.L.pt_mlp_adam(_ptr(self.p), _ptr(self.g), _ptr(self.m), _ptr(self.v), self.step_no, float(lr),
                                  0.9, 0.999, 1e-8, _stream()), "pt_mlp_adam")

    def fit(self, X, T, epochs, lr0=2e-3, lr1=2e-5, qat_epochs=1, log=None):
        n = X.shape[0]
        nb = n // self.batch
        total = epochs * nb
        it = 0
        for ep in range(epochs):
            qat = ep >= epochs - qat_epochs
            shift = (ep * 7919 * self.batch) % max(1, n - nb * self.batch + 1)
            for b in range(nb):
                lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * it / max(1, total)))
                s = shift + b * self.batch
                self.step(X[s:s + self.batch], T[s:s + self.batch], lr, qat)
                it += 1
            if log is not None:
                log(ep, float(self.loss.item()))
        return self.p


def forward_f32(params, X, qat=False):
    torch = _torch()
    L = lib()
    n = X.shape[0]
    Y = torch.empty((n, 2), dtype=torch.float32, device=X.device)
    work = torch.empty(int(L.pt_mlp_work_bytes(n)), dtype=torch.uint8, device=X.device)
    _check(L.pt_mlp_forward(_ptr(params), _ptr(X), n, int(bool(qat)), _ptr(Y), _ptr(work), work.numel(), _stream()),
           "pt_mlp_forward")
    return Y


class SurrogateModel:
    """Served network (pt_sur_model_create): BF16 tensor-core layers plus the
    error-bound table (nk x ns cells; 1 = exact kernel)."""

    def __init__(self, params, table=None, nk=64, ns=64):
        L = lib()
        if table is None:
            table = np.zeros((nk, ns), np.uint8)
        table = np.ascontiguousarray(np.asarray(table, np.uint8))
        self.table = table
        nk, ns = table.shape
        norm = (ctypes.c_float * 6)(*NORM)
        h = _c_void_p()
        _check(L.pt_sur_model_create(_ptr(params), norm, K_LO, K_HI,
                                     table.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), nk, ns, ctypes.byref(h)),
               "pt_sur_model_create")
        self.handle = h
        self.nk, self.ns = nk, ns

    def terms(self, k, z, n_fallback=None, work=None, out=None):
        """(lambda_e, lambda_d', eta_d) like pt_ma_terms (pt_ma_surrogate)."""
        torch = _torch()
        if out is None:
            out = (torch.empty_like(z), torch.empty_like(z), torch.empty_like(z))
        le, ld, ed = out
        need = int(lib().pt_sur_work_bytes(z.numel()))
        if work is None or work.numel() < need:
            work = torch.empty(need, dtype=torch.uint8, device=z.device)
        _check(lib().pt_ma_surrogate(self.handle, _ptr(k), _ptr(z), z.numel(), _ptr(le), _ptr(ld), _ptr(ed),
                                     _ptr(n_fallback), _ptr(work), work.numel(), _stream()), "pt_ma_surrogate")
        return le, ld, ed

    def network(self, X):
        torch = _torch()
        Y = torch.empty_like(X)
        _check(lib().pt_sur_mlp_eval(self.handle, _ptr(X), X.shape[0], _ptr(Y), _stream()), "pt_sur_mlp_eval")
        return Y

    def timed_out(self):
        e = _c_int()
        _check(lib().pt_sur_model_error(self.handle, ctypes.byref(e)), "pt_sur_model_error")
        return bool(e.value)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().pt_sur_model_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exact_terms(k, z):
    torch = _torch()
    le = torch.empty_like(z)
    ld = torch.empty_like(z)
    ed = torch.empty_like(z)
    _check(lib().pt_ma_terms(_ptr(k), _ptr(z), z.numel(), _ptr(le), _ptr(ld), _ptr(ed), _stream()), "pt_ma_terms")
    return le, ld, ed


def cell_errors(model, k, z, nk, ns):
    """Per-cell maximum of 4|d lambda_d| + 2|d eta_d| (network vs exact) on (k, z)."""
    torch = _torch()
    _, ld_r, ed_r = exact_terms(k, z)
    free = SurrogateModel(model.params if hasattr(model, "params") else model, None, nk, ns) \
        if not isinstance(model, SurrogateModel) else model
    _, ld_s, ed_s = free.terms(k, z)
    cm = torch.zeros(nk * ns, dtype=torch.float32, device=z.device)
    _check(lib().pt_sur_cell_errors(_ptr(k), _ptr(z), _ptr(ld_r), _ptr(ed_r), _ptr(ld_s), _ptr(ed_s), z.numel(),
                                    K_LO, K_HI, nk, ns, _ptr(cm), _stream()), "pt_sur_cell_errors")
    return cm.view(nk, ns)


def validation_points(n, seed=7, device="cuda"):
    """(k, z) validation sample over the band (a generator stream disjoint from training)."""
    _, _, kz = datagen(n, seed=seed, offset=0, device=device, with_kz=True)
    return kz[:, 0].contiguous(), kz[:, 1].contiguous()


def build_table(params, nk=64, ns=64, n_val=4_000_000, threshold=5e-6, seed=7):
    """Error-bound table: a cell uses the network only if its worst validation
    bound 4|d lambda_d| + 2|d eta_d| stays under `threshold` (half the 1e-5
    flux budget, leaving margin for points between validation samples)."""
    k, z = validation_points(n_val, seed)
    free = SurrogateModel(params, np.zeros((nk, ns), np.uint8))
    cm = cell_errors(free, k, z, nk, ns)
    free.close()
    cm_h = cm.cpu().numpy()
    table = (cm_h > threshold).astype(np.uint8)
    return table, cm_h
