"""FP64 CPU oracle for the transit-model hot path (test infrastructure).

This package is the plain, slow, obviously-correct reference the CUDA library
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package never
does.  The arithmetic lives in ``pt_oracle.c`` (plain C99, FP64, optional
OpenMP over parameter vectors); this module compiles it with gcc on first use
and wraps it with ctypes and numpy.  Nothing here is shared with the CUDA path.

Conventions (the same readings the CUDA library documents):
  * t0 = time of inferior conjunction, true anomaly pi/2 - omega;
  * z of a point behind the star = ``Z_BEHIND``;
  * supersamples at t + t_exp ((s + 1/2)/n_ss - 1/2), unweighted mean (Sec. 3.2);
  * Gimenez series keeps j = 0 .. n_j - 1 (Sec. 2.1.1, Eq. gimenez).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_LOCK = threading.Lock()
_LIB = None

Z_BEHIND = 1.0e30

_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile pt_oracle.c into _liboracle.so (gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            for name, res, args in [
                ("pto_rc", _D, [_D, _D]),
                ("pto_rf", _D, [_D, _D, _D]),
                ("pto_rd", _D, [_D, _D, _D]),
                ("pto_rj", _D, [_D, _D, _D, _D]),
                ("pto_ellk", _D, [_D]),
                ("pto_elle", _D, [_D, _D]),
                ("pto_ellpi", _D, [_D, _D]),
                ("pto_lambda_e", _D, [_D, _D]),
                ("pto_ma_terms", None, [_D, _D, _PD]),
                ("pto_flux_quad", _D, [_D, _D, _D, _D]),
                ("pto_jacobi_g", None, [_I, _D, _D, _D, _PD]),
                ("pto_gimenez_a", _D, [_I, _I]),
                ("pto_gimenez_alpha", None, [_I, _I, _D, _D, _PD]),
                ("pto_flux_gimenez", _D, [_I, _I, _D, _D, _PD]),
                ("pto_ring_alpha", _D, [_I, _D, _D]),
                ("pto_ring_flux", _D, [_I, _PD, _D, _D]),
                ("pto_z_circ", _D, [_D, _D, _D, _D, _D]),
                ("pto_kepler_newton", _I, [_D, _D, _I, _D, _PD]),
                ("pto_z_ecc", _D, [_D, _D, _D, _D, _D, _D, _D, _I, _D, ctypes.POINTER(_I)]),
                ("pto_inc_from_b", _D, [_D, _D, _D, _D]),
                ("pto_z_batch", _I, [_PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I, _I, _D, _PD]),
                ("pto_lc_ma", _I, [_PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I, _PD, _I, _PD, _I, _I, _D,
                                   _PD, _I]),
                ("pto_lc_gimenez", _I, [_PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I, _PD, _I, _PD, _I, _I,
                                        _I, _I, _D, _PD, _I]),
                ("pto_ssr", None, [_PD, _PD, _PD, _I, _I, _I, _PD]),
                ("pto_max_threads", _I, []),
                ("pto_ma_terms_batch", None, [ctypes.c_long, _PD, _PD, _PD, _I]),
                ("pto_overlap_derivs", None, [_D, _D, _PD]),
                ("pto_flux_theta", _D, [_D, _PD, _I, _D]),
                ("pto_flux_grad", _D, [_D, _PD, _I, _D, _PD]),
                ("pto_ssr_grad", None, [_PD, _I, _PD, _I, _I, _D, _PD, _PD, _PD, _PD, _I]),
                ("pto_ma_table", None, [_D, _D, _I, _I, _PD]),
                ("pto_ma_interp", None, [_PD, _D, _D, _I, _I, _D, _D, _PD]),
                ("pto_flux_quad_interp", _D, [_PD, _D, _D, _I, _I, _D, _D, _D, _D]),
                ("pto_lc_ma_interp", _I, [_PD, _D, _D, _I, _I, _PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I,
                                          _PD, _I, _PD, _I, _I, _D, _PD, _I]),
                ("pto_gimenez_zi_table", None, [_I, _I, _D, _I, _I, _PD]),
                ("pto_gimenez_zi_alpha", None, [_I, _I, _I, _D, _PD, _D, _PD]),
                ("pto_lc_gimenez_zi", _I, [_PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I, _PD, _I, _PD, _I, _I, _I,
                                           _I, _I, _I, _D, _PD, _I]),
                ("pto_lc_ma_khat", _I, [_PD, _I, _PD, _PD, _PD, _PD, _PD, _PD, _I, _PD, _PD, _I, _I, _D, _PD,
                                        _I]),
                ("pto_mlp_nparams", _I, []),
                ("pto_mlp_forward", None, [_PD, _PD, _I, _PD]),
                ("pto_mlp_loss_grad", _D, [_PD, _PD, _PD, _I, _PD]),
            ]:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_PD)


# ---------------------------------------------------------------- scalars
def rf(x, y, z):
    return _lib().pto_rf(x, y, z)


def rd(x, y, z):
    return _lib().pto_rd(x, y, z)


def rj(x, y, z, p):
    return _lib().pto_rj(x, y, z, p)


def rc(x, y):
    return _lib().pto_rc(x, y)


def ellk(m):
    """K(m), m = k^2."""
    return _lib().pto_ellk(1.0 - m)


def elle(m):
    """E(m), m = k^2."""
    return _lib().pto_elle(m, 1.0 - m)


def ellpi(n, m):
    """Pi(n|m) = int dth / ((1 - n sin^2) sqrt(1 - m sin^2)), n < 1."""
    return _lib().pto_ellpi(n, 1.0 - m)


def lambda_e(p, z):
    return _lib().pto_lambda_e(p, z)


def ma_terms(p, z):
    """(lambda_e, lambda_d, eta_d) of Mandel & Agol (lambda_d without 2/3 Theta(p-z))."""
    out = np.zeros(3)
    _lib().pto_ma_terms(p, z, _ptr(out))
    return out


def ma_terms_batch(p, z, n_threads=0):
    """ma_terms at many points: [n, 3] of (lambda_e, lambda_d, eta_d)."""
    p, z = (np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel()) for x in np.broadcast_arrays(p, z))
    out = np.zeros((z.size, 3))
    _lib().pto_ma_terms_batch(z.size, _ptr(p), _ptr(z), _ptr(out), int(n_threads))
    return out


def flux_quad(p, z, u1, u2):
    return _lib().pto_flux_quad(p, z, u1, u2)


def flux_quad_vec(p, z, u1, u2):
    p, z, u1, u2 = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64) for x in (p, z, u1, u2)))
    f = _lib().pto_flux_quad
    return np.array([f(a, b, c, d) for a, b, c, d in zip(p.ravel(), z.ravel(), u1.ravel(), u2.ravel())]
                    ).reshape(p.shape)


def jacobi_g(n, p, q, x):
    g = np.zeros(n)
    _lib().pto_jacobi_g(n, p, q, x, _ptr(g))
    return g


def gimenez_a(n, j):
    return _lib().pto_gimenez_a(n, j)


def gimenez_alpha(N, n_j, k, z):
    out = np.zeros(N + 1)
    _lib().pto_gimenez_alpha(N, n_j, k, z, _ptr(out))
    return out


def flux_gimenez(k, z, u, n_j):
    u = _arr(u)
    return _lib().pto_flux_gimenez(u.size, n_j, k, z, _ptr(u))


def ring_alpha(n, k, z):
    """alpha_n from its definition: (1/pi) x the mu^n-weighted area of the
    stellar disk covered by the planet, a ring integral (tanh-sinh)."""
    return _lib().pto_ring_alpha(int(n), float(k), float(z))


def ring_flux(u, k, z):
    """Flux of the general law u_1..u_N (Eq. ld_general) from its definition:
    1 - blocked / total light, both as ring integrals."""
    u = _arr(u)
    return _lib().pto_ring_flux(u.size, _ptr(u), float(k), float(z))


def z_circ(t, t0, P, a, inc):
    return _lib().pto_z_circ(t, t0, P, a, inc)


def kepler_newton(M, e, max_iter=50, tol=1e-14):
    E = ctypes.c_double()
    it = _lib().pto_kepler_newton(M, e, max_iter, tol, ctypes.byref(E))
    return E.value, it


def z_ecc(t, t0, P, a, inc, e, w, max_iter=50, tol=1e-14):
    st = ctypes.c_int()
    z = _lib().pto_z_ecc(t, t0, P, a, inc, e, w, max_iter, tol, ctypes.byref(st))
    return z, st.value


def inc_from_b(b, a, e=0.0, w=0.5 * np.pi):
    return _lib().pto_inc_from_b(b, a, e, w)


# ---------------------------------------------------------------- batched
def _orbit(orbit, n_v):
    t0 = _arr(orbit["t0"], n_v)
    P = _arr(orbit["P"], n_v)
    a = _arr(orbit["a"], n_v)
    inc = _arr(orbit["inc"], n_v)
    e = orbit.get("e")
    w = orbit.get("w")
    e = None if e is None else _arr(e, n_v)
    w = None if (e is None or w is None) else _arr(w, n_v)
    if e is not None and w is None:
        raise ValueError("eccentric orbit needs w")
    return t0, P, a, inc, e, w


def z_batch(t, orbit, n_ss=1, t_exp=0.0):
    """z[v, t*n_ss + s] for every vector, time and supersample."""
    t = _arr(t)
    n_v = len(np.atleast_1d(orbit["t0"]))
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    z = np.zeros((n_v, t.size * n_ss))
    nbad = _lib().pto_z_batch(_ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc), _ptr(e), _ptr(w),
                              n_v, n_ss, t_exp, _ptr(z))
    return z, nbad


def lc_ma(t, orbit, k, ld, n_ss=1, t_exp=0.0, n_threads=0):
    """Quadratic MA flux cube [n_v, n_b, n_t]; ld is [n_v, n_b, 2] (u1, u2);
    k is [n_v] or [n_v, n_b]."""
    t = _arr(t)
    ld = np.ascontiguousarray(np.asarray(ld, dtype=np.float64))
    n_v, n_b = ld.shape[0], ld.shape[1]
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64))
    kpb = 1 if k.ndim == 2 else 0
    flux = np.zeros((n_v, n_b, t.size))
    nbad = _lib().pto_lc_ma(_ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc), _ptr(e), _ptr(w), n_v,
                            _ptr(k), kpb, _ptr(ld), n_b, n_ss, t_exp, _ptr(flux), n_threads)
    return flux, nbad


def lc_ma_khat(t, orbit, k, ld, n_ss=1, t_exp=0.0, n_threads=0):
    """Quadratic MA flux cube with per-passband k through the k^2 / k_hat^2
    scaling of Sec. 3.5; k and ld are [n_v, n_b] and [n_v, n_b, 2]."""
    t = _arr(t)
    ld = np.ascontiguousarray(np.asarray(ld, dtype=np.float64))
    n_v, n_b = ld.shape[0], ld.shape[1]
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, dtype=np.float64), (n_v, n_b)))
    flux = np.zeros((n_v, n_b, t.size))
    nbad = _lib().pto_lc_ma_khat(_ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc), _ptr(e), _ptr(w), n_v,
                                 _ptr(k), _ptr(ld), n_b, n_ss, t_exp, _ptr(flux), n_threads)
    return flux, nbad


class MATable:
    """Interpolation table of the Mandel-Agol terms (Sec. 2.2.3): n_k radius
    ratios over [k_lo, k_hi] x n_z separations over [0, 1 + k_hi]; the values
    are (lambda_e, lambda_d + 2/3 Theta(k - z), eta_d) of ma_terms."""

    def __init__(self, k_lo, k_hi, n_k, n_z):
        if n_k < 2 or n_z < 2 or not k_hi > k_lo:
            raise ValueError("need n_k, n_z >= 2 and k_hi > k_lo")
        self.k_lo, self.k_hi, self.n_k, self.n_z = float(k_lo), float(k_hi), int(n_k), int(n_z)
        self.tab = np.zeros((n_k, n_z, 3))
        _lib().pto_ma_table(self.k_lo, self.k_hi, self.n_k, self.n_z, _ptr(self.tab))

    def _args(self):
        return _ptr(self.tab), self.k_lo, self.k_hi, self.n_k, self.n_z

    def terms(self, k, z):
        """Interpolated (lambda_e, lambda_d + 2/3 Theta, eta_d) for one (k, z)."""
        out = np.zeros(3)
        _lib().pto_ma_interp(*self._args(), float(k), float(z), _ptr(out))
        return out

    def terms_vec(self, k, z):
        k = np.broadcast_to(np.asarray(k, dtype=np.float64), np.shape(z)).ravel()
        z = np.asarray(z, dtype=np.float64).ravel()
        out = np.zeros((z.size, 3))
        for i in range(z.size):
            out[i] = self.terms(k[i], z[i])
        return out

    def flux(self, k, z, u1, u2):
        return _lib().pto_flux_quad_interp(*self._args(), float(k), float(z), float(u1), float(u2))


def lc_ma_interp(table, t, orbit, k, ld, n_ss=1, t_exp=0.0, n_threads=0):
    """lc_ma with the terms read from an MATable (Sec. 2.2.3)."""
    t = _arr(t)
    ld = np.ascontiguousarray(np.asarray(ld, dtype=np.float64))
    n_v, n_b = ld.shape[0], ld.shape[1]
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64))
    kpb = 1 if k.ndim == 2 else 0
    flux = np.zeros((n_v, n_b, t.size))
    nbad = _lib().pto_lc_ma_interp(*table._args(), _ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc),
                                   _ptr(e), _ptr(w), n_v, _ptr(k), kpb, _ptr(ld), n_b, n_ss, t_exp, _ptr(flux),
                                   n_threads)
    return flux, nbad


def lc_gimenez(t, orbit, k, ld, n_j, n_ss=1, t_exp=0.0, n_threads=0):
    """Gimenez flux cube [n_v, n_b, n_t]; ld is [n_v, n_b, N] (u_1..u_N of Eq. ld_general)."""
    t = _arr(t)
    ld = np.ascontiguousarray(np.asarray(ld, dtype=np.float64))
    n_v, n_b, N = ld.shape
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64))
    kpb = 1 if k.ndim == 2 else 0
    flux = np.zeros((n_v, n_b, t.size))
    nbad = _lib().pto_lc_gimenez(_ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc), _ptr(e), _ptr(w),
                                 n_v, _ptr(k), kpb, _ptr(ld), N, n_b, n_j, n_ss, t_exp, _ptr(flux), n_threads)
    return flux, nbad


def gimenez_zi_table(N, n_j, k, n_in, n_edge):
    """alpha_0..alpha_N on the z nodes of the interpolated Gimenez model
    (Sec. 3.3): [n_in + n_edge, N + 1]."""
    tab = np.zeros((n_in + n_edge, N + 1))
    _lib().pto_gimenez_zi_table(int(N), int(n_j), float(k), int(n_in), int(n_edge), _ptr(tab))
    return tab


def gimenez_zi_alpha(tab, k, z, n_in, n_edge):
    tab = np.ascontiguousarray(tab, dtype=np.float64)
    N = tab.shape[1] - 1
    out = np.zeros(N + 1)
    _lib().pto_gimenez_zi_alpha(N, int(n_in), int(n_edge), float(k), _ptr(tab), float(z), _ptr(out))
    return out


def lc_gimenez_zi(t, orbit, k, ld, n_j, n_in, n_edge, n_ss=1, t_exp=0.0, n_threads=0):
    """lc_gimenez with the series read from z tables (Sec. 3.3)."""
    t = _arr(t)
    ld = np.ascontiguousarray(np.asarray(ld, dtype=np.float64))
    n_v, n_b, N = ld.shape
    t0, P, a, inc, e, w = _orbit(orbit, n_v)
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64))
    kpb = 1 if k.ndim == 2 else 0
    flux = np.zeros((n_v, n_b, t.size))
    nbad = _lib().pto_lc_gimenez_zi(_ptr(t), t.size, _ptr(t0), _ptr(P), _ptr(a), _ptr(inc), _ptr(e), _ptr(w),
                                    n_v, _ptr(k), kpb, _ptr(ld), N, n_b, n_j, int(n_in), int(n_edge), n_ss, t_exp,
                                    _ptr(flux), n_threads)
    return flux, nbad


def ssr(flux, y, wt=None):
    flux = np.ascontiguousarray(np.asarray(flux, dtype=np.float64))
    n_v, n_b, n_t = flux.shape
    y = _arr(y, n_b * n_t)
    wt = None if wt is None else _arr(wt, n_b * n_t)
    out = np.zeros((n_v, n_b))
    _lib().pto_ssr(_ptr(flux), _ptr(y), _ptr(wt), n_v, n_b, n_t, _ptr(out))
    return out


def max_threads():
    return _lib().pto_max_threads()


# ---------------------------------------------------------------- gradients
THETA = ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")


def overlap_derivs(p, z):
    """(dI1/dp, dI1/dz, dImu/dp, dImu/dz, dImu2/dp, dImu2/dz) of the overlap integrals."""
    out = np.zeros(6)
    _lib().pto_overlap_derivs(p, z, _ptr(out))
    return out


def flux_theta(t, th, n_ss=1, t_exp=0.0):
    th = _arr(th, 9)
    return _lib().pto_flux_theta(t, _ptr(th), n_ss, t_exp)


def flux_grad(t, th, n_ss=1, t_exp=0.0):
    th = _arr(th, 9)
    g = np.zeros(9)
    f = _lib().pto_flux_grad(t, _ptr(th), n_ss, t_exp, _ptr(g))
    return f, g


def ssr_grad(t, th, y, wt=None, n_ss=1, t_exp=0.0, n_threads=0):
    """SSR [n_v] and d SSR / d theta [n_v, 9] for theta rows (t0, P, a, b, e, w, k, u1, u2)."""
    t = _arr(t)
    th = np.ascontiguousarray(np.asarray(th, dtype=np.float64).reshape(-1, 9))
    y = _arr(y, t.size)
    wt = None if wt is None else _arr(wt, t.size)
    n_v = th.shape[0]
    ssr = np.zeros(n_v)
    grad = np.zeros((n_v, 9))
    _lib().pto_ssr_grad(_ptr(t), t.size, _ptr(th), n_v, n_ss, t_exp, _ptr(y), _ptr(wt), _ptr(ssr), _ptr(grad),
                        n_threads)
    return ssr, grad


# ---------------------------------------------------------------- surrogate network
def mlp_nparams():
    return _lib().pto_mlp_nparams()


def mlp_forward(params, X):
    """y [n, 2] of the 2-128-128-128-2 SiLU network (flattened FP64 params)."""
    p = _arr(params, mlp_nparams())
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 2))
    Y = np.zeros_like(X)
    _lib().pto_mlp_forward(_ptr(p), _ptr(X), X.shape[0], _ptr(Y))
    return Y


def mlp_loss_grad(params, X, T):
    """(loss, grad) for L = mean_i sum_o (y_io - t_io)^2."""
    p = _arr(params, mlp_nparams())
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 2))
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(-1, 2))
    g = np.zeros(p.size)
    loss = _lib().pto_mlp_loss_grad(_ptr(p), _ptr(X), _ptr(T), X.shape[0], _ptr(g))
    return loss, g
