"""Test helpers: one seeded workload, two views of it.

GPU-side parameters are FP32 except times, t0 and P (FP64).  The oracle gets
the same FP32-rounded values widened to FP64, so both sides evaluate the
model at identical inputs."""
import numpy as np

F32_KEYS = ("a", "inc", "e", "w")


def f32(x):
    return None if x is None else np.asarray(x, dtype=np.float32).astype(np.float64)


def oracle_orbit(orbit):
    out = dict(t0=np.asarray(orbit["t0"], np.float64), P=np.asarray(orbit["P"], np.float64))
    for key in F32_KEYS:
        out[key] = f32(orbit.get(key))
    return out


def gpu_inputs(wl, device="cuda"):
    import torch
    import paper_1504_07433_gb300 as pt
    t = torch.as_tensor(np.asarray(wl["t"], np.float64), device=device)
    orb = pt.orbit_to_device(wl["orbit"], device)
    k = torch.as_tensor(np.asarray(wl["k"], np.float32), device=device)
    ld = torch.as_tensor(np.asarray(wl["ld"], np.float32), device=device)
    return t, orb, k, ld
