"""Benchmark: flux points per second of the transit-model hot path on GB300.

Workload (one step): the long-cadence series -- 50,000 exposure times over
1,000 d, 29.4-min exposures supersampled x10, 256 eccentric parameter vectors
drawn from the seeded priors, one passband -- evaluated with BOTH models:
quadratic Mandel-Agol (pt_ma_quad) and the Gimenez series with 8
general-law coefficients (pt_gimenez) at N_J = 192 Jacobi terms, the
smallest depth whose truncation error stays within 1e-5 over the workload's
priors (Sec. 2.1.1; the study is tests/golden/gimenez_truncation.json).  A
flux point is one (exposure time, parameter vector, passband) output; a step
produces 2 x 50,000 x 256 of them.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; between steps a 256 MiB buffer is written to flush
L2 (outside the events).  Barrier + synchronize on both sides; the max over
ranks is reported.  Under torchrun every rank runs its own replica (the path
has no exchange step), so scaling is weak.

Further legs (each with its error against the FP64 oracle, computed in the
CPU-baseline leg at the end, the one place the benchmark runs the oracle):
end to end from host buffers (flux cubes back, and the likelihood-only form
of Sec. 3.4), the single light curve of 1,000 points (latency and CUDA-graph
replay), interpolated Mandel-Agol (Sec. 2.2.3), Gimenez interpolated in z
(Sec. 3.3), the adjoint, batched spectrophotometry and the surrogate.

--impl reference times the FP64 oracle (the CPU reference) on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "flux points/sec (time×sample×passband) on 1 GB300 at ≤1e-5 max abs error vs FP64"
UNIT = "flux points/s"
N_LD = 8
N_J = 192                # smallest depth within 1e-5 (less the FP32 budget) over the long-cadence priors
SAMPLE_V = 64            # vectors in the CPU-oracle sample (about 10 s of host work)
GOLDEN = os.path.join(ROOT, "tests", "golden", "gimenez_truncation.json")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of one gim_cheb_kernel launch (dram__bytes_read.sum +
# dram__bytes_write.sum) from its ncu capture, per vector of the long-cadence
# workload, and the build it was taken on (null for any other depth)
TRAFFIC = {"per_vector_bytes": (2.398208e6 + 7.424e3) / 128.0, "n_j": 192}


def whole_job_rate(ms_local, pts_per_rank, ws, device="cpu"):
    """The job's time per step is the slowest rank's (a MAX all-reduce when
    ws > 1); the rate counts the points of every rank (weak scaling: each
    rank evaluates its own replica).  Returns (ms, points/s)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, pts_per_rank * ws / (ms * 1e-3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _timed(torch, stream, K, flush, fn, warm=3):
    """Mean CUDA-event time (ms) of fn on `stream`, L2 flushed before each call."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ms = []
    for i in range(K):
        if flush is not None:
            flush.fill_(i & 0xff)
        e0, e1 = _events(torch, 2)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


def _host(x):
    return None if x is None else x.detach().cpu().numpy()


# ---------------------------------------------------------------------------
# Legs.  Each returns (result dict for the JSON line, host payload the CPU
# leg checks against the oracle).
# ---------------------------------------------------------------------------
def bench_plain(pt, torch, dev, stream, n_calls=500):
    """The single light curve of 1,000 points (circular, 1 vector, 1
    passband): latency-bound.  Mean time per call with calls issued back to
    back (CUDA events around n_calls calls, and host wall time), and per
    replay of the call captured in a CUDA graph."""
    from paper_1504_07433_gb300 import workloads as W
    wl = W.plain()
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device=dev)
    orb = pt.orbit_to_device(wl["orbit"], dev)
    k = torch.as_tensor(wl["k"], dtype=torch.float32, device=dev)
    ld = torch.as_tensor(wl["ld"], dtype=torch.float32, device=dev)
    work = torch.empty(pt.ma_quad_work_bytes(t.numel(), 1, 1), dtype=torch.uint8, device=dev)
    flux = torch.empty((1, 1, t.numel()), dtype=torch.float32, device=dev)

    def call():
        pt.ma_quad(t, orb, k, ld, work=work, flux=flux)

    for _ in range(20):
        call()
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    w0 = time.perf_counter()
    e0.record(stream)
    for _ in range(n_calls):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    wall_us = (time.perf_counter() - w0) / n_calls * 1e6
    call_us = e0.elapsed_time(e1) / n_calls * 1e3
    out = {"workload": wl["name"], "us_per_call": call_us, "host_wall_us_per_call": wall_us,
           "value": t.numel() / (call_us * 1e-6), "unit": "flux points/s",
           "gpu_launches_per_call": 2}   # one geometry: set-up + the tile kernel
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            call()
        stream.wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            call()
        for _ in range(20):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        e0.record(stream)
        for _ in range(n_calls):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        out["graph_replay_us"] = e0.elapsed_time(e1) / n_calls * 1e3
    except Exception as exc:   # reported, not fatal: the direct calls are the leg's number
        out["graph_replay_error"] = str(exc)[:200]
    return out, {"wl": wl, "flux": _host(flux)}


def bench_ma_interp(pt, torch, dev, stream, K, flush, t, orb, k, ld, wl, f_exact, k_lo=0.05, k_hi=0.2, n_chk=16):
    """Interpolated Mandel-Agol light curves (Sec. 2.2.3) on the long-cadence
    workload: a table over the workload's k range at the paper's default grid
    (n_k = 128, n_z = 256), timed like the exact MA call."""
    tab = pt.MATable(k_lo, k_hi, 128, 256)
    n_t, n_v = t.numel(), k.numel()
    work = torch.empty(pt.ma_quad_work_bytes(n_t, n_v, 1), dtype=torch.uint8, device=dev)
    f = torch.empty_like(f_exact)

    def run():
        pt.ma_quad_interp(tab, t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work, flux=f)

    m = _timed(torch, stream, K, flush, run)
    err = float((f.double() - f_exact.double()).abs().max().item())
    tab.close()
    out = {"workload": wl["name"], "table": "k in [%.2f, %.2f], n_k = 128, n_z = 256" % (k_lo, k_hi),
           "ms_per_call": m, "value": n_t * n_v / (m * 1e-3), "unit": "flux points/s",
           "max_abs_diff_vs_exact_fp32": err, "gpu_launches_per_call": 2}
    return out, {"flux": _host(f[:n_chk, 0]), "k_lo": k_lo, "k_hi": k_hi, "n_chk": n_chk}


def bench_gimenez_zi(pt, torch, dev, stream, K, flush, plan, t, orb, k, ldg, wl, f_series, n_in=64, n_edge=64,
                     n_chk=16):
    """Gimenez model interpolated in z (Sec. 3.3) on the long-cadence
    workload, timed like the series call."""
    n_t, n_v = t.numel(), k.numel()
    work = torch.empty(int(pt.load_library().pt_gimenez_zi_work_bytes(plan.handle, n_in, n_edge, n_t, n_v, 1, 0)),
                       dtype=torch.uint8, device=dev)
    f = torch.empty_like(f_series)

    def run():
        pt.gimenez_zi(plan, t, orb, k, ldg, n_in=n_in, n_edge=n_edge, n_ss=wl["n_ss"], t_exp=wl["t_exp"], work=work,
                      flux=f)

    m = _timed(torch, stream, K, flush, run)
    err = float((f.double() - f_series.double()).abs().max().item())
    out = {"workload": wl["name"], "grid": "n_in = %d, n_edge = %d" % (n_in, n_edge), "ms_per_call": m,
           "value": n_t * n_v / (m * 1e-3), "unit": "flux points/s", "max_abs_diff_vs_series_fp32": err,
           "gpu_launches_per_call": 6}
    return out, {"flux": _host(f[:n_chk, 0]), "n_in": n_in, "n_edge": n_edge, "n_chk": n_chk}


def bench_adjoint(pt, torch, dev, stream, K, flush, n_v=4096, n_chk=8):
    """Adjoint workload: 4,096 eccentric vectors x 10,000 times, forward +
    gradient of the SSR w.r.t. 9 parameters per vector (pt_ma_quad_bwd).
    Reported in flux points (time x vector) per second, forward and backward
    together; y is a synthetic light curve (not timed)."""
    from paper_1504_07433_gb300 import workloads as W
    wl = W.adjoint(n_v=n_v)
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device=dev)
    th = pt.theta_to_device(wl["theta"], dev)
    rng = np.random.default_rng(77)
    y_h = (1.0 + rng.normal(0.0, 1e-4, t.numel())).astype(np.float32)
    y = torch.as_tensor(y_h, device=dev)
    work = torch.empty(pt.load_library().pt_ma_quad_bwd_work_bytes(t.numel()), dtype=torch.uint8, device=dev)
    res = {}

    def run():
        res["out"] = pt.ma_quad_bwd(t, th, y, work=work)

    m = _timed(torch, stream, K, flush, run)
    ssr, grad, _ = res["out"]
    pts = t.numel() * th["t0"].numel()
    idx = np.random.default_rng(78).choice(th["t0"].numel(), min(n_chk, th["t0"].numel()), replace=False)
    out = {"workload": wl["name"], "ms_per_call": m, "value": pts / (m * 1e-3), "unit": "flux points/s (fwd+grad)",
           "gpu_launches_per_call": 2}
    return out, {"wl": wl, "y": y_h, "idx": idx, "grad": _host(grad)[idx], "ssr": _host(ssr)[idx]}


def bench_batched(pt, torch, dev, stream, K, flush, n_walkers=1024, modes=("ssr", "cube"), n_chk=32):
    """Batched spectrophotometry: 1,024 walkers x 64 passbands (own k and LD)
    x 32 light curves of 500-5,000 points, one graph-captured persistent
    launch per evaluation, autotuned.  Fused SSR (no flux cube) and the full
    FP32 flux cube (~23 GB written per evaluation); in SSR mode also the
    k^2 / k_hat^2 scaling (Sec. 3.5) and the interpolated terms (Sec. 2.2.3)."""
    from paper_1504_07433_gb300 import workloads as W
    wl = W.batched(n_walkers=n_walkers)
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device=dev)
    orb = pt.orbit_to_device(wl["orbit"], dev)
    k = torch.as_tensor(wl["k"], dtype=torch.float32, device=dev)
    ld = torch.as_tensor(wl["ld"], dtype=torch.float32, device=dev)
    y = torch.as_tensor(wl["y"], dtype=torch.float32, device=dev)
    n_v, n_b, n_t = k.shape[0], k.shape[1], t.numel()
    pts = n_v * n_b * n_t
    out = {"workload": wl["name"], "flux_points_per_call": pts}
    rng = np.random.default_rng(91)
    pairs = np.stack([rng.choice(n_v, n_chk, replace=False), rng.integers(0, n_b, n_chk)], axis=1)
    payload = {"wl": wl, "pairs": pairs}

    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, y=y, want_flux=False, want_ssr=True, autotune=True)
    m = _timed(torch, stream, K, flush, plan.run, warm=2)
    out["ssr_mode"] = dict(plan.info(), ms_per_call=m, value=pts / (m * 1e-3), unit="flux points/s")
    payload["ssr"] = _host(plan.ssr)[pairs[:, 0], pairs[:, 1]]
    plan.close()
    del plan
    torch.cuda.empty_cache()
    # per-passband k through the k^2 / k_hat^2 scaling (Sec. 3.5): timed in
    # SSR mode; its departure from per-passband k on a 16-walker flux cube
    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, y=y, want_flux=False, want_ssr=True, autotune=True,
                        k_mode=1)
    m = _timed(torch, stream, K, flush, plan.run, warm=2)
    sub = {kk: (None if vv is None else vv[:16]) for kk, vv in orb.items()}
    fe = pt.BatchPlan(t, wl["lc_offsets"], sub, k[:16].contiguous(), ld[:16].contiguous(), want_flux=True).run()[0]
    fk = pt.BatchPlan(t, wl["lc_offsets"], sub, k[:16].contiguous(), ld[:16].contiguous(), want_flux=True,
                      k_mode=1).run()[0]
    err = float((fk.double() - fe.double()).abs().max().item())
    out["khat_ssr_mode"] = dict(plan.info(), ms_per_call=m, value=pts / (m * 1e-3), unit="flux points/s",
                                max_abs_diff_vs_per_band_k_16_walkers=err)
    payload["khat_flux_w0"] = _host(fk[0])
    plan.close()
    del plan, fk
    torch.cuda.empty_cache()
    # per-passband k with the Mandel-Agol terms from the interpolation table of
    # Sec. 2.2.3 (the paper's own GPU method): timed in SSR mode; its departure
    # from the exact terms on the same 16-walker flux cube
    grid = (0.09, 0.11, 128, 512)   # the workload's radius ratios; n_z = 512 keeps the grid error < 1e-5
    table = pt.MATable(*grid)
    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, y=y, want_flux=False, want_ssr=True, autotune=True,
                        k_mode=2, table=table)
    m = _timed(torch, stream, K, flush, plan.run, warm=2)
    fi = pt.BatchPlan(t, wl["lc_offsets"], sub, k[:16].contiguous(), ld[:16].contiguous(), want_flux=True,
                      k_mode=2, table=table).run()[0]
    err = float((fi.double() - fe.double()).abs().max().item())
    out["interp_ssr_mode"] = dict(plan.info(), ms_per_call=m, value=pts / (m * 1e-3), unit="flux points/s",
                                  table="k in [%.2f, %.2f], n_k = %d, n_z = %d" % grid,
                                  max_abs_diff_vs_exact_fp32_16_walkers=err)
    payload["interp_grid"] = grid
    payload["interp_flux_w0"] = _host(fi[0])
    plan.close()
    del plan, fe, fi, table
    torch.cuda.empty_cache()
    if "cube" not in modes:
        return out, payload
    plan = pt.BatchPlan(t, wl["lc_offsets"], orb, k, ld, want_flux=True, want_ssr=False, autotune=True)
    m = _timed(torch, stream, K, flush, plan.run, warm=2)
    peaks, src = _peaks()
    gbs = 4.0 * pts / (m * 1e-3) / 1e9
    out["cube_mode"] = dict(plan.info(), ms_per_call=m, value=pts / (m * 1e-3), unit="flux points/s",
                            store_gbs=gbs, store_frac_of_hbm=gbs / float(peaks.get("hbm_gbs", 6800.0)))
    cube_w = [0, int(rng.integers(1, n_v))]
    payload["cube_walkers"] = cube_w
    payload["cube"] = [_host(plan.flux[v]) for v in cube_w]
    plan.close()
    del plan
    torch.cuda.empty_cache()
    return out, payload


def bench_surrogate(torch, dev, stream, n_infer=1_000_000_000, epochs=40, n_chk=10_000_000):
    """Surrogate network: trained here on 1e7 exact-kernel samples (40 epochs,
    the library's own kernels), error-bound table from 4e6 validation points,
    then 1e9 band points through pt_ma_surrogate (BF16 tensor cores + exact
    fallback) against the exact FP32 kernel pt_ma_terms on the same points."""
    import paper_1504_07433_gb300.surrogate as S
    t0 = time.perf_counter()
    X, T, _ = S.datagen(10_000_000, seed=1504, device=dev)
    tr = S.Trainer(S.init_params(0, device=dev), batch=16384, device=dev)
    tr.fit(X, T, epochs=epochs, lr0=1e-3, lr1=1e-6, qat_epochs=min(3, epochs))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, T
    table, cm = S.build_table(tr.p, nk=64, ns=64, n_val=4_000_000, threshold=5e-6)
    model = S.SurrogateModel(tr.p, table)
    k, z = S.validation_points(n_infer, seed=5, device=dev)
    outs = tuple(torch.empty_like(z) for _ in range(3))
    work = torch.empty(int(S.lib().pt_sur_work_bytes(z.numel())), dtype=torch.uint8, device=dev)
    nfb = torch.zeros(1, dtype=torch.int32, device=dev)
    from paper_1504_07433_gb300 import _check, _ptr, _stream

    def run_exact():
        _check(S.lib().pt_ma_terms(_ptr(k), _ptr(z), z.numel(), _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2]),
                                   _stream()), "pt_ma_terms")

    def run_sur():
        model.terms(k, z, nfb, work, outs)

    # the paper's interpolation tables (Sec. 2.2.3) over the same k range, with
    # a grid fine enough that their error is comparable with the surrogate's
    # (over this wide k range the k spacing dominates the error in the band:
    # the contact z = 1 + k moves across a cell)
    import paper_1504_07433_gb300 as pt
    itab = pt.MATable(0.01, 0.3, 512, 2048)

    def run_interp():
        _check(S.lib().pt_ma_terms_interp(itab.handle, _ptr(k), _ptr(z), z.numel(), _ptr(outs[0]), _ptr(outs[1]),
                                          _ptr(outs[2]), _stream()), "pt_ma_terms_interp")

    idx = torch.as_tensor(np.unique(np.random.default_rng(66).integers(0, n_infer, n_chk)), device=dev)
    payload = {"k": _host(k[idx]), "z": _host(z[idx])}
    res = {}
    share = None
    for name, fn in (("exact", run_exact), ("surrogate", run_sur), ("interp", run_interp)):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(3):
            nfb.zero_()
            e0, e1 = _events(torch, 2)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = float(np.mean(ms))
        payload[name] = [_host(o[idx]) for o in outs]
        if name == "surrogate":
            share = 1.0 - int(nfb.item()) / n_infer
    # points the network served differ from the exact FP32 kernel's values
    served = np.any(np.stack([payload["surrogate"][i] != payload["exact"][i] for i in range(3)]), axis=0)
    payload["served"] = served
    out = {"workload": "%.0e (k, z) points over k in [0.01, 0.3], z in [|1-k|, 1+k]" % n_infer,
           "train_s": t_train, "train_samples": 10_000_000, "epochs": epochs,
           "table_cells_exact": float(table.mean()), "network_share": share,
           "exact_ms": res["exact"], "surrogate_ms": res["surrogate"],
           "exact_points_per_s": n_infer / (res["exact"] * 1e-3),
           "surrogate_points_per_s": n_infer / (res["surrogate"] * 1e-3),
           "gain_vs_exact": res["exact"] / res["surrogate"], "timed_out": model.timed_out(),
           "interp_table": "k in [0.01, 0.3], n_k = 512, n_z = 2048 (Sec. 2.2.3)", "interp_ms": res["interp"],
           "interp_points_per_s": n_infer / (res["interp"] * 1e-3), "interp_gain_vs_exact": res["exact"] / res["interp"],
           "tensor_tflops": share * n_infer * 2 * 2 * 128 * 128 / (res["surrogate"] * 1e-3) / 1e12,
           "check_sample": "%d of the points (seeded), of which %d network-served" % (n_chk, int(served.sum()))}
    model.close()
    itab.close()
    del k, z, outs, work
    torch.cuda.empty_cache()
    return out, payload


# ---------------------------------------------------------------------------
# CPU leg: the oracle timed on the host cores, and every leg's error against it
# ---------------------------------------------------------------------------
def _oracle_sample(wl, n_v, n_t=None, v0=0):
    """Inputs of vectors v0 .. v0 + n_v (and optionally the first n_t times),
    with the FP32 parameters the GPU sees widened to FP64."""
    f32 = lambda x: None if x is None else np.asarray(x, np.float32).astype(np.float64)
    sl = slice(v0, v0 + n_v)
    o = wl["orbit"]
    orb = dict(t0=np.asarray(o["t0"])[sl], P=np.asarray(o["P"])[sl], a=f32(o["a"][sl]), inc=f32(o["inc"][sl]),
               e=f32(o["e"][sl]) if o.get("e") is not None else None,
               w=f32(o["w"][sl]) if o.get("w") is not None else None)
    t = wl["t"] if n_t is None else wl["t"][:n_t]
    return t, orb, f32(wl["k"][sl]), f32(wl["ld"][sl]), (f32(wl["ld_gim"][sl]) if "ld_gim" in wl else None)


def run_oracle_step(wl, n_v, n_t=None, n_threads=0):
    """One oracle pass (both models) over a sample; returns (seconds, flux points, (fm, fg))."""
    import oracle
    t, orb, k, ld, ldg = _oracle_sample(wl, n_v, n_t)
    t0 = time.perf_counter()
    fm, _ = oracle.lc_ma(t, orb, k, ld, n_ss=wl["n_ss"], t_exp=wl["t_exp"], n_threads=n_threads)
    fg, _ = oracle.lc_gimenez(t, orb, k, ldg, N_J, n_ss=wl["n_ss"], t_exp=wl["t_exp"], n_threads=n_threads)
    dt = time.perf_counter() - t0
    return dt, fm.size + fg.size, (fm, fg)


def _rate(fn, n_points, min_s=0.3):
    """Oracle points per second of `fn` (which computes `n_points` points per call),
    repeating the call until `min_s` seconds have passed; returns (last result, rate)."""
    t0 = time.perf_counter()
    calls = 0
    while True:
        out = fn()
        calls += 1
        dt = time.perf_counter() - t0
        if dt >= min_s:
            return out, n_points * calls / dt


def _maxerr(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))


def cpu_leg(wl, n_v, n_t, n_ss, head, legs):
    """Oracle timings (all host cores, and one thread on a smaller sample) and
    the error of every leg against the oracle.  `head` holds the headline's
    GPU fluxes of the first SAMPLE_V vectors; `legs` maps a leg name to its
    payload."""
    import oracle
    oracle.build()
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    nv = min(SAMPLE_V, n_v)
    dt, p, (rm, rg) = run_oracle_step(wl, nv)
    cores = oracle.max_threads()
    n1 = max(1, nv // 16)
    dt1, p1, _ = run_oracle_step(wl, n1, n_threads=1)
    cpu = {"value": p / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d of %d vectors x %d times x %d supersamples, MA + Gimenez(N=%d, n_j=%d): %.1f s"
                     % (nv, n_v, n_t, n_ss, N_LD, N_J, dt),
           "value_1_thread": p1 / dt1,
           "sample_1_thread": "%d vectors, same times, one thread: %.1f s" % (n1, dt1)}
    # oracle rates per workload: all host cores and one thread, each on the leg's own check sample
    per = {"long_cadence": {"value": p / dt, "value_1_thread": p1 / dt1,
                            "unit": "flux points/s (MA + Gimenez N=8)"}}
    cpu["per_workload"] = per
    errs = {"headline": {"ma": _maxerr(head["fm"], rm[:, 0]), "gimenez": _maxerr(head["fg"], rg[:, 0]),
                         "sample": "first %d vectors, every time" % nv}}
    if "e2e_ssr" in legs:
        L = legs["e2e_ssr"]
        y = f32(L["y"])
        s_ma = oracle.ssr(rm, y)[:, 0]
        s_g = oracle.ssr(rg, y)[:, 0]
        errs["e2e_ssr"] = {"ma_rel": float(np.max(np.abs(L["ssr_ma"][:nv] - s_ma) / s_ma)),
                           "gimenez_rel": float(np.max(np.abs(L["ssr_g"][:nv] - s_g) / s_g)),
                           "sample": "first %d vectors (relative error of the residual sums)" % nv}
    if "plain" in legs:
        L = legs["plain"]
        t, orb, k, ld, _ = _oracle_sample(L["wl"], 1)
        (ref, _), r_all = _rate(lambda: oracle.lc_ma(t, orb, k, ld), len(t))
        _, r_one = _rate(lambda: oracle.lc_ma(t, orb, k, ld, n_threads=1), len(t))
        per["plain"] = {"value": r_all, "value_1_thread": r_one, "unit": "flux points/s (MA)",
                        "sample": "all %d times" % len(t)}
        errs["plain"] = {"ma": _maxerr(L["flux"], ref), "sample": "every point"}
    if "ma_interp" in legs:
        L = legs["ma_interp"]
        c = L["n_chk"]
        t, orb, k, ld, _ = _oracle_sample(wl, c)
        tab = oracle.MATable(float(np.float32(L["k_lo"])), float(np.float32(L["k_hi"])), 128, 256)
        ref_same, _ = oracle.lc_ma_interp(tab, t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"])
        errs["ma_interp"] = {"vs_oracle_same_method": _maxerr(L["flux"], ref_same[:, 0]),
                             "vs_oracle_exact": _maxerr(L["flux"], rm[:c, 0]),
                             "oracle_method_vs_exact": _maxerr(ref_same[:, 0], rm[:c, 0]),
                             "sample": "first %d vectors, every time" % c}
    if "gimenez_zi" in legs:
        L = legs["gimenez_zi"]
        c = L["n_chk"]
        t, orb, k, _, ldg = _oracle_sample(wl, c)
        ref_same, _ = oracle.lc_gimenez_zi(t, orb, k, ldg, N_J, L["n_in"], L["n_edge"], n_ss=n_ss, t_exp=wl["t_exp"])
        errs["gimenez_zi"] = {"vs_oracle_same_method": _maxerr(L["flux"], ref_same[:, 0]),
                              "vs_oracle_series": _maxerr(L["flux"], rg[:c, 0]),
                              "oracle_method_vs_series": _maxerr(ref_same[:, 0], rg[:c, 0]),
                              "sample": "first %d vectors, every time" % c}
    if "adjoint" in legs:
        L = legs["adjoint"]
        th = L["wl"]["theta"]
        names = ("t0", "P", "a", "b", "e", "w", "k", "u1", "u2")
        rows = np.stack([np.asarray(th[nm])[L["idx"]].astype(np.float64) if nm in ("t0", "P")
                         else f32(np.asarray(th[nm])[L["idx"]]) for nm in names], axis=1)
        n_pts = rows.shape[0] * len(L["wl"]["t"])
        (ssr_r, grad_r), r_all = _rate(lambda: oracle.ssr_grad(L["wl"]["t"], rows, f32(L["y"])), n_pts)
        _, r_one = _rate(lambda: oracle.ssr_grad(L["wl"]["t"], rows[:1], f32(L["y"]), n_threads=1),
                         len(L["wl"]["t"]))
        per["adjoint"] = {"value": r_all, "value_1_thread": r_one,
                          "unit": "flux points/s (residual sum + 9-component gradient)",
                          "sample": "%d vectors x %d times (one thread: 1 vector)" % (rows.shape[0], len(L["wl"]["t"]))}
        rel = np.abs(L["grad"] - grad_r) / np.maximum(np.abs(grad_r), 1e-30)
        # the scale of the sum: sum_t |2 (f - y) df/dtheta_i| (the gradient of t0 is a small
        # difference of ingress and egress terms, so |grad| alone overstates its error)
        yv = f32(L["y"])
        scale = np.zeros_like(grad_r)
        for j in range(rows.shape[0]):
            for ti, tt in enumerate(L["wl"]["t"]):
                f, gp = oracle.flux_grad(tt, rows[j])
                scale[j] += np.abs(2.0 * (f - yv[ti]) * gp)
        rels = np.abs(L["grad"] - grad_r) / np.maximum(scale, 1e-30)
        errs["adjoint"] = {"max_rel_per_component": {nm: float(rel[:, i].max()) for i, nm in enumerate(names)},
                           "median_rel_per_component": {nm: float(np.median(rel[:, i])) for i, nm in enumerate(names)},
                           "max_rel_to_term_scale_per_component": {nm: float(rels[:, i].max())
                                                                   for i, nm in enumerate(names)},
                           "ssr_max_rel": float(np.max(np.abs(L["ssr"] - ssr_r) / ssr_r)),
                           "sample": "%d seeded vectors, every time" % len(L["idx"])}
    if "batched" in legs:
        L = legs["batched"]
        bw = L["wl"]
        pairs = L["pairs"]
        o = bw["orbit"]
        orb = dict(t0=np.asarray(o["t0"])[pairs[:, 0]], P=np.asarray(o["P"])[pairs[:, 0]],
                   a=f32(o["a"])[pairs[:, 0]], inc=f32(o["inc"])[pairs[:, 0]])
        kp = f32(bw["k"])[pairs[:, 0], pairs[:, 1]][:, None]
        ldp = f32(bw["ld"])[pairs[:, 0], pairs[:, 1]][:, None, :]
        n_pts = len(pairs) * len(bw["t"])
        (ref, _), r_all = _rate(lambda: oracle.lc_ma(bw["t"], orb, kp, ldp), n_pts)
        o1 = {key: val[:1] for key, val in orb.items()}
        _, r_one = _rate(lambda: oracle.lc_ma(bw["t"], o1, kp[:1], ldp[:1], n_threads=1), len(bw["t"]))
        per["batched"] = {"value": r_all, "value_1_thread": r_one,
                          "unit": "flux points/s (MA, per-passband k)",
                          "sample": "%d (walker, passband) light curves x %d times (one thread: 1)"
                                    % (len(pairs), len(bw["t"]))}
        yy = f32(bw["y"])[pairs[:, 1]]
        ssr_ref = np.sum((yy - ref[:, 0]) ** 2, axis=1)
        e = {"ssr_max_rel": float(np.max(np.abs(L["ssr"] - ssr_ref) / ssr_ref)),
             "sample": "%d seeded (walker, passband) residual sums" % len(pairs)}
        w0 = dict(t0=np.asarray(o["t0"])[:1], P=np.asarray(o["P"])[:1], a=f32(o["a"])[:1], inc=f32(o["inc"])[:1])
        ref_k, _ = oracle.lc_ma_khat(bw["t"], w0, f32(bw["k"])[:1], f32(bw["ld"])[:1])
        e["khat_walker0_vs_oracle_khat"] = _maxerr(L["khat_flux_w0"], ref_k[0])
        if "interp_flux_w0" in L:
            ref_i, _ = oracle.lc_ma_interp(oracle.MATable(*L["interp_grid"]), bw["t"], w0, f32(bw["k"])[:1],
                                           f32(bw["ld"])[:1])
            ref_x, _ = oracle.lc_ma(bw["t"], w0, f32(bw["k"])[:1], f32(bw["ld"])[:1])
            e["interp_walker0_vs_oracle_interp"] = _maxerr(L["interp_flux_w0"], ref_i[0])
            e["interp_walker0_vs_oracle_exact"] = _maxerr(L["interp_flux_w0"], ref_x[0])
        if "cube" in L:
            worst = 0.0
            for v, cube in zip(L["cube_walkers"], L["cube"]):
                ov = dict(t0=np.asarray(o["t0"])[[v]], P=np.asarray(o["P"])[[v]], a=f32(o["a"])[[v]],
                          inc=f32(o["inc"])[[v]])
                ref_c, _ = oracle.lc_ma(bw["t"], ov, f32(bw["k"])[[v]], f32(bw["ld"])[[v]])
                worst = max(worst, _maxerr(cube, ref_c[0]))
            e["cube_max_abs"] = worst
            e["cube_sample"] = "walkers %s, all 64 passbands, every time" % L["cube_walkers"]
        errs["batched"] = e
    if "surrogate" in legs:
        L = legs["surrogate"]
        kk, zz = L["k"].astype(np.float64), L["z"].astype(np.float64)
        ref, r_all = _rate(lambda: oracle.ma_terms_batch(kk, zz), len(kk))
        n1 = min(len(kk), 100_000)
        _, r_one = _rate(lambda: oracle.ma_terms_batch(kk[:n1], zz[:n1], n_threads=1), n1)
        per["surrogate_domain"] = {"value": r_all, "value_1_thread": r_one,
                                   "unit": "(k, z) points/s (lambda_e, lambda_d, eta_d)",
                                   "sample": "%d points (one thread: %d)" % (len(kk), n1)}
        ref[:, 1] += np.where(kk > zz, 2.0 / 3.0, 0.0)

        def bound(terms, mask=None):
            b = (2 * np.abs(terms[0] - ref[:, 0]) + 4 * np.abs(terms[1] - ref[:, 1])
                 + 2 * np.abs(terms[2] - ref[:, 2]))
            return float(b.max()) if mask is None else float(b[mask].max()) if mask.any() else None

        s = L["served"]
        errs["surrogate"] = {"flux_err_bound_served": bound(L["surrogate"], s),
                             "flux_err_bound_all": bound(L["surrogate"]),
                             "flux_err_bound_exact_fp32": bound(L["exact"]),
                             "flux_err_bound_interp": bound(L["interp"]),
                             "bound": "2|d lambda_e| + 4|d lambda_d| + 2|d eta_d| against the FP64 oracle "
                                      "(the largest flux error over quadratic laws with q1, q2 in [0, 1])",
                             "sample": "%d seeded points, %d network-served" % (len(kk), int(s.sum()))}
    try:
        g = json.load(open(GOLDEN))
        worst = {int(k): v for k, v in g["priors_worst"].items()}
        errs["gimenez_truncation"] = {
            "n_j": N_J, "max_abs_vs_exact_over_priors": worst.get(N_J),
            "max_abs_vs_exact_over_priors_at_n_j_128": worst.get(128),
            "source": "tests/golden/gimenez_truncation.json (oracle series vs the occulted flux from its "
                      "definition; Sec. 2.1.1, Fig. 1 quantity)"}
    except Exception as exc:   # the study is a committed file; report its absence rather than fail
        errs["gimenez_truncation"] = {"error": str(exc)}
    return cpu, errs


def only_main(args):
    """One extra leg alone, at full or reduced size (profiler capture cases)."""
    import torch
    import paper_1504_07433_gb300 as pt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    pt.load_library(build_if_missing=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    K = args.steps
    if args.only == "adjoint":
        out, _ = bench_adjoint(pt, torch, dev, stream, K, flush, n_v=512 if args.small else 4096)
    elif args.only == "batched":
        out, _ = bench_batched(pt, torch, dev, stream, K, flush, n_walkers=64 if args.small else 1024,
                               modes=("ssr",) if args.small else ("ssr", "cube"))
    elif args.only == "plain":
        out, _ = bench_plain(pt, torch, dev, stream)
    else:
        out, _ = bench_surrogate(torch, dev, stream, n_infer=10_000_000 if args.small else 1_000_000_000,
                                 epochs=4 if args.small else 40, n_chk=10_000)
    print(json.dumps({"only": args.only, "small": bool(args.small), "result": out}), flush=True)
    return 0


def reference_main(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1504_07433_gb300 import workloads as W
    import oracle
    oracle.build()
    wl = W.long_cadence()
    n_t_sample = 12500
    for _ in range(args.warmup):
        run_oracle_step(wl, SAMPLE_V, n_t_sample)
    times, pts = [], 0
    for _ in range(args.steps):
        dt, p, _ = run_oracle_step(wl, SAMPLE_V, n_t_sample)
        times.append(dt)
        pts = p
    tot = float(np.sum(times))
    value = pts * args.steps / tot
    sample = "%d vectors x first %d times x %d supersamples, MA + Gimenez(N=%d, n_j=%d), per step" % (
        SAMPLE_V, n_t_sample, wl["n_ss"], N_LD, N_J)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "models": "MA quadratic + Gimenez N=%d n_j=%d" % (N_LD, N_J),
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the plain / interpolation / adjoint / batched / surrogate legs")
    ap.add_argument("--n-v", type=int, default=256, help="parameter vectors (smaller only for profiler captures)")
    ap.add_argument("--n-t", type=int, default=50000, help="exposure times (smaller only for profiler captures)")
    ap.add_argument("--n-j", type=int, default=N_J, help="Gimenez series depth (other values only for studies)")
    ap.add_argument("--only", default=None, choices=["adjoint", "batched", "surrogate", "plain"],
                    help="run one extra leg alone (profiler captures); prints its JSON object")
    ap.add_argument("--small", action="store_true", help="with --only: a reduced size for profiler captures")
    ap.add_argument("--heat-s", type=float, default=1.0,
                    help="seconds of extra untimed steps before the timed region, with the clock sampler running")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_main(args)

    import torch
    import torch.distributed as dist

    import paper_1504_07433_gb300 as pt
    from paper_1504_07433_gb300 import workloads as W

    if args.only:
        return only_main(args)
    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pt.load_library(build_if_missing=True)
    n_j = args.n_j

    wl = W.long_cadence(n_v=args.n_v, n_t=args.n_t)
    n_t, n_v, n_ss = wl["t"].size, wl["k"].size, wl["n_ss"]
    t = torch.as_tensor(wl["t"], dtype=torch.float64, device=dev)
    orb = pt.orbit_to_device(wl["orbit"], dev)
    k = torch.as_tensor(wl["k"], dtype=torch.float32, device=dev)
    ld = torch.as_tensor(wl["ld"], dtype=torch.float32, device=dev)
    ldg = torch.as_tensor(wl["ld_gim"], dtype=torch.float32, device=dev)
    plan = pt.GimenezPlan(N_LD, n_j)
    fm = torch.empty((n_v, 1, n_t), dtype=torch.float32, device=dev)
    fg = torch.empty_like(fm)
    wm = torch.empty(pt.ma_quad_work_bytes(n_t, n_v, 1), dtype=torch.uint8, device=dev)
    wg = torch.empty(plan.work_bytes(n_t, n_v, 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # the two models are independent evaluations of the same inputs: the
    # Mandel-Agol call runs on a second stream beside the Gimenez call, so
    # that each fills the SMs the other's small set-up kernels leave idle
    side = torch.cuda.Stream(device=dev)

    def step():
        e_in = torch.cuda.Event()
        e_in.record(stream)
        side.wait_event(e_in)
        with torch.cuda.stream(side):
            pt.ma_quad(t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"], work=wm, flux=fm)
        e_m = torch.cuda.Event()
        e_m.record(side)
        pt.gimenez(plan, t, orb, k, ldg, n_ss=n_ss, t_exp=wl["t_exp"], work=wg, flux=fg)
        stream.wait_event(e_m)

    # algorithmic work: in-transit (time, supersample, vector) evaluations, from the FP64-Newton z kernel
    zz, _ = pt.z_ecc(t, orb, n_ss=n_ss, t_exp=wl["t_exp"])
    n_intr = int((zz < (1.0 + k[:, None])).sum().item())
    del zz
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    ev = [_events(torch, 3) for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    h0 = time.perf_counter()
    while time.perf_counter() - h0 < args.heat_s:   # keeps the GPU busy while the sampler starts
        step()
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        step()
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = float(np.mean([ev[i][0].elapsed_time(ev[i][2]) for i in range(K)]))
    # each model alone (one stream, one after the other): the per-call times,
    # and the series-evaluation kernel's own time from events the library
    # records around its launch
    evk = [_events(torch, 2) for _ in range(K)]
    for i in range(K):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        pt.ma_quad(t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"], work=wm, flux=fm)
        ev[i][1].record(stream)
        plan.time_evaluation(evk[i][0], evk[i][1])
        pt.gimenez(plan, t, orb, k, ldg, n_ss=n_ss, t_exp=wl["t_exp"], work=wg, flux=fg)
        ev[i][2].record(stream)
    plan.time_evaluation()
    torch.cuda.synchronize()
    ma_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    g_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]
    k_ms = [evk[i][0].elapsed_time(evk[i][1]) for i in range(K)]
    pts_per_step = 2 * n_t * n_v * 1
    step_ms, value = whole_job_rate(step_ms, pts_per_step, ws, dev)
    head = {"fm": _host(fm[:SAMPLE_V, 0]), "fg": _host(fg[:SAMPLE_V, 0])}
    legs = {}

    # every parameter of a step in one pinned host buffer and one device buffer,
    # so that a step uploads them with a single copy
    par_np = {kk: np.asarray(wl["orbit"][kk], np.float64 if kk in ("t0", "P") else np.float32)
              for kk in ("t0", "P", "a", "inc", "e", "w")}
    par_np.update(k=np.asarray(wl["k"], np.float32), ld=np.asarray(wl["ld"], np.float32),
                  ldg=np.asarray(wl["ld_gim"], np.float32))
    offs, off = {}, 0
    for kk, v in par_np.items():
        offs[kk] = off
        off += (v.nbytes + 255) // 256 * 256
    par_bytes = off
    par_np_bytes = sum(v.nbytes for v in par_np.values())
    host_pack = torch.empty(par_bytes, dtype=torch.uint8).pin_memory()
    for kk, v in par_np.items():
        host_pack[offs[kk]:offs[kk] + v.nbytes].copy_(torch.from_numpy(v.view(np.uint8).ravel()))
    dev_pack = torch.empty(par_bytes, dtype=torch.uint8, device=dev)
    dv = {kk: dev_pack[offs[kk]:offs[kk] + v.nbytes].view(torch.float64 if v.dtype == np.float64 else torch.float32)
          .view(v.shape) for kk, v in par_np.items()}
    dev_par = {kk: dv[kk] for kk in ("t0", "P", "a", "inc", "e", "w")}
    k_d, ld_d, ldg_d = dv["k"], dv["ld"], dv["ldg"]

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_t = torch.as_tensor(wl["t"], dtype=torch.float64).pin_memory()
        # results come back on a copy stream while the next model computes:
        # device and pinned host outputs are double-buffered, and events
        # keep a buffer from being rewritten before its copy has finished
        out_m = [torch.empty(fm.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        out_g = [torch.empty(fg.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        fm2 = [fm, torch.empty_like(fm)]
        fg2 = [fg, torch.empty_like(fg)]
        cs = torch.cuda.Stream(device=dev)
        ev_m = [torch.cuda.Event() for _ in range(2)]
        ev_g = [torch.cuda.Event() for _ in range(2)]
        cp_m = [torch.cuda.Event() for _ in range(2)]
        cp_g = [torch.cuda.Event() for _ in range(2)]
        t_d = torch.empty_like(host_t, device=dev)
        h2d = host_t.numel() * 8 + par_np_bytes
        d2h = out_m[0].numel() * 4 + out_g[0].numel() * 4

        last_m = [None]

        def e2e_step(i):
            b = i % 2
            if last_m[0] is not None:   # the inputs are rewritten once the last MA call has read them
                stream.wait_event(last_m[0])
            t_d.copy_(host_t, non_blocking=True)
            dev_pack.copy_(host_pack, non_blocking=True)
            o = dict(dev_par)
            e_in = torch.cuda.Event()
            e_in.record(stream)
            side.wait_event(e_in)
            side.wait_event(cp_m[b])
            with torch.cuda.stream(side):
                pt.ma_quad(t_d, o, k_d, ld_d, n_ss=n_ss, t_exp=wl["t_exp"], work=wm, flux=fm2[b])
            ev_m[b].record(side)
            last_m[0] = ev_m[b]
            stream.wait_event(cp_g[b])
            pt.gimenez(plan, t_d, o, k_d, ldg_d, n_ss=n_ss, t_exp=wl["t_exp"], work=wg, flux=fg2[b])
            ev_g[b].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_m[b])
                out_m[b].copy_(fm2[b], non_blocking=True)
                cp_m[b].record(cs)
                cs.wait_event(ev_g[b])
                out_g[b].copy_(fg2[b], non_blocking=True)
                cp_g[b].record(cs)

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        e0, e1 = _events(torch, 2)
        e0.record(stream)
        for i in range(K):
            e2e_step(i)
        stream.wait_stream(cs)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1) / K
        e_ms, e_value = whole_job_rate(e_ms, pts_per_step, ws, dev)
        e2e = {"value": e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms}
        del out_m, out_g, fm2, fg2

    # the likelihood form (Sec. 3.4): observations stay on the device, each
    # step uploads the parameter vectors, evaluates both models with the
    # residual sums fused (no flux cube leaves the device) and reads the sums
    # back -- what a sampler does per proposal
    e2e_ssr = None
    if not args.no_e2e:
        rng = np.random.default_rng(3404)
        y_h = (1.0 + rng.normal(0.0, 1e-3, (1, n_t))).astype(np.float32)
        y_d = torch.as_tensor(y_h, device=dev)
        ssr_both = torch.empty((2, n_v, 1), dtype=torch.float32, device=dev)
        out_s = torch.empty((2, n_v, 1), dtype=torch.float32).pin_memory()

        def ssr_step():
            dev_pack.copy_(host_pack, non_blocking=True)
            o = dict(dev_par)
            e_in = torch.cuda.Event()
            e_in.record(stream)
            side.wait_event(e_in)
            with torch.cuda.stream(side):
                pt.ma_quad(t, o, k_d, ld_d, n_ss=n_ss, t_exp=wl["t_exp"], y=y_d, want_flux=False, want_ssr=True,
                           work=wm, ssr=ssr_both[0])
            e_m = torch.cuda.Event()
            e_m.record(side)
            pt.gimenez(plan, t, o, k_d, ldg_d, n_ss=n_ss, t_exp=wl["t_exp"], y=y_d, want_flux=False, want_ssr=True,
                       work=wg, ssr=ssr_both[1])
            stream.wait_event(e_m)
            out_s.copy_(ssr_both, non_blocking=True)

        # one step at a time with L2 flushed before each (outside the events),
        # as the device-side legs: this step's data (pair lists, times,
        # observations) would otherwise stay in L2 from one step to the next
        s_ms = _timed(torch, stream, K, flush, ssr_step)
        s_ms, s_value = whole_job_rate(s_ms, pts_per_step, ws, dev)
        e2e_ssr = {"value": s_value, "unit": UNIT, "h2d_bytes_per_step": int(par_np_bytes),
                   "d2h_bytes_per_step": int(out_s.numel() * 4), "ms_per_step": s_ms,
                   "form": "parameters up, residual sums of both models fused on the device, sums back; "
                           "L2 flushed before each step"}
        legs["e2e_ssr"] = {"y": y_h, "ssr_ma": out_s[0, :, 0].numpy().astype(np.float64),
                           "ssr_g": out_s[1, :, 0].numpy().astype(np.float64)}
        # the same two calls on the device alone (no copies), for comparison
        def ssr_dev():
            e_in = torch.cuda.Event()
            e_in.record(stream)
            side.wait_event(e_in)
            with torch.cuda.stream(side):
                pt.ma_quad(t, orb, k, ld, n_ss=n_ss, t_exp=wl["t_exp"], y=y_d, want_flux=False, want_ssr=True,
                           work=wm, ssr=ssr_both[0])
            e_m = torch.cuda.Event()
            e_m.record(side)
            pt.gimenez(plan, t, orb, k, ldg, n_ss=n_ss, t_exp=wl["t_exp"], y=y_d, want_flux=False,
                       want_ssr=True, work=wg, ssr=ssr_both[1])
            stream.wait_event(e_m)
        e2e_ssr["device_only_ms_per_step"] = _timed(torch, stream, K, flush, ssr_dev)

    # roofline of the dominant kernel (the Gimenez series evaluation):
    # algorithmic work = evaluating the N + 1 truncated series at each
    # in-transit (time, supersample, vector): one multiply-add per series
    # coefficient and order, 2 (N + 1) N_J FP32 flops.  The kernel executes
    # 2 (N + 2) N_J (the shared Chebyshev recurrence on top); the paper's
    # per-term Jacobi recursion (Sec. 2.1.4: the recursion a + b x, two
    # products, a sum and the accumulation T_j G_j, 7 flops per (n, j) term)
    # would spend 7 (N + 1) N_J: reported as a ratio, not as a rate.
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak_tflops = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    g_mean_ms = float(np.mean(g_ms))
    k_mean_ms = float(np.mean(k_ms))
    flops = 2.0 * (N_LD + 1) * n_j * n_intr
    exec_flops = 2.0 * (N_LD + 2) * n_j * n_intr
    paper_flops = 7.0 * (N_LD + 1) * n_j * n_intr
    achieved = flops / (k_mean_ms * 1e-3) / 1e12
    traffic = None
    if TRAFFIC["n_j"] == n_j and (n_t, n_ss) == (50000, 10):
        traffic = TRAFFIC["per_vector_bytes"] * n_v
    roofline = {"bound": "alu", "kernel": "gim_cheb_kernel (CUDA events recorded around its launch inside pt_gimenez)",
                "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu
                # capture of this kernel, per vector (times, pair lists, records and coefficient rows
                # all grow with the vectors); null unless the capture was taken at this depth
                "traffic": traffic,
                "traffic_source": "ncu capture of this kernel at n_j = %d, scaled per vector" % TRAFFIC["n_j"],
                "peak_source": "FP32 lanes %d SM x 128 x 2 flop x %.0f MHz (%s sm_max_mhz); of %s"
                               % (n_sm, sm_max, peak_src, peak_src),
                "algorithmic_flops_per_launch": flops, "in_transit_evaluations": n_intr,
                "kernel_ms": k_mean_ms, "call_ms": g_mean_ms,
                "call_frac": flops / (g_mean_ms * 1e-3) / 1e12 / fp32_peak_tflops,
                "executed_flops_per_launch": exec_flops,
                "executed_frac": exec_flops / (k_mean_ms * 1e-3) / 1e12 / fp32_peak_tflops,
                "paper_recursion_flops_ratio": paper_flops / flops}

    extra = {}
    launches = 10 * K   # MA: set-up, window, scan, pairs; Gimenez: table, coefficients, set-up, window, scan, series
    if not args.no_extra:
        extra["plain"], legs["plain"] = bench_plain(pt, torch, dev, stream)
        extra["ma_interp"], legs["ma_interp"] = bench_ma_interp(pt, torch, dev, stream, K, flush, t, orb, k, ld, wl, fm)
        extra["gimenez_zi"], legs["gimenez_zi"] = bench_gimenez_zi(pt, torch, dev, stream, K, flush, plan, t, orb, k,
                                                                   ldg, wl, fg)
        extra["adjoint"], legs["adjoint"] = bench_adjoint(pt, torch, dev, stream, K, flush)
        extra["batched"], legs["batched"] = bench_batched(pt, torch, dev, stream, K, flush)
        extra["surrogate"], legs["surrogate"] = bench_surrogate(torch, dev, stream)

    cpu = None
    max_err = None
    if rank == 0 and not args.no_cpu_baseline:
        if n_j == N_J:
            cpu, max_err = cpu_leg(wl, n_v, n_t, n_ss, head, legs)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
                "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["name"], "models": "MA quadratic + Gimenez N=%d n_j=%d" % (N_LD, n_j),
                           "n_t": n_t, "n_v": n_v, "n_ss": n_ss, "n_b": 1, "flux_points_per_step": pts_per_step,
                           "l2": "flushed between timed steps (256 MiB write outside the events)",
                           "parallelism": "replicas x%d" % ws},
                "components_ms": {"ma_quad": float(np.mean(ma_ms)), "gimenez": g_mean_ms},
                "max_abs_err_vs_oracle": max_err,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "e2e_ssr": e2e_ssr,
                **extra,
                "gpu_launches": launches, "clocks": dict(clocks, window="%.1f s of untimed steps + the timed region"
                                                         % args.heat_s) if clocks else None,
                "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
