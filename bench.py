#!/usr/bin/env python
"""Throughput of batched projection + backprojection inside the iterative solvers.

Workload (default, cgls_2048x1024_b16): 16 slices of 2048x2048 pixels, 1024
angles over [0, pi), 2048 detector bins; a seeded random-ellipsoid phantom with
analytic projections and 5% Gaussian noise; CGLS, 50 iterations per solve,
matrix values in BF16 with 16-bit column offsets (4.25 bytes per nonzero),
FP32 vectors and accumulation, FP64 dots and step scalars, the residual
recomputed every 10 iterations.  One step is one full CGLS solve of the
16-slice batch (interleave, 50 iterations replayed from CUDA graphs,
de-interleave).  The matrix is built once before timing (its build time is
reported separately).  `--workload sirt_512x360_b64` gives the SIRT line:
64 slices of 512x512, 360 angles, Poisson noise at 1e4 photons/ray, SIRT 100.

Metric: slice-iterations per second (one slice-iteration = one application of
A and of A^T to one slice plus the solver update), summed over all ranks.

The line also carries the roofline of the dominant SpMM pass, the plain FP32
CSR SpMV comparator, the end-to-end rate with host copies, the CPU oracle as a
baseline and (CGLS) the iterations each form needs to reach the FP64 oracle's
50-iteration data fit.

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]
Multi-GPU: one process per GPU (torchrun); every rank solves its own batch
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "proj+backproj slice-iters/s"
UNIT = "slice-iters/s"
DATA = ("synthetic: seeded random ellipsoids (16 per volume), analytic line integrals, "
        "Poisson noise at 1e4 photons/ray")
DATA_OF = {"sirt": DATA,
           "cgls": "synthetic: seeded random ellipsoids (16 per volume), analytic line integrals, 5% Gaussian noise"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="cgls_2048x1024_b16")
    p.add_argument("--batch-width", type=int, default=0, help="0 = autotuned")
    p.add_argument("--format", default="auto", choices=["auto", "sell", "sell16", "csr"],
                   help="matrix storage streamed by the kernels (auto: the workload's 16-bit form for CGLS, "
                        "autotuned over FP32 formats for SIRT)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip e2e / plain-CSR legs")
    p.add_argument("--col-blocks", type=int, default=-1,
                   help="16-bit A stored as this many bands of image rows (-1: enough bands that one band of "
                        "the gathered image batch fits in 48 MB of L2)")
    p.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                   help="N > 1: weak = every rank solves its own copy of the batch; strong = the batch's slices "
                        "are split over the ranks (Sec. 3.1's plan) and gathered on rank 0 inside the timed step")
    p.add_argument("--order", default="auto", choices=["auto", "rows", "tiles", "staged"],
                   help="row-group order of the A^T passes (same bits, different speed)")
    p.add_argument("--no-csr", action="store_true",
                   help="CGLS: build without the FP32 CSR pair (implies --no-extras: the comparators and the "
                        "accuracy leg need it); for hardware-counter captures in a few GB")
    p.add_argument("--iters", type=int, default=0, help="override the solver iterations (profiling runs)")
    p.add_argument("--no-graph", action="store_true", help="launch kernels directly (profiling runs)")
    p.add_argument("--model", default="line", choices=["line", "strip"],
                   help="matrix model: chord lengths (line) or areas in unit-width strips (strip)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def bus_id_of(dev):
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return None


# ---------------------------------------------------------------------------
# oracle (CPU) leg: the FP64 reference timed on the host cores
# ---------------------------------------------------------------------------
def oracle_sample(w, slices=1, iters=1, steps=1, warmup=0, model="line"):
    """Time oracle SIRT on a bounded sample of the workload; returns a dict."""
    import oracle
    from paper_2003_12677_b300 import inputs
    g = oracle.Geometry(w.n, w.n, w.n, w.n_theta, model=model)
    t0 = time.perf_counter()
    A = oracle.build_matrix(g)
    AT = A.transpose()
    build_s = time.perf_counter() - t0
    case = inputs.workload_case(w.name, slices=list(range(slices)))
    b = case.sino.reshape(slices, -1)
    for _ in range(warmup):
        oracle.sirt(A, AT, b, iters)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.sirt(A, AT, b, iters)
    dt = time.perf_counter() - t0
    return {"value": slices * iters * steps / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d slice(s) x %d SIRT iteration(s) x %d step(s) of the %s workload, FP64, matrix "
                      "stored (oracle build %.1f s untimed)" % (slices, iters, steps, w.name, build_s),
            "seconds": dt}


def oracle_sample_cgls(w, angle_stride=1, steps=1, warmup=0):
    """The oracle's matrix-free CGLS (its stored matrix would not fit in host
    memory at this size) timed on one slice: each step is one CGLS iteration
    (A p, A^T r and the vector updates) over every angle_stride-th angle of the
    workload, i.e. 1/angle_stride of a slice-iteration."""
    import numpy as np
    import oracle
    from paper_2003_12677_b300 import inputs
    th = np.arange(w.n_theta) * math.pi / w.n_theta
    sel = np.arange(0, w.n_theta, angle_stride)
    g = oracle.Geometry(w.n, w.n, w.n, len(sel), angles=th[sel] if angle_stride > 1 else None)
    case = inputs.workload_case(w.name, slices=[0])
    b = case.sino.reshape(w.n_theta, w.n)[sel].reshape(1, -1).astype(np.float64)
    p = case.phantom.reshape(1, -1).astype(np.float64)       # any search direction costs the same
    state = [np.zeros_like(p), b, p, np.ones(1), np.zeros(1, np.int32)]
    for _ in range(warmup):
        oracle.cgls_resume_mf(g, *state, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.cgls_resume_mf(g, *state, 1)
    dt = time.perf_counter() - t0
    share = len(sel) / w.n_theta
    return {"value": steps * share / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d step(s) of one matrix-free FP64 CGLS iteration of slice 0 of the %s workload over %d of "
                      "its %d angles (%.3g slice-iterations per step)" % (steps, w.name, len(sel), w.n_theta, share),
            "seconds": dt}


def oracle_sample_gd(w, slices=1):
    """The oracle's matrix-free loss and gradient (one projection and one
    backprojection per slice: one slice-iteration) timed on a bounded sample."""
    import numpy as np
    import oracle
    from paper_2003_12677_b300 import inputs
    g = oracle.Geometry(w.n, w.n, w.n, w.n_theta)
    case = inputs.workload_case(w.name, slices=list(range(slices)))
    x = np.zeros((slices, g.cols))
    b = case.sino.reshape(slices, -1)
    t0 = time.perf_counter()
    oracle.loss_grad_mf(g, x, b)
    dt = time.perf_counter() - t0
    return {"value": slices / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d slice(s) x one matrix-free FP64 loss-and-gradient evaluation (A x, A^T r, TV) of the %s "
                      "workload" % (slices, w.name), "seconds": dt}


def uneven_accuracy_leg(tomo, torch, reqs, pairs, iters, max_iters=45):
    """Config 5's FP32 vs BF16 comparison at equal accuracy (the data-fit
    reading of the CGLS bar): for slice 0 of one request per geometry with
    n <= 1024, the FP32-valued persistent CGLS sets the target (its data fit
    ||b - A x|| after `iters` iterations, to 1e-4) and the BF16-valued one is
    walked one launch per iteration until it reaches it.  Data fits come from
    tomo_residual_norm on the FP32 matrix (FP64 accumulation).  One geometry
    at a time, so that only one FP32 matrix is resident."""
    seen, rows = set(), []
    for i, r in enumerate(reqs):
        if r.n > 1024 or (r.n, r.n_theta) in seen:
            continue
        seen.add((r.n, r.n_theta))
        M32 = tomo.Matrix(r.n, r.n_theta, values="f32")   # SELL for the solve, CSR for the data fit
        sino = pairs[i][1][:1].contiguous()
        x32 = tomo.cgls_batched([(M32, sino)], iters, batch_width=16, fmt="sell")[0]
        target = float(tomo.residual_norm(M32, sino, x32)[0])
        xs, st = tomo.cgls_batched([(pairs[i][0], sino)], 0, batch_width=16, fmt="sell16", return_state=True)
        reach, fit_same = None, None
        for k in range(1, max_iters + 1):
            xs, st = tomo.cgls_batched([(pairs[i][0], sino)], 1, batch_width=16, fmt="sell16", resume=st,
                                       return_state=True)
            f = float(tomo.residual_norm(M32, sino, xs[0])[0])
            if k == iters:
                fit_same = f
            if reach is None and f <= target * (1 + 1e-4):
                reach = k
            if reach is not None and k >= iters:
                break
        rows.append({"n": r.n, "n_theta": r.n_theta, "fp32_fit": target, "bf16_fit_same_iters": fit_same,
                     "bf16_iters_to_fp32_fit": reach})
        del M32, x32, xs, st
        torch.cuda.empty_cache()
    ks = [t["bf16_iters_to_fp32_fit"] for t in rows if t["bf16_iters_to_fp32_fit"] is not None]
    return {"target": "FP32-valued persistent CGLS data fit after %d iterations, slice 0 of one request per "
                      "geometry with n <= 1024, to 1e-4" % iters,
            "geometries": len(rows), "reached": len(ks),
            "bf16_iters_max": max(ks) if ks else None, "bf16_iters_median": sorted(ks)[len(ks) // 2] if ks else None,
            "table": rows}


def oracle_sample_uneven(reqs):
    """The oracle's matrix-free CGLS, one iteration of the first slice of one
    request of each image size in the batch (its per-slice work spans 64x)."""
    import numpy as np
    import oracle
    from paper_2003_12677_b300 import inputs
    picks = {}
    for r in reqs:
        picks.setdefault(r.n, r)
    t, done = 0.0, []
    for n in sorted(picks):
        r = picks[n]
        g = oracle.Geometry(r.n, r.n, r.n, r.n_theta)
        b = inputs.make_case(r.n, r.n_theta, 1, r.seed, "ellipses2d", "poisson", 1e5).sino.reshape(1, -1)
        p = np.ones((1, g.cols))
        state = [np.zeros((1, g.cols)), b.astype(np.float64), p, np.ones(1), np.zeros(1, np.int32)]
        t0 = time.perf_counter()
        oracle.cgls_resume_mf(g, *state, 1)
        t += time.perf_counter() - t0
        done.append("%dx%d" % (r.n, r.n_theta))
    return {"value": len(done) / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "one matrix-free FP64 CGLS iteration of one slice of one request per image size (%s); the "
                      "batch's per-slice work varies with the size" % ", ".join(done), "seconds": t}


def oracle_sample_bb(w, slices, iters):
    """The oracle's BB-SIRT (Sec. 3.1) timed on a bounded sample of the workload."""
    import oracle
    from paper_2003_12677_b300 import inputs
    g = oracle.Geometry(w.n, w.n, w.n, w.n_theta)
    t0 = time.perf_counter()
    A = oracle.build_matrix(g)
    AT = A.transpose()
    build_s = time.perf_counter() - t0
    b = inputs.workload_case(w.name, slices=list(range(slices))).sino.reshape(slices, -1)
    t0 = time.perf_counter()
    oracle.sirt_bb(A, AT, w.n, b, iters)
    dt = time.perf_counter() - t0
    return {"value": slices * iters / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d slice(s) x %d BB-SIRT iteration(s) of the %s workload, FP64, matrix stored (oracle "
                      "build %.1f s untimed)" % (slices, iters, w.name, build_s), "seconds": dt}


def oracle_sample_fubini(w, slices, iters, solver):
    """The Fubini-Radon oracle timed on a bounded sample: a forward + adjoint
    pair per slice-iteration ("pair"), or its gridded BB-SIRT ("sirt")."""
    import oracle
    from oracle import fubini as fb
    from paper_2003_12677_b300 import inputs
    fg = fb.FGeometry(w.n, w.n, w.n_theta)
    t0 = time.perf_counter()
    S = fb.gridding_matrix(fg)
    build_s = time.perf_counter() - t0
    case = inputs.workload_case(w.name, slices=list(range(slices)))
    t0 = time.perf_counter()
    if solver == "pair":
        x = case.phantom.reshape(slices, -1)
        for _ in range(iters):
            fb.fubini_backproject(fg, fb.fubini_project(fg, x, S), S)
    else:
        fb.fubini_sirt_bb(fg, case.sino.reshape(slices, -1), iters, S)
    dt = time.perf_counter() - t0
    what = ("forward + adjoint pair(s)" if solver == "pair" else
            "iteration(s) of the oracle's gridded BB-SIRT (its SIRT with the exact normal operator sums the "
            "exact transform: minutes per slice-iteration at this size, so the gridded one, equal up to the "
            "gridding error, stands in)")
    return {"value": slices * iters / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d slice(s) x %d %s of the %s workload, FP64 with numpy's FFT (gridding matrix %.1f s "
                      "untimed)" % (slices, iters, what, w.name, build_s), "seconds": dt}


def spmm_roofline(M, B, fmt, tm, kinds, torch, local, clk):
    """Roofline of the dominant SpMM pass from the per-kernel CUDA-event
    timing tm: algorithmic bytes (matrix once, gathered vector once, the
    epilogue's own reads and writes, kinds[k] = (name, extra vector bytes per
    row-or-column of the output, per slice)) over its average launch time."""
    kind = 0 if tm.ms[0] >= tm.ms[1] else 1
    avg_ms = tm.ms[kind] / max(tm.launches[kind], 1)
    rows, cols, nnz = M.rows, M.cols, M.nnz
    bnnz = 4.25 if fmt == "sell16" else 8
    mat_bytes = (rows + 1 if kind == 0 else cols + 1) * 8 + nnz * bnnz
    gathered_len, out_len = (cols, rows) if kind == 0 else (rows, cols)
    name, out_vecs = kinds[kind]
    alg = mat_bytes + gathered_len * B * 4 + out_vecs * out_len * B * 4
    peak, src = measured_peaks()
    achieved = alg / (avg_ms / 1000.0) / 1e9
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    gathered = nnz * B * 4
    roof = {"bound": "hbm", "kernel": name % ((KERNEL[fmt], B) if "%s" in name else (B,)), "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": src + " (burst copy)",
            "alg_bytes_per_launch": alg, "avg_launch_ms": avg_ms,
            "kernel_share": tm.ms[kind] / max(sum(tm.ms[k] for k in range(3)), 1e-12)}
    ceil = {"operand_delivery": {"achieved": gathered / (avg_ms / 1000.0) / 1e9, "unit": "GB/s",
                                 "peak": sms * 128 * mhz * 1e6 / 1e9, "bytes_per_launch": gathered,
                                 "peak_source": "128 B/clk/SM x %d SMs x median SM clock" % sms}}
    for c in ceil.values():
        c["frac"] = c["achieved"] / c["peak"]
    return roof, ceil


KERNEL = {"sell": "sell", "sell16": "sell16", "csr": "f32"}


def workload_config(w, B, fmt, model="line"):
    return {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "n_p": w.n, "slices": w.n_z, "model": model,
            "solver": w.solver, "iters": w.iters, "batch_width": B, "format": fmt,
            "values": (w.values if w.values != "f32" else "bf16") if fmt == "sell16" else "f32",
            "l2": "working set larger than L2: A and A^T are streamed from HBM every iteration"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if w.solver == "cgls":
        # a whole CGLS iteration of one slice takes ~20 s on 16 host cores, so each
        # step samples one eighth of its angles
        res = oracle_sample_cgls(w, angle_stride=8, steps=args.steps, warmup=args.warmup)
        cfg = workload_config(w, min(16, w.n_z), "sell16" if w.values != "f32" else "sell", args.model)
    else:
        res = oracle_sample(w, slices=4, iters=2, steps=args.steps, warmup=args.warmup, model=args.model)
        cfg = workload_config(w, 0, "sell", args.model)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * res["seconds"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA_OF.get(w.solver, DATA), "config": cfg,
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# alternate workloads (not the default line): CGLS with 16-bit values,
# TV-regularised gradient descent through autograd, the uneven batch
# ---------------------------------------------------------------------------
def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(bus_id_of(torch.cuda.current_device()))
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clocks.stop()


def _rasterize_gpu(ell, n, device):
    """Sum of ellipse densities at pixel centres (input synthesis on the GPU)."""
    import torch
    c = torch.arange(n, device=device, dtype=torch.float32) + 0.5 - n / 2
    Y, X = torch.meshgrid(c, c, indexing="ij")
    img = torch.zeros((n, n), device=device)
    for x0, y0, A, B_, phi, rho in ell:
        cph, sph = math.cos(phi), math.sin(phi)
        u = (X - x0) * cph + (Y - y0) * sph
        v = -(X - x0) * sph + (Y - y0) * cph
        img += rho * (((u / A) ** 2 + (v / B_) ** 2) <= 1.0).float()
    return img


def run_alternate(args, w):
    import numpy as np
    import torch
    import paper_2003_12677_b300 as tomo
    from paper_2003_12677_b300 import inputs

    torch.cuda.set_device(0)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None}
    if args.workload == "uneven_256":
        reqs = inputs.uneven_requests()
        geos = sorted({(r.n, r.n_theta) for r in reqs}, key=lambda g: -g[0] * g[0] * g[1])
        t0 = time.perf_counter()
        # the persistent solver streams the 16-bit SELL pair (no tiled A^T copy); A in
        # column bands where a 16-slice image batch exceeds 48 MB (the default line's rule)
        def nbands(nn):
            return args.col_blocks if args.col_blocks >= 0 else max(1, math.ceil(nn * nn * 16 * 4 / (48 << 20)))
        mats = {g: tomo.Matrix(g[0], g[1], values="bf16", fp32_sell=False, keep_csr=False, at_tiles=False,
                               col_blocks=min(nbands(g[0]), 64, g[0])) for g in geos}
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        pairs = []
        for r in reqs:
            M = mats[(r.n, r.n_theta)]
            rng = np.random.default_rng(r.seed)
            ph = torch.stack([_rasterize_gpu(inputs.random_ellipses(r.n, rng), r.n, "cuda") for _ in range(r.n_z)])
            p = tomo.project(M, ph.contiguous(), batch_width=4, fmt="sell16")
            s = 2.0 / p.amax(dim=(1, 2), keepdim=True).clamp_min(1e-6)
            g = torch.Generator(device="cuda").manual_seed(r.seed)
            counts = torch.poisson(1e5 * torch.exp(-s * p), generator=g)
            pairs.append((M, (-torch.log(counts.clamp_min(1.0) / 1e5) / s).contiguous()))
            del ph, p, counts
        iters = args.iters or 30
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # drop the input-synthesis temporaries before the large workspace
        ws = {"ws": None}

        def step():
            ws["out"] = None
            ws["out"] = tomo.cgls_batched(pairs, iters, batch_width=16, fmt="sell16", workspace=ws["ws"])

        from paper_2003_12677_b300 import _lib as _l
        import ctypes as _ct
        _reqs = (_l.Request * len(pairs))()
        for i, (M_, s_) in enumerate(pairs):
            _reqs[i].A, _reqs[i].n_z = M_.handle.value, s_.shape[0]
            _reqs[i].sino, _reqs[i].x = s_.data_ptr(), s_.data_ptr()
        _o = _l.ExecOpts()
        _o.batch_width, _o.format = 16, 1
        _nb = _ct.c_size_t()
        _l.call("tomo_cgls_batched_workspace", _reqs, len(pairs), _ct.byref(_o), _ct.byref(_nb))
        ws["ws"] = torch.empty(_nb.value, dtype=torch.uint8, device="cuda")

        ms, clk = _timed(step, args.steps, args.warmup)
        slices = sum(r.n_z for r in reqs)
        line.update({"value": slices * iters / (ms / 1000.0), "ms_per_step": ms, "dtype": "f32-accumulate/bf16-values",
                     "data": "synthetic: 256 seeded requests, random-ellipse phantoms rasterised on the GPU, "
                             "projected, Poisson noise at 1e5 photons/ray",
                     "config": {"workload": "uneven_256", "requests": len(reqs), "geometries": len(geos),
                                "slices": slices, "iters": iters, "solver": "cgls (one persistent launch)",
                                "batch_width": 16, "format": "sell16", "nnz_total": sum(m.nnz for m in mats.values()),
                                "workspace_bytes": ws["ws"].numel(),
                                "device_bytes_in_use": torch.cuda.mem_get_info()[1] - torch.cuda.mem_get_info()[0]},
                     "clocks": clk, "build_s": build_s, "gpu_launches": args.steps})
        # roofline of the persistent launch over its algorithmic bytes: per
        # iteration and packed batch of 16 slices, both 16-bit matrices once
        # (4.25 B/nnz) and the CGLS vectors (q, r, p, s, x streams of 4 B)
        per_geo = {}
        for r in reqs:
            per_geo[(r.n, r.n_theta)] = per_geo.get((r.n, r.n_theta), 0) + r.n_z
        alg = 0.0
        for g, nzs in per_geo.items():
            M_ = mats[g]
            batches = math.ceil(nzs / 16)
            alg += iters * batches * (2 * M_.nnz * 4.25 + (5 * M_.rows + 7 * M_.cols) * 16 * 4)
        peak, src = measured_peaks()
        ach = alg / (ms / 1000.0) / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": "k_cgls_persistent<16, SELL16> (the whole batched solve)",
                            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                            "peak_source": src + " (burst copy)", "alg_bytes_per_launch": alg,
                            "avg_launch_ms": ms}
        if not args.no_extras:
            ws["ws"] = ws["out"] = None
            torch.cuda.empty_cache()
            line["accuracy"] = uneven_accuracy_leg(tomo, torch, reqs, pairs, 30)   # config 5's 30 iterations
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample_uneven(reqs)
        print(json.dumps(line))
        return 0

    case = inputs.workload_case(args.workload)
    sino = torch.from_numpy(case.sino).cuda()
    if w.solver == "fubini":
        t0 = time.perf_counter()
        F = tomo.Fubini(w.n, w.n_theta)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        x = torch.from_numpy(case.phantom).cuda()
        iters = args.iters or 10
        y = torch.empty_like(sino)

        def step():
            for _ in range(iters):
                yy = F.project(x)
                F.backproject(yy)

        ms, clk = _timed(step, args.steps, args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        F.backproject(sino, filtered=True)
        e0.record()
        for _ in range(iters):
            F.backproject(sino, filtered=True)
        e1.record()
        torch.cuda.synchronize()
        fbp_ms = e0.elapsed_time(e1) / iters
        line.update({"value": w.n_z * iters / (ms / 1000.0), "ms_per_step": ms, "dtype": "f32 (complex64 FFTs)",
                     "data": DATA, "config": {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "slices": w.n_z,
                                              "iters": iters, "operator": "Fubini-Radon: 2D FFT, Kaiser-Bessel "
                                              "gridding SpMM (kw = 6), 1D FFTs (register FFTs at this size); "
                                              "one forward + one adjoint per slice-iteration"},
                     "clocks": clk, "build_s": build_s, "fbp": {"ms_per_64_slices": fbp_ms,
                                                               "slices_per_s": w.n_z / (fbp_ms / 1000.0)},
                     # per 16-slice group: forward rows, columns, S, radial; adjoint
                     # radial, short and long rows of S^T, columns, rows
                     "gpu_launches": args.steps * iters * 9 * math.ceil(w.n_z / 16)})
        # whole-pair roofline over modelled bytes: the compulsory reads and writes
        # per slice of each kernel that runs at this size (power-of-two grid and
        # n_p: register-FFT passes), S / S^T read once per 16-slice group.
        # Forward: rows (image in, n x G complex out), columns (those in, the
        # G x G spectrum out), S (spectrum in, polar samples out), radial
        # (samples in, sinogram out); the adjoint the same in reverse.
        G, rows_p = 2 * w.n, w.n_theta * w.n
        img, mid, grid_c, pol_c, sino_b = w.n * w.n * 4, w.n * G * 8, G * G * 8, rows_p * 8, rows_p * 4
        per_slice_dir = (img + mid) + (mid + grid_c) + (grid_c + pol_c) + (pol_c + sino_b)
        mat = 2 * (rows_p * 36 * 8) / 16
        bytes_step = iters * w.n_z * (2 * per_slice_dir + mat)
        peak, src = measured_peaks()
        ach = bytes_step / (ms / 1000.0) / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": "forward + adjoint, all kernels (modelled bytes)",
                            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                            "peak_source": src + " (burst copy)", "alg_bytes_per_slice_iter": bytes_step / (
                                iters * w.n_z)}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample_fubini(w, slices=16, iters=6, solver="pair")
        print(json.dumps(line))
        return 0
    if w.solver == "fubini_normal":
        t0 = time.perf_counter()
        F = tomo.Fubini(w.n, w.n_theta)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        iters = args.iters or w.iters
        t0 = time.perf_counter()
        F.normal(sino.new_zeros((1, w.n, w.n)), "hamming")  # taps and their spectrum, once
        torch.cuda.synchronize()
        taps_s = time.perf_counter() - t0

        def step():
            F.sirt_bb_normal(sino, iters)

        ms, clk = _timed(step, args.steps, args.warmup)
        mg, _ = _timed(lambda: F.sirt_bb(sino, iters), 1, 1)
        x = torch.from_numpy(case.phantom).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        F.normal(x, "hamming")
        e0.record()
        for _ in range(10):
            F.normal(x, "hamming")
        e1.record()
        torch.cuda.synchronize()
        n_ms = e0.elapsed_time(e1) / 10
        xn, hn = F.sirt_bb_normal(sino, iters, history=True)
        xg = F.sirt_bb(sino, iters)
        dev = float(torch.linalg.vector_norm(xn - xg) / torch.linalg.vector_norm(xg))
        line.update({"value": w.n_z * iters / (ms / 1000.0), "ms_per_step": ms, "dtype": "f32 (FP32 FFTs)",
                     "data": DATA, "config": {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "slices": w.n_z,
                                              "iters": iters, "solver": "SIRT, Hamming-ramp preconditioned, BB "
                                              "step; normal operator in one step (2n x 2n convolution)"},
                     "clocks": clk, "build_s": build_s, "taps_s": taps_s,
                     "normal_apply": {"ms_per_64_slices": n_ms, "slices_per_s": w.n_z / (n_ms / 1000.0)},
                     "gridded_sirt_bb": {"value": w.n_z * iters / (mg / 1000.0), "unit": UNIT,
                                         "form": "the same SIRT projecting and backprojecting every iteration"},
                     "vs_gridded": {"speedup": mg / ms, "iterate_rel_diff": dev,
                                    "gradnorm_ratio_last_first": float((hn[-1] / hn[0]).median())},
                     # this library's kernels per solve (cuFFT's not counted): the filtered
                     # backprojection of b, then per iteration a pad, product and gradient
                     # kernel per pass of 32 slices (none at x = 0) and one step kernel
                     "gpu_launches": args.steps * (5 * math.ceil(w.n_z / 16) + 2
                                                   + (iters - 1) * (3 * math.ceil(w.n_z / 32) + 1))})
        # roofline of one application of N (the three fused passes) over the
        # compulsory bytes: rows (image read, half spectrum H written), columns
        # (H read and written), inverse rows (H read, result written); and the
        # FFT arithmetic, 5 L log2 L flops per length-L complex transform
        n = w.n
        L = 2 * n
        H = (n + 1) * n * 8
        nbytes = w.n_z * (n * n * 4 + H + 2 * H + H + n * n * 4)
        nflops = w.n_z * (n // 2 + 2 * (n + 1) + n // 2) * 5 * L * math.log2(L)
        peak, src = measured_peaks()
        ach = nbytes / (n_ms / 1000.0) / 1e9
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2032.0
        fpeak = sms * 128 * 2 * mhz * 1e6 / 1e12
        line["roofline"] = {"bound": "hbm", "kernel": "normal operator: k_cv_rows + k_cv_cols + k_cv_rows_inv",
                            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                            "peak_source": src + " (burst copy)", "alg_bytes_per_launch": nbytes,
                            "avg_launch_ms": n_ms}
        line["ceilings"] = {"fp32": {"achieved": nflops / (n_ms / 1000.0) / 1e12, "unit": "TFLOP/s",
                                     "peak": fpeak, "peak_source": "128 FP32 FMA/clk/SM",
                                     "frac": nflops / (n_ms / 1000.0) / 1e12 / fpeak}}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample_fubini(w, slices=8, iters=12, solver="sirt")
        print(json.dumps(line))
        return 0
    if w.solver == "sirt_bb":
        fmt = args.format if args.format != "auto" else "sell"
        t0 = time.perf_counter()
        M = tomo.Matrix(w.n, w.n_theta)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        B = args.batch_width or 64
        iters = args.iters or w.iters
        x = torch.empty((w.n_z, w.n, w.n), device="cuda")
        wsb = torch.empty(M.workspace_size(4, w.n_z, B, fmt), dtype=torch.uint8, device="cuda")

        def step():
            tomo.sirt_bb(M, sino, iters, batch_width=B, fmt=fmt, out=x, workspace=wsb)

        ms, clk = _timed(step, args.steps, args.warmup)
        tm = tomo.new_timing()
        tomo.sirt_bb(M, sino, iters, batch_width=B, fmt=fmt, out=x, workspace=wsb, timing=tm)
        tot = sum(tm.ms[k] for k in range(3))
        # convergence against the classical SIRT of the default line (100 iterations)
        xs = tomo.sirt(M, sino, 100, batch_width=B, fmt=fmt)
        r100 = torch.linalg.vector_norm((tomo.project(M, xs) - sino).reshape(w.n_z, -1), dim=1)
        _, h = tomo.sirt_bb(M, sino, iters + 1, history=True, batch_width=B, fmt=fmt)
        below = (h[1:] <= r100[None, :].double())  # h[k] = ||b - A x_k||, k = 1..iters
        first = [int(torch.nonzero(below[:, z]).min()) + 1 if bool(below[:, z].any()) else None
                 for z in range(w.n_z)]
        reached = [f for f in first if f is not None]
        line.update({"value": w.n_z * iters / (ms / 1000.0), "ms_per_step": ms, "dtype": "f32",
                     "data": DATA, "config": {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "slices": w.n_z,
                                              "iters": iters, "solver": "SIRT, Hamming-ramp preconditioned, BB step",
                                              "batch_width": B, "format": fmt},
                     "clocks": clk, "build_s": build_s, "nnz": M.nnz, "gpu_launches": args.steps * int(
                         sum(tm.launches[k] for k in range(3))),
                     "time_split": {"A": tm.ms[0] / tot, "A^T": tm.ms[1] / tot, "filter+vector+scalar": tm.ms[2] / tot},
                     # A pass: r = b - A x (b read, r written); A^T pass: g = A^T P^T P r (g written)
                     **dict(zip(("roofline", "ceilings"), spmm_roofline(
                         M, B, fmt, tm, [("k_spmm_%s<%d, EpiResidual> (A pass)", 2),
                                         ("k_spmm_%s<%d, EpiStore> (A^T pass)", 1)], torch,
                         torch.cuda.current_device(), clk))),
                     "convergence": {"classical_sirt_100_resid_median": float(r100.median()),
                                     "bb_iters_to_reach_it": {"median": sorted(reached)[len(reached) // 2]
                                                              if reached else None,
                                                              "max": max(reached) if reached else None,
                                                              "slices_reached": len(reached)}}})
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample_bb(w, slices=8, iters=20)
        print(json.dumps(line))
        return 0
    # gradient descent on ||A x - b||^2 + mu TV(x) through the autograd Function
    t0 = time.perf_counter()
    M = tomo.Matrix(w.n, w.n_theta)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    B = args.batch_width or 32
    iters = args.iters or w.iters
    mu, eps = 1e-3, 1e-3
    # step size 1/(2 sigma_max^2): power iteration on A^T A (20 steps)
    v = torch.rand((1, w.n, w.n), device="cuda")
    for _ in range(20):
        v = tomo.backproject(M, tomo.project(M, v))
        lam = v.norm().item()
        v = v / lam
    eta = 1.0 / (2.0 * lam + 8.0 * mu / eps)
    x = torch.zeros((w.n_z, w.n, w.n), device="cuda")

    def step():
        xs = x.clone().requires_grad_(True)
        for _ in range(iters):
            r = tomo.radon(xs, M, batch_width=B) - sino
            loss = (r * r).sum() + mu * tomo.tv_loss(xs, eps)
            g, = torch.autograd.grad(loss, xs)
            with torch.no_grad():
                xs -= eta * g
        return xs

    ms, clk = _timed(step, args.steps, args.warmup)
    line.update({"value": w.n_z * iters / (ms / 1000.0), "ms_per_step": ms, "dtype": "f32",
                 "data": "synthetic: seeded random ellipsoids, analytic line integrals, 5% Gaussian noise",
                 "config": {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "slices": w.n_z, "iters": iters,
                            "solver": "gradient descent on ||Ax-b||^2 + 1e-3 TV through torch.autograd",
                            "batch_width": B, "format": "sell", "step": eta},
                 "clocks": clk, "build_s": build_s, "nnz": M.nnz})
    # roofline of the dominant SpMM pass: the autograd step runs one projection
    # (forward) and one backprojection (backward) per iteration, the same
    # kernels as this timed pair on the same batch
    tm = tomo.new_timing()
    yy = tomo.project(M, x, batch_width=B, timing=tm)
    tomo.backproject(M, yy, batch_width=B, timing=tm)
    line["roofline"], line["ceilings"] = spmm_roofline(
        M, B, "sell", tm, [("k_spmm_%s<%d, EpiStore> (A pass, forward)", 1),
                           ("k_spmm_%s<%d, EpiStore> (A^T pass, backward)", 1)], torch, torch.cuda.current_device(), clk)
    line["gpu_launches"] = args.steps * iters * 2 * (3 * math.ceil(w.n_z / B)) + args.steps * iters
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample_gd(w, slices=1)
    print(json.dumps(line))
    return 0


def cusparse_leg(M, B, torch):
    """The paper's GPU path as context: the same A and A^T (exported CSR) as
    torch sparse CSR tensors, y = A x and x' = A^T y through cuSPARSE SpMM
    (torch.sparse.mm) at batch width B and as SpMV (width 1).  No solver
    update is included, which favours this leg slightly."""
    def csr(transpose):
        rp, col, val = M.export_csr(transpose=transpose)
        n = len(rp) - 1
        return torch.sparse_csr_tensor(torch.from_numpy(rp.astype("int32")), torch.from_numpy(col),
                                       torch.from_numpy(val), size=(n, M.rows if transpose else M.cols)).cuda()

    A, AT = csr(False), csr(True)
    out = {"unit": UNIT, "form": "torch.sparse.mm on CSR (cuSPARSE SpMM / SpMV), A and A^T stored"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for width, reps in ((B, 10), (1, 10)):
        x = torch.rand((M.cols, width), device="cuda")
        for _ in range(3):
            y = torch.sparse.mm(A, x)
            x = torch.sparse.mm(AT, y)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            y = torch.sparse.mm(A, x)
            x = torch.sparse.mm(AT, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["value" if width == B else "value_width1"] = width / (ms / 1000.0)
        out["batch_width" if width == B else "spmv_width"] = width
    del A, AT
    torch.cuda.empty_cache()
    return out


def kernel_hash():
    """Hash of the code the SpMM passes and their matrix layouts compile from
    (the solver kernels, their device building blocks, the handle's layout
    constants and the matrix build), with comments and blank space removed:
    stored DRAM counters are used only while it is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2003_12677_b300", "csrc")
    for f in ("ops.cu", "spmm.cuh", "internal.cuh", "build.cu"):
        with open(os.path.join(d, f)) as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def code_only(src):
    """C / CUDA source without its comments, blank space collapsed."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_names(solver, fmt, B, staged=False):
    """(name template, output vectors read or written per output row and slice) of the
    A pass (kind 0) and the A^T pass (kind 1) of a solver's iteration; staged: the
    A^T pass is the tiled 16-bit one (detector windows staged in shared memory)."""
    at = "k_spmm_tile16<%d, %s> (A^T pass, staged tiles" if staged else "k_spmm_%s<%d, %s> (A^T pass"
    if solver == "sirt":   # r = R o (b - A x): b read, r written; x += lam C o A^T r: x read + written
        return [("k_spmm_%s<%d, EpiSirtResidual> (A pass)", 2),
                (at.replace("%s>", "EpiSirtUpdate>", 1) + ")", 2)]
    # CGLS: q = A p and s = A^T r, each written once with its squared norm
    return [("k_spmm_%s<%d, EpiStoreNorm> (A pass, q = A p)", 1),
            (at.replace("%s>", "EpiStoreNorm>", 1) + ", s = A^T r)", 1)]


def golden_fit(w):
    """The oracle's stored data-fit history of slice 0 (tests/golden), if any."""
    path = os.path.join(ROOT, "tests", "golden", "%s_slice0.json" % w.name.rsplit("_", 1)[0])
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def accuracy_leg(tomo, torch, M, w, sino, B, fmt, rate, plain_rate, max_iters=90):
    """Iterations each form needs to reach the FP64 oracle's 50-iteration data
    fit ||b - A x_50|| of slice 0 (stored by tests/golden/make_cgls_2048.py),
    to 1e-4: the benchmarked batch (slice 0 of it) and the plain FP32 CSR
    SpMV form.  The data fit of every GPU iterate is tomo_residual_norm (FP64
    accumulation).  CGLS iterates are not reproducible one by one past the
    first few in any precision (FP32 runs lag the FP64 one by a few
    iterations), so the forms are compared at equal data fit."""
    gold = golden_fit(w)
    if gold is None:
        return {"error": "no stored oracle data fit for %s" % w.name}
    k50 = 50
    target = gold["resnorm"][k50 - 1] * (1 + 1e-4)
    b0 = sino[:1].contiguous()
    rws = M._workspace(5, 1, 0, "sell")
    idx = torch.tensor(gold["sample_index"], device="cuda", dtype=torch.int64)

    def walk(sino_in, bw, f, recompute):
        x, st = tomo.cgls(M, sino_in, 0, batch_width=bw, fmt=f, return_state=True)
        fits, samples = [], {}
        for k in range(1, max_iters + 1):
            rc = recompute if (recompute and k % 10 == 0) else 0
            x, st = tomo.cgls(M, sino_in, 1, recompute_every=rc, batch_width=bw, fmt=f, resume=st,
                              return_state=True)
            fit = float(tomo.residual_norm(M, b0, x[:1].contiguous(), workspace=rws)[0])
            fits.append(fit)
            if str(k) in gold.get("samples", {}):
                ref = torch.tensor([float(v) for v in gold["samples"][str(k)]], device="cuda", dtype=torch.float64)
                got = x[0].reshape(-1)[idx].double()
                samples[str(k)] = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
            if fit <= target and k >= k50:
                return k, fits, samples
        return None, fits, samples

    k_b, fits_b, samp_b = walk(sino, B, fmt, 1)          # the benchmarked batch and form (recompute every 10)
    k_p, fits_p, samp_p = walk(b0, 1, "csr", 0)          # the plain FP32 CSR SpMV form, one slice
    out = {"target": "FP64 oracle's data fit ||b - A x_50|| of slice 0, to 1e-4 (matrix-free oracle, stored)",
           "target_fit": target, "oracle_fit_by_iter": {str(k): gold["resnorm"][k - 1] for k in (1, 10, 25, 50)},
           "iters_to_target": {"%s_b%d" % (fmt, B): k_b, "plain_f32_csr": k_p},
           "fit_at_50": {"%s_b%d" % (fmt, B): fits_b[k50 - 1] if len(fits_b) >= k50 else None,
                         "plain_f32_csr": fits_p[k50 - 1] if len(fits_p) >= k50 else None},
           "first_iterates_rel_l2_sampled": {"%s_b%d" % (fmt, B): samp_b, "plain_f32_csr": samp_p,
                                             "pixels": len(gold["sample_index"])}}
    if k_b and k_p:
        t_b, t_p = k_b / rate, k_p / plain_rate
        out["seconds_per_slice_to_target"] = {"%s_b%d" % (fmt, B): t_b, "plain_f32_csr": t_p}
        out["speedup_at_same_accuracy"] = t_p / t_b
    return out


def run_main(args, w):
    """SIRT or CGLS over the workload's slice batch: the metric line."""
    import torch
    import torch.distributed as dist
    import paper_2003_12677_b300 as tomo
    from paper_2003_12677_b300 import inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    cgls = w.solver == "cgls"
    tomo.set_launch(order=args.order)
    fmt = args.format
    if cgls and fmt == "auto":
        fmt = "sell16" if w.values != "f32" else "sell"
    values = (w.values if w.values != "f32" else "bf16") if fmt == "sell16" else "f32"
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if cgls:   # the 16-bit pair streamed by the solve, the FP32 CSR pair for the comparators and the data fit
        if args.no_csr:
            args.no_extras = True
        bw = args.batch_width or min(16, w.n_z)
        bands = args.col_blocks if args.col_blocks >= 0 else (
            max(1, math.ceil(w.n * w.n * bw * 4 / (48 << 20))) if fmt == "sell16" else 0)
        M = tomo.Matrix(w.n, w.n_theta, values=values, fp32_sell=fmt == "sell", keep_csr=not args.no_csr,
                        model=args.model, col_blocks=min(bands, 64, w.n) if fmt == "sell16" else 0)
    else:
        M = tomo.Matrix(w.n, w.n_theta, values=values, model=args.model)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    tune = None
    if cgls:
        if fmt == "sell16" and args.batch_width == 0:
            tune = M.autotune(w.n_z, allow_16bit="only")   # the workload's 16-bit values
            B = tune["batch_width"]
        else:
            B = args.batch_width or min(16, w.n_z)
    elif args.batch_width == 0 or fmt == "auto":
        tune = M.autotune(w.n_z)
        B = args.batch_width or tune["batch_width"]
        if fmt == "auto":
            fmt = tune["format"]
    else:
        B = args.batch_width

    case = inputs.workload_case(args.workload)
    sino = torch.from_numpy(case.sino).cuda()
    x = torch.zeros((w.n_z, w.n, w.n), device="cuda")
    op = 3 if cgls else 2
    wsb = torch.empty(M.workspace_size(op, w.n_z, B, fmt), dtype=torch.uint8, device="cuda")
    graph = not args.no_graph
    recompute = 10 if cgls else 0

    def solve(sn, out, timing=None):
        if cgls:
            tomo.cgls(M, sn, w.iters, recompute_every=recompute, batch_width=B, fmt=fmt, out=out, workspace=wsb,
                      use_graph=graph, timing=timing)
        else:
            tomo.sirt(M, sn, w.iters, batch_width=B, fmt=fmt, out=out, workspace=wsb, use_graph=graph,
                      timing=timing)

    def step():
        solve(sino, x)

    strong = args.scaling == "strong"
    if strong:
        # one stack over all ranks: each solves its slices (whole-stack batch width kept), rank 0 gathers
        from paper_2003_12677_b300.distributed import solve_sharded

        def solve_part(sn):
            out = torch.empty((sn.shape[0], w.n, w.n), device="cuda")
            solve(sn, out)
            return out

        def step():  # noqa: F811
            solve_sharded(solve_part, sino, out_shape=(w.n, w.n))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(bus_id_of(local))
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    units_per_step = (1 if strong else world) * w.n_z * w.iters
    value = units_per_step / (ms / 1000.0)

    dtype = "f32" if fmt != "sell16" else "f32-accumulate/%s-values" % values
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if strong else "weak",
            "vs_baseline": None, "dtype": dtype, "data": DATA_OF[w.solver],
            "config": workload_config(w, B, fmt, args.model), "clocks": clk, "build_s": build_s, "nnz": M.nnz}
    if cgls:
        line["config"]["solver"] = "cgls, FP64 dots and step scalars, residual recomputed every %d" % recompute
        if fmt == "sell16":
            line["config"]["col_blocks"] = min(bands, 64, w.n)
    if tune is not None:
        line["autotune"] = {"chosen": [tune["batch_width"], tune["format"], tune["order"], tune["blocks_per_sm"]],
                            "columns": ["batch_width", "format", "A^T order", "blocks per SM (0 = all)",
                                        "slice-iters/s of a SIRT pair"],
                            "table": [[t["batch_width"], t["format"], t["order"], t["blocks_per_sm"],
                                       round(t["slice_iters_per_s"])] for t in tune["table"]]}

    # per-kernel device time of one extra solve (CUDA events around every launch)
    tm = tomo.new_timing()
    solve(sino, x, tm)
    launches = int(sum(tm.launches[k] for k in range(3)))
    line["gpu_launches"] = launches * args.steps
    tot = sum(tm.ms[k] for k in range(3))
    line["time_split"] = {"A": tm.ms[0] / tot, "A^T": tm.ms[1] / tot, "vector+scalar": tm.ms[2] / tot}
    # average device time of one pass of each kind (CUDA events around every launch)
    line["pass_ms"] = {"A": tm.ms[0] / max(tm.launches[0], 1), "A^T": tm.ms[1] / max(tm.launches[1], 1),
                       "passes_per_solve": {"A": int(tm.launches[0]), "A^T": int(tm.launches[1])}}
    # the A^T pass streams the tiled 16-bit A^T when the resolved order is "staged"
    staged = (fmt == "sell16" and B == 16 and M.has_at_tiles and
              (args.order == "staged" or (args.order == "auto" and (tune is None or tune["order"] in ("staged", "auto")))))
    line["config"]["at_order"] = "staged" if staged else (tune["order"] if tune and args.order == "auto" else args.order)
    kinds = kernel_names(w.solver, fmt, B, staged)
    roof, ceil = spmm_roofline(M, B, fmt, tm, kinds, torch, local, clk)
    kind = 0 if tm.ms[0] >= tm.ms[1] else 1
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        key = "%s/B%d/%s/k%d" % (w.name, B, fmt, kind)
        if key in tj.get("per_launch_bytes", {}):
            if tj.get("kernel_hash") == kernel_hash():
                roof["traffic"] = tj["per_launch_bytes"][key]
            else:
                sys.stderr.write("bench: stored DRAM counters (profiles/traffic.json) predate the current SpMM "
                                 "sources: roofline traffic reported as null\n")
                roof["traffic_note"] = "stored DRAM counters predate the current kernels"
    line["roofline"] = roof
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    ceil["fma"] = {"achieved": 2.0 * M.nnz * B / (roof["avg_launch_ms"] / 1000.0) / 1e12, "unit": "TFLOP/s",
                   "peak": sms * 128 * 2 * mhz * 1e6 / 1e12, "peak_source": "128 FP32 FMA/clk/SM"}
    ceil["fma"]["frac"] = ceil["fma"]["achieved"] / ceil["fma"]["peak"]
    line["ceilings"] = ceil
    bnnz = 4.25 if fmt == "sell16" else 8
    vec = (3 * M.rows + 3 * M.cols) if not cgls else (5 * M.rows + 7 * M.cols)
    step_bytes = w.iters * ((M.rows + M.cols + 2) * 8 + 2 * M.nnz * bnnz + vec * B * 4) * math.ceil(w.n_z / B)
    line["hbm_gbs_step"] = step_bytes / (ms / 1000.0) / 1e9

    if not args.no_extras:
        # end to end through the public API: pinned host sinogram in, tomogram out
        sino_h = torch.from_numpy(case.sino).pin_memory()
        x_h = torch.empty((w.n_z, w.n, w.n), pin_memory=True)
        sd = torch.empty_like(sino)

        def e2e_step():
            sd.copy_(sino_h, non_blocking=True)
            solve(sd, x)
            x_h.copy_(x, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            e2e_step()
        e1.record()
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / args.steps
        line["e2e"] = {"value": units_per_step / (ems / 1000.0), "unit": UNIT,
                       "h2d_bytes_per_step": sino_h.numel() * 4, "d2h_bytes_per_step": x_h.numel() * 4,
                       "ms_per_step": ems}

        # the plain FP32 CSR SpMV form (one slice per pass) on the same GPU
        nzp, itp = (1, 5) if cgls else (4, 10)
        xp = torch.zeros((nzp, w.n, w.n), device="cuda")
        sp = sino[:nzp].contiguous()
        wsp = torch.empty(M.workspace_size(op, nzp, 1, "csr"), dtype=torch.uint8, device="cuda")

        def plain():
            if cgls:
                tomo.cgls(M, sp, itp, batch_width=1, out=xp, workspace=wsp, fmt="csr")
            else:
                tomo.sirt(M, sp, itp, batch_width=1, out=xp, workspace=wsp, fmt="csr")

        plain()
        torch.cuda.synchronize()
        e0.record()
        plain()
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        line["plain_f32_csr"] = {"value": world * nzp * itp / (pms / 1000.0), "unit": UNIT,
                                 "form": "FP32 CSR SpMV (batch width 1, warp per row)",
                                 "sample": "%d slice(s) x %d %s iterations" % (nzp, itp, w.solver.upper())}
        line["speedup_vs_plain_f32_csr"] = value / line["plain_f32_csr"]["value"]
        if cgls and rank == 0:
            line["accuracy"] = accuracy_leg(tomo, torch, M, w, sino, B, fmt, value / world,
                                            line["plain_f32_csr"]["value"] / world)
        if not cgls:
            try:
                line["cusparse_f32_csr"] = cusparse_leg(M, B, torch)
            except Exception as e:  # context only, never fatal for the GPU number
                line["cusparse_f32_csr"] = {"error": str(e)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            if cgls:
                line["cpu_baseline"] = oracle_sample_cgls(w, angle_stride=1)
            else:
                line["cpu_baseline"] = oracle_sample(w, slices=8, iters=48, steps=1, model=args.model)
        except Exception as e:  # reported, never fatal for the GPU number
            line["cpu_baseline"] = {"error": str(e)}

    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    from paper_2003_12677_b300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.iters:
        import dataclasses
        w = dataclasses.replace(w, iters=args.iters)
    if args.impl == "reference":
        return run_reference(args, w)
    if w.solver in ("sirt", "cgls") and args.workload != "uneven_256":
        return run_main(args, w)
    return run_alternate(args, w)


if __name__ == "__main__":
    sys.exit(main())
