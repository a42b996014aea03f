#!/usr/bin/env python
"""Throughput of batched projection + backprojection inside SIRT.

Workload (default): 64 slices of 512x512 pixels, 360 angles over [0, pi), 512
detector bins; seeded random-ellipsoid phantom with analytic projections and
Poisson noise at 1e4 photons/ray; SIRT, 100 iterations per solve.  One step is
one full SIRT solve of the 64-slice batch (interleave, 100 iterations of the
fused A / A^T passes replayed from a CUDA graph, de-interleave).  The matrix is
built once before timing (its build time is reported separately).

Metric: slice-iterations per second (one slice-iteration = one application of
A and of A^T to one slice plus the SIRT update), summed over all ranks.

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU: one process per GPU (torchrun); every rank solves its own batch
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sirt_512x360_b64")
    p.add_argument("--batch-width", type=int, default=0, help="0 = autotuned")
    p.add_argument("--format", default="auto", choices=["auto", "sell", "sell16", "csr"],
                   help="matrix storage streamed by the kernels (auto = autotuned over FP32 formats)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip e2e / plain-CSR legs")
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
    roof = {"bound": "hbm", "kernel": name % (KERNEL[fmt], B), "achieved": achieved, "peak": peak, "unit": "GB/s",
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
    res = oracle_sample(w, slices=4, iters=2, steps=args.steps, warmup=args.warmup, model=args.model)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * res["seconds"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": workload_config(w, 0, "sell", args.model),
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
        mats = {g: tomo.Matrix(g[0], g[1], values="bf16", fp32_sell=False, keep_csr=False) for g in geos}
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
                                              "gridding SpMM (kw = 6), 1D FFTs; one forward + one adjoint per "
                                              "slice-iteration"},
                     "clocks": clk, "build_s": build_s, "fbp": {"ms_per_64_slices": fbp_ms,
                                                               "slices_per_s": w.n_z / (fbp_ms / 1000.0)},
                     "gpu_launches": args.steps * iters * 2 * 7 * math.ceil(w.n_z / 16)})
        # whole-pair roofline over modelled bytes: every kernel's compulsory reads
        # and writes per slice, each cuFFT 2D transform as two passes over the
        # complex G x G grid, 1D transforms as one pass, S / S^T read once per
        # 16-slice group
        G, rows_p = 2 * w.n, w.n_theta * w.n
        grid_c, pol_c = G * G * 8, rows_p * 8
        per_slice_dir = (w.n * w.n * 4 + grid_c) + 4 * grid_c + 2 * grid_c + grid_c + pol_c \
            + 2 * pol_c + 2 * pol_c + (pol_c + rows_p * 4)
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
    if w.solver == "cgls":
        fmt = args.format if args.format != "auto" else "sell16"
        t0 = time.perf_counter()
        M = tomo.Matrix(w.n, w.n_theta, values=w.values, fp32_sell=False)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        B = args.batch_width or 16
        iters = args.iters or w.iters
        x = torch.empty((w.n_z, w.n, w.n), device="cuda")
        wsb = torch.empty(M.workspace_size(3, w.n_z, B, fmt), dtype=torch.uint8, device="cuda")

        def step():
            tomo.cgls(M, sino, iters, recompute_every=10, batch_width=B, fmt=fmt, out=x, workspace=wsb)

        ms, clk = _timed(step, args.steps, args.warmup)
        value = w.n_z * iters / (ms / 1000.0)
        # FP32 comparators on the same GPU: CSR at the same width, and the plain SpMV form
        xc = torch.empty_like(x)
        wsc = torch.empty(M.workspace_size(3, w.n_z, B, "csr"), dtype=torch.uint8, device="cuda")
        mc, _ = _timed(lambda: tomo.cgls(M, sino, 5, batch_width=B, fmt="csr", out=xc, workspace=wsc), 1, 1)
        x1 = torch.empty((1, w.n, w.n), device="cuda")
        ws1 = torch.empty(M.workspace_size(3, 1, 1, "csr"), dtype=torch.uint8, device="cuda")
        m1, _ = _timed(lambda: tomo.cgls(M, sino[:1].contiguous(), 3, batch_width=1, fmt="csr", out=x1, workspace=ws1),
                       1, 1)
        line.update({"value": value, "ms_per_step": ms, "dtype": "f32-accumulate/%s-values" % w.values,
                     "data": "synthetic: seeded random ellipsoids, analytic line integrals, 5% Gaussian noise",
                     "config": {"workload": w.name, "n": w.n, "n_theta": w.n_theta, "slices": w.n_z, "iters": iters,
                                "solver": "cgls, residual recomputed every 10", "batch_width": B, "format": fmt},
                     "clocks": clk, "build_s": build_s, "nnz": M.nnz,
                     "fp32_csr_same_width": {"value": w.n_z * 5 / (mc / 1000.0), "unit": UNIT},
                     "plain_f32_csr": {"value": 3 / (m1 / 1000.0), "unit": UNIT,
                                       "form": "FP32 CSR SpMV (batch width 1, warp per row)"}})
        line["speedup_vs_plain_f32_csr"] = value / line["plain_f32_csr"]["value"]
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
    """Hash of the sources the SpMM kernels compile from (the solver kernels
    and their device building blocks): stored DRAM counters are used only
    while it is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2003_12677_b300", "csrc")
    for f in ("ops.cu", "spmm.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    args = parse()
    from paper_2003_12677_b300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.iters:
        import dataclasses
        w = dataclasses.replace(w, iters=args.iters)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist
    import paper_2003_12677_b300 as tomo

    if w.solver != "sirt" or args.workload == "uneven_256":
        return run_alternate(args, w)

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    fmt = args.format
    values = (w.values if w.values != "f32" else "bf16") if fmt == "sell16" else "f32"
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M = tomo.Matrix(w.n, w.n_theta, values=values, model=args.model)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    tune = None
    if args.batch_width == 0 or fmt == "auto":
        tune = M.autotune(w.n_z)
        B = args.batch_width or tune["batch_width"]
        if fmt == "auto":
            fmt = tune["format"]
    else:
        B = args.batch_width

    case = inputs.workload_case(args.workload)
    sino = torch.from_numpy(case.sino).cuda()
    x = torch.zeros((w.n_z, w.n, w.n), device="cuda")
    wsb = torch.empty(M.workspace_size(2, w.n_z, B, fmt), dtype=torch.uint8, device="cuda")

    graph = not args.no_graph

    def step():
        tomo.sirt(M, sino, w.iters, batch_width=B, fmt=fmt, out=x, workspace=wsb, use_graph=graph)

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
    units_per_step = world * w.n_z * w.iters
    value = units_per_step / (ms / 1000.0)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fmt != "sell16" else "f32-accumulate/%s-values" % values,
            "data": DATA, "config": workload_config(w, B, fmt, args.model), "clocks": clk,
            "build_s": build_s, "nnz": M.nnz}
    if tune is not None:
        line["autotune"] = {"chosen": [tune["batch_width"], tune["format"]],
                            "table": [[t["batch_width"], t["format"], round(t["slice_iters_per_s"])]
                                      for t in tune["table"]]}

    # per-kernel device time of one extra solve (CUDA events around every launch)
    tm = tomo.new_timing()
    tomo.sirt(M, sino, w.iters, batch_width=B, fmt=fmt, out=x, workspace=wsb, timing=tm)
    launches = int(sum(tm.launches[k] for k in range(3)))
    line["gpu_launches"] = launches * args.steps
    kind = 0 if tm.ms[0] >= tm.ms[1] else 1
    avg_ms = tm.ms[kind] / max(tm.launches[kind], 1)
    rows, cols, nnz = M.rows, M.cols, M.nnz
    bnnz = 4.25 if fmt == "sell16" else 8
    mat_bytes = (rows + 1 if kind == 0 else cols + 1) * 8 + nnz * bnnz
    if kind == 0:   # r = R o (b - A x): matrix, x gathered once, b, R, r
        vec_bytes = cols * B * 4 + 2 * rows * B * 4 + rows * 4
        kname = "k_spmm_%s<%d, EpiSirtResidual> (A pass)" % (KERNEL[fmt], B)
    else:           # x += lambda C o A^T r: matrix, r gathered once, x read+write, C
        vec_bytes = rows * B * 4 + 2 * cols * B * 4 + cols * 4
        kname = "k_spmm_%s<%d, EpiSirtUpdate> (A^T pass)" % (KERNEL[fmt], B)
    alg = mat_bytes + vec_bytes
    peak, src = measured_peaks()
    achieved = alg / (avg_ms / 1000.0) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        key = "%s/B%d/%s/k%d" % (w.name, B, fmt, kind)
        if tj.get("kernel_hash") == kernel_hash() and key in tj.get("per_launch_bytes", {}):
            traffic = tj["per_launch_bytes"][key]
    line["roofline"] = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic, "peak_source": src + " (burst copy)",
                        "alg_bytes_per_launch": alg, "avg_launch_ms": avg_ms,
                        "kernel_share": tm.ms[kind] / max(sum(tm.ms[k] for k in range(3)), 1e-12)}
    # the two on-chip ceilings beside HBM: gathered-operand delivery (each
    # nonzero brings B*4 bytes of the gathered vector row through L1, at most
    # 128 B per clock per SM) and FP32 FMA (2 flops per nonzero per slice)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    gathered = nnz * B * 4
    line["ceilings"] = {
        "operand_delivery": {"achieved": gathered / (avg_ms / 1000.0) / 1e9, "unit": "GB/s",
                             "peak": sms * 128 * mhz * 1e6 / 1e9, "bytes_per_launch": gathered,
                             "peak_source": "128 B/clk/SM x %d SMs x median SM clock" % sms},
        "fma": {"achieved": 2.0 * nnz * B / (avg_ms / 1000.0) / 1e12, "unit": "TFLOP/s",
                "peak": sms * 128 * 2 * mhz * 1e6 / 1e12, "peak_source": "128 FP32 FMA/clk/SM"}}
    for c in line["ceilings"].values():
        c["frac"] = c["achieved"] / c["peak"]
    step_bytes = w.iters * ((rows + cols + 2) * 8 + 2 * nnz * bnnz
                            + (3 * rows + 3 * cols) * B * 4) * math.ceil(w.n_z / B)
    line["hbm_gbs_step"] = step_bytes / (ms / 1000.0) / 1e9

    if not args.no_extras:
        # end to end through the public API: pinned host sinogram in, tomogram out
        sino_h = torch.from_numpy(case.sino).pin_memory()
        x_h = torch.empty((w.n_z, w.n, w.n), pin_memory=True)
        sd = torch.empty_like(sino)

        def e2e_step():
            sd.copy_(sino_h, non_blocking=True)
            tomo.sirt(M, sd, w.iters, batch_width=B, fmt=fmt, out=x, workspace=wsb)
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
        nzp, itp = 4, 10
        xp = torch.zeros((nzp, w.n, w.n), device="cuda")
        wsp = torch.empty(M.workspace_size(2, nzp, 1, "csr"), dtype=torch.uint8, device="cuda")
        sp = sino[:nzp].contiguous()
        tomo.sirt(M, sp, itp, batch_width=1, out=xp, workspace=wsp, fmt="csr")
        torch.cuda.synchronize()
        e0.record()
        tomo.sirt(M, sp, itp, batch_width=1, out=xp, workspace=wsp, fmt="csr")
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        line["plain_f32_csr"] = {"value": world * nzp * itp / (pms / 1000.0), "unit": UNIT,
                                 "form": "FP32 CSR SpMV (batch width 1, warp per row)",
                                 "sample": "%d slices x %d SIRT iterations" % (nzp, itp)}
        line["speedup_vs_plain_f32_csr"] = value / line["plain_f32_csr"]["value"]
        try:
            line["cusparse_f32_csr"] = cusparse_leg(M, B, torch)
        except Exception as e:  # context only, never fatal for the GPU number
            line["cusparse_f32_csr"] = {"error": str(e)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_sample(w, slices=8, iters=48, steps=1, model=args.model)
        except Exception as e:  # reported, never fatal for the GPU number
            line["cpu_baseline"] = {"error": str(e)}

    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
