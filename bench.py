#!/usr/bin/env python
"""Benchmark: Fresnel planes/s of the six-plane relay at 4096^2 (complex64) on GB300.

One step = one pass of the relay system (obscured + spidered pupil generated in the first
pass, lens 5 m, PSD surface, lens 2 m, PSD surface, field stop; five angular-spectrum hops of
0.5-5 m), i.e. 5 Fresnel planes, run through libcoro's fused plan (11 launches).

Printed JSON (one line, rank 0): value = planes/s over all ranks (replicas: every rank runs its
own system, no collective on the data path), device-timed with CUDA events; e2e = the same
through host buffers (PSD maps host->device and the output field device->host inside the
timed region); roofline of the dominant pass kind against the measured HBM copy bandwidth;
the FP64 oracle timed on host cores as cpu_baseline; the plain GPU form (torch.fft + torch
elementwise, complex64) for comparison; and, when the library has it, the Lyot coronagraph
PSF rate.

``--impl reference`` times the FP64 oracle (the slow plain program) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coronagraph PSFs/s & Fresnel planes/s at 4096² vs plain GPU form; % of roofline"
UNIT = "planes/s"
HOPS = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="coro", choices=["coro", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.lines: list[str] = []
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ helpers

def measured_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def pass_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("fft_engine.cuh", "passes.cuh", "passes_launch.cuh", "passes_f32.cu"):
        with open(os.path.join(ROOT, "paper_1806_06467_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind: str) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernels."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != pass_source_hash():
        return None
    return t.get(kind, {}).get("dram_bytes_per_launch")


def relay_setup(n: int, seed: int, device):
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    w = inputs.RelayWorkload(n=n, npix=n // 4, seed=seed)
    maps_np = [m.astype(np.float32) for m in w.psd_maps()]
    maps = [torch.from_numpy(m).to(device) for m in maps_np]
    r = w.diam_m / 2
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=r, obscuration=w.obscuration,
                        n_spiders=w.n_spiders, spider_width=w.spider_width_frac * w.diam_m),
           coro.element(coro.EL_LENS, plane=1, focal_length=w.lens1_m),
           coro.element(coro.EL_OPD_MAP, plane=2, opd=maps[0]),
           coro.element(coro.EL_LENS, plane=3, focal_length=w.lens2_m),
           coro.element(coro.EL_OPD_MAP, plane=4, opd=maps[1]),
           coro.element(coro.EL_CIRCLE, plane=5, radius=w.field_stop_frac * r)]
    return w, maps_np, maps, els


# ------------------------------------------------------------------------------ oracle arms

def oracle_hop_runner(n: int, seed: int):
    """One plane of the relay per call on the FP64 oracle: element, then an AS hop."""
    import numpy as np

    from oracle import optics, propagation
    from paper_1806_06467_gb300 import inputs
    w = inputs.RelayWorkload(n=n, npix=n // 4, seed=seed)
    m0, m1 = w.psd_maps()
    r = w.diam_m / 2
    z = w.distances()
    state = {"e": np.ones((n, n), complex), "p": 0}

    def element(p):
        dx, lam = w.dx, w.wavelength_m
        if p == 0:
            return optics.circular_aperture(n, dx, r, w.obscuration, w.n_spiders, w.spider_width_frac * w.diam_m)
        if p == 1:
            return optics.thin_lens(n, dx, lam, w.lens1_m)
        if p == 2:
            return optics.phasor(m0, lam)
        if p == 3:
            return optics.thin_lens(n, dx, lam, w.lens2_m)
        return optics.phasor(m1, lam)

    def step():
        p = state["p"] % HOPS
        if p == 0:
            state["e"] = np.ones((n, n), complex)
        e = state["e"] * element(p)
        state["e"] = propagation.angular_spectrum(e, w.dx, w.wavelength_m, z[p])
        state["p"] += 1

    return step


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    step = oracle_hop_runner(args.n, 0)
    t0 = time.perf_counter()
    step()                                      # calibrate one sample
    t_one = time.perf_counter() - t0
    warm = max(0, min(args.warmup, 1))
    for _ in range(warm):
        step()
    # bounded: at most ~150 s of timed oracle work whatever --steps asks
    k = max(1, min(args.steps, int(150.0 / max(t_one, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    dt = time.perf_counter() - t0
    value = k / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": k, "warmup": warm, "ms_per_step": 1e3 * dt / k, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"relay6_{args.n}", "n": args.n, "planes_per_step": 1,
                      "note": "FP64 numpy oracle, one element + angular-spectrum hop per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{k} single {args.n}^2 planes of the relay (FP64 oracle)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(n: int) -> dict:
    step = oracle_hop_runner(n, 0)
    step()
    k, t0 = 0, time.perf_counter()
    while k < 2 or time.perf_counter() - t0 < 8.0:
        step()
        k += 1
        if k >= 4:
            break
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} planes (element + angular-spectrum hop) of the {n}^2 relay, FP64 numpy"}


# ------------------------------------------------------------------------------ plain GPU form

def plain_gpu(n: int, maps_np, w, steps: int, warmup: int, device) -> dict:
    """Unfused torch form: precomputed complex64 element and transfer arrays, torch.fft."""
    import torch

    # element and transfer arrays built once (FP64 torch on the device), outside the timed region
    dx, lam = w.dx, w.wavelength_m
    r = w.diam_m / 2
    k = torch.arange(n, device=device, dtype=torch.float64) - n // 2
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    r2 = k2 * (dx * dx)
    x = (k * dx)[None, :].expand(n, n)
    y = (k * dx)[:, None].expand(n, n)

    def phase(ph):
        return torch.polar(torch.ones_like(ph), ph).to(torch.complex64)

    half = w.spider_width_frac * w.diam_m / 2
    ro = w.obscuration * r
    ap = (r2 <= r * r) & ~(r2 < ro * ro) & ~((x.abs() < half) | (y.abs() < half))
    stop = r2 <= (w.field_stop_frac * r) ** 2
    maps_t = [torch.from_numpy(m).to(device).double() for m in maps_np]
    els_t = [ap.to(torch.complex64), phase(-torch.pi * r2 / (lam * w.lens1_m)), phase(2 * torch.pi * maps_t[0] / lam),
             phase(-torch.pi * r2 / (lam * w.lens2_m)), phase(2 * torch.pi * maps_t[1] / lam), stop.to(torch.complex64)]
    hs = [torch.fft.ifftshift(phase(-torch.pi * lam * z * k2 / (n * dx) ** 2)) for z in w.distances()]

    def step():
        e = torch.ones((n, n), dtype=torch.complex64, device=device)
        for p in range(6):
            e = e * els_t[p]
            if p < HOPS:
                e = torch.fft.fftshift(torch.fft.ifft2(hs[p] * torch.fft.fft2(torch.fft.ifftshift(e))))
        return e

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"value": HOPS * 1e3 / ms, "unit": UNIT, "ms_per_step": ms,
            "form": "torch.fft.fft2/ifft2 (cuFFT) + torch elementwise complex64, unfused, per hop"}


# ------------------------------------------------------------------------------ main arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)

    from paper_1806_06467_gb300 import build, coro
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()

    ctx = coro.Context(local)
    stream = torch.cuda.current_stream(device)
    n = args.n
    w, maps_np, maps, els = relay_setup(n, seed=rank, device=device)
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=els, init_uniform=True)
    n_pass = plan.launch_count
    info = [plan.pass_info(i) for i in range(n_pass)]
    field = torch.empty((1, n, n), dtype=torch.complex64, device=device)

    for _ in range(args.warmup):
        plan.execute(field)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    # -------- timed region: K steps, one event between consecutive passes
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_pass + 1)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        evs[k][0].record(stream)
        for i in range(n_pass):
            plan.execute_range(field, i, 1)
            evs[k][i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(evs[k][0].elapsed_time(evs[k][n_pass]) for k in range(args.steps))
    per_pass = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(n_pass)] for k in range(args.steps)])
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    value = HOPS * args.steps * world / (t_max / 1e3)

    # -------- roofline of the dominant pass kind
    kinds = {"row": [0.0, 0.0, 0], "col": [0.0, 0.0, 0]}
    for i, (is_row, nbytes) in enumerate(info):
        kk = "row" if is_row else "col"
        kinds[kk][0] += per_pass[:, i].sum()
        kinds[kk][1] += nbytes * args.steps
        kinds[kk][2] += args.steps
    dom = max(kinds, key=lambda k: kinds[k][0])
    t_dom, b_dom, l_dom = kinds[dom]
    peak, peak_src = measured_peaks()
    achieved = b_dom / (t_dom / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(dom), "kernel": f"{dom}_pass_kernel",
                "bytes_per_launch": b_dom / l_dom, "us_per_launch": 1e3 * t_dom / l_dom,
                "time_share": t_dom / per_pass.sum(), "peak_source": f"{peak_src} hbm_gbs (copy)"}
    other = "col" if dom == "row" else "row"
    if kinds[other][2]:
        t_o, b_o, l_o = kinds[other]
        roofline["other_kernel"] = {"kernel": f"{other}_pass_kernel", "achieved": b_o / (t_o / 1e3) / 1e9,
                                    "frac": b_o / (t_o / 1e3) / 1e9 / peak, "us_per_launch": 1e3 * t_o / l_o,
                                    "time_share": t_o / per_pass.sum()}

    # -------- end to end through host buffers
    e2e = None
    if not args.no_e2e:
        host_maps = [torch.from_numpy(m).pin_memory() for m in maps_np]
        host_out = torch.empty((1, n, n), dtype=torch.complex64).pin_memory()
        k_e2e = max(3, args.steps // 2)
        for it in range(1 + k_e2e):
            if it == 1:
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            for hm, dm in zip(host_maps, maps):
                dm.copy_(hm, non_blocking=True)
            plan.execute(field)
            host_out.copy_(field, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k_e2e
        e2e = {"value": HOPS * 1e3 / ms * world, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(m.nbytes for m in maps_np)),
               "d2h_bytes_per_step": int(host_out.numel() * 8), "ms_per_step": ms}

    extras = {}
    if rank == 0 and not args.no_plain:
        extras["plain_gpu"] = plain_gpu(n, maps_np, w, max(3, args.steps // 4), 2, device)
        extras["plain_gpu"]["speedup_of_coro"] = value / world / extras["plain_gpu"]["value"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)

    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
               "config": {"workload": f"relay6_{n}", "n": n, "npix": n // 4, "planes_per_step": HOPS,
                          "batch": 1, "parallelism": f"replicas{world}",
                          "l2": f"inputs larger than L2 ({n * n * 8 / 1e6:.0f} MB field + 2 x {n * n * 4 / 1e6:.0f} MB maps)"},
               "gpu_launches": n_pass * args.steps, "roofline": roofline, "cpu_baseline": cpu,
               "e2e": e2e, "clocks": clk}
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
