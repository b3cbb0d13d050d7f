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
    ap.add_argument("--pass-kernels", default=None, metavar="ROW,COL",
                    help="run the relay on these kernels (coro_fresnel_plan_set_pass_kernel) instead of the "
                         "tuner's pick, e.g. for a profiler capture, where the tuner times serialised launches")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-coronagraph", action="store_true")
    ap.add_argument("--bf16", action="store_true", help="also time the 3xBF16 coronagraph plan")
    ap.add_argument("--psf-lambdas", type=int, default=21, help="wavelengths in the coronagraph batch")
    ap.add_argument("--psf-probes", type=int, default=8, help="DM probe states in the coronagraph batch")
    ap.add_argument("--coronagraph-only", default=None, choices=["tf32", "bf16", "ext"],
                    help="time only the broadband Lyot batch at this precision (for profiler captures)")
    ap.add_argument("--gemm-tile", type=int, default=0,
                    help="with --coronagraph-only: run this GEMM tile width instead of the plan's tuned one")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_throughput(units_per_rank: float, ms: float, world: int, device=None) -> tuple[float, float]:
    """Replicas only: every rank runs its own system on its own GPU, with no exchange on the
    data path. Whole-job throughput = all ranks' units / the slowest rank's time (max over
    ranks; the only collective). Returns (units per second, max ms)."""
    t_max = ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return units_per_rank * world / (t_max / 1e3), t_max


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
    for f in ("fft_engine.cuh", "fft_pair.cuh", "passes.cuh", "passes_launch.cuh", "passes_f32.cu"):
        with open(os.path.join(ROOT, "paper_1806_06467_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str) -> float | None:
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if taken on the
    current pass sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != pass_source_hash():
        return None
    return t.get("kernels", {}).get(kernel, {}).get("dram_bytes_per_launch")


def relay_setup(n: int, seed: int, device):
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    w = inputs.RelayWorkload(n=n, npix=n // 4, seed=seed)
    maps_np = [m.astype(np.float32) for m in w.psd_maps()]
    maps = [torch.from_numpy(m).to(device) for m in maps_np]
    return w, maps_np, maps, relay_elements(w, maps)


def relay_elements(w, maps):
    """The six relay planes, the two PSD surfaces read from the device maps `maps`."""
    from paper_1806_06467_gb300 import coro
    r = w.diam_m / 2
    return [coro.element(coro.EL_APERTURE, plane=0, radius=r, obscuration=w.obscuration,
                         n_spiders=w.n_spiders, spider_width=w.spider_width_frac * w.diam_m),
            coro.element(coro.EL_LENS, plane=1, focal_length=w.lens1_m),
            coro.element(coro.EL_OPD_MAP, plane=2, opd=maps[0]),
            coro.element(coro.EL_LENS, plane=3, focal_length=w.lens2_m),
            coro.element(coro.EL_OPD_MAP, plane=4, opd=maps[1]),
            coro.element(coro.EL_CIRCLE, plane=5, radius=w.field_stop_frac * r)]


# ------------------------------------------------------------------------------ oracle arms
#
# The FP64 oracle (the slow plain program) on the host cores: one core, and every core through a
# spawn-started process pool of independent replicas (one relay, or one PSF, per worker), the
# way the GPU arm's replicas run independent systems. Workers are started with one BLAS thread
# each, so "one core" means one core.

def oracle_relay_runner(n: int, seed: int):
    """One plane of the relay per call on the FP64 oracle: element, then an AS hop; the relay
    restarts from the uniform field every HOPS calls."""
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

    def plane():
        p = state["p"] % HOPS
        if p == 0:
            state["e"] = np.ones((n, n), complex)
        e = state["e"] * element(p)
        state["e"] = propagation.angular_spectrum(e, w.dx, w.wavelength_m, z[p])
        state["p"] += 1

    return plane


def _relay_worker(job):
    """(n, seed, planes_warm, planes_timed or None, budget_s): runs warm-up planes, then timed
    planes (a fixed count, or as many as fit the budget); returns (planes, t_start, t_end)."""
    n, seed, warm, count, budget = job
    plane = oracle_relay_runner(n, seed)
    t_plane = None
    for _ in range(warm):
        t0 = time.time()
        plane()
        t_plane = time.time() - t0
    if count is None:
        count = max(1, int(budget / max(t_plane or budget, 1e-3)))
    t0 = time.time()
    for _ in range(count):
        plane()
    return count, t0, time.time()


def _psf_worker(job):
    """(item index, n_lambda): one PSF of the broadband batch's Lyot system at that wavelength
    on the FP64 oracle (occulter chain and peak); returns (t_start, t_end)."""
    idx, n_lambda = job
    import numpy as np

    from oracle import coronagraph, optics
    from paper_1806_06467_gb300 import inputs
    bw = inputs.BroadbandWorkload(n_lambda=n_lambda)
    lw = bw.lyot
    lam = bw.wavelengths()[idx % n_lambda]
    rr = bw.lambda_c_m / lam
    m_occ = int(bw.occulter_sizes()[idx % n_lambda])
    opd = optics.zernike_opd(lw.n, 1.0 / lw.npix, 0.5, lw.zernike(), lw.zernike_first)
    pupil = coronagraph.pupil_field(lw.n, lw.npix, lam, opd)
    p = coronagraph.LyotParams(n=lw.n, npix=lw.npix, m_occ=m_occ, du_occ=lw.du_occ * rr,
                               spot_radius=lw.spot_radius_lamd * rr, lyot_frac=lw.lyot_frac, m_det=lw.m_det,
                               du_det=lw.du_det * rr)
    t0 = time.time()
    coronagraph.lyot_psf(pupil, p, lw.dh_inner * rr, lw.dh_outer * rr)
    return t0, time.time()


def _oracle_pool(workers: int):
    """Spawn-started pool whose workers run numpy with one BLAS thread."""
    import multiprocessing as mp
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in keep:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(workers)
    finally:
        for v, old in keep.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def run_reference(args):
    """The reference arm of this tier: the FP64 oracle on every host core, one relay replica per
    core, each step the full five-plane relay at args.n (the GPU arm's step), warm-up steps as
    asked while they fit the time budget, timed steps bounded so the run ends within a few
    minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    try:
        # calibration: one plane per worker (also their first-touch warm-up)
        cal = pool.map(_relay_worker, [(args.n, c, 0, 1, 0.0) for c in range(cores)])
        t_plane = max(t1 - t0 for _, t0, t1 in cal)
        t_step = HOPS * t_plane
        budget = 150.0
        warm = max(0, min(args.warmup, int(0.4 * budget / t_step)))
        steps = max(1, min(args.steps, int(0.6 * budget / t_step)))
        res = pool.map(_relay_worker, [(args.n, c, HOPS * warm, HOPS * steps, 0.0) for c in range(cores)])
    finally:
        pool.close()
        pool.join()
    planes = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    value = planes / wall
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": steps, "warmup": warm, "ms_per_step": 1e3 * wall / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"relay6_{args.n}", "n": args.n, "npix": args.n // 4, "planes_per_step": HOPS,
                      "batch": 1, "parallelism": f"replicas{cores} (host cores)",
                      "note": "FP64 numpy oracle (textbook radix-2 FFT), one relay replica per host core"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{steps} five-plane relay steps at {args.n}^2 on each of {cores} cores "
                                      f"after {warm} warm-up steps"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(n: int, n_lambda: int = 21) -> dict:
    """Bounded samples of the oracle on the host: relay planes on one core and on every core,
    Lyot PSFs of the broadband batch on one core and on every core."""
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    try:
        one = pool.apply(_relay_worker, ((n, 0, 0, 2, 0.0),))
        allc = pool.map(_relay_worker, [(n, c, 0, 1, 0.0) for c in range(cores)])
        psf1 = pool.apply(_psf_worker, ((n_lambda // 2, n_lambda),))
        psfs = pool.map(_psf_worker, [(i, n_lambda) for i in range(cores)])
    finally:
        pool.close()
        pool.join()
    value = one[0] / (one[2] - one[1])
    all_value = sum(r[0] for r in allc) / (max(r[2] for r in allc) - min(r[1] for r in allc))
    psf_one = 1.0 / (psf1[1] - psf1[0])
    psf_all = cores / (max(t1 for _, t1 in psfs) - min(t0 for t0, _ in psfs))
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{one[0]} planes (element + angular-spectrum hop, textbook radix-2 FFT) of the {n}^2 relay, "
                      "FP64 numpy, one core",
            "all_cores": {"value": all_value, "unit": UNIT, "cores": cores,
                          "sample": f"one plane on each of {cores} cores (independent relays, spawn pool)"},
            "psf": {"value": psf_one, "unit": "PSFs/s", "cores": 1,
                    "sample": "one Lyot PSF of the broadband batch (1024^2 pupil, occulter, Babinet, Lyot stop, "
                              "512^2 detector, peak), FP64 oracle, one BLAS thread"},
            "psf_all_cores": {"value": psf_all, "unit": "PSFs/s", "cores": cores,
                              "sample": f"one PSF per core at {cores} wavelengths of the batch"}}


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


# ------------------------------------------------------------------------------ coronagraph PSFs

_TF32_PEAK = None


def tensor_peak(kind: str, device=None) -> tuple[float, str]:
    """Dense tensor peak (TFLOP/s) for a kernel timed in a short region: BF16 is the driver's
    measured burst cuBLAS figure (MEASURED_PEAKS.json bf16_tflops); TF32 is measured here, once
    per run, as the best of ten 8192^3 FP32 matmuls with TF32 tensor cores allowed (cuBLAS),
    timed with CUDA events."""
    global _TF32_PEAK
    if kind == "tf32":
        if _TF32_PEAK is None:
            import torch
            old = torch.backends.cuda.matmul.allow_tf32
            torch.backends.cuda.matmul.allow_tf32 = True
            a = torch.randn((8192, 8192), device=device)
            b = torch.randn((8192, 8192), device=device)
            c = a @ b
            best = float("inf")
            for _ in range(10):
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record()
                c = a @ b
                t1.record()
                torch.cuda.synchronize()
                best = min(best, t0.elapsed_time(t1))
            torch.backends.cuda.matmul.allow_tf32 = old
            del a, b, c
            _TF32_PEAK = 2 * 8192 ** 3 / (best / 1e3) / 1e12
        return _TF32_PEAK, "measured in this run: cuBLAS TF32 8192^3 matmul, best of 10 (burst)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16_tflops (MEASURED_PEAKS.json, burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback bf16 burst"


def broadband_pupils(ctx, device, n_lambda: int = 21, n_probe: int = 8):
    """168 pupil fields (21 wavelengths x 8 DM sinc probes): clear aperture, Zernike 4-21 at 5 nm
    RMS and the probe's DM surface (Gaussian influence, FWHM 1 pitch), built by the library."""
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    bw = inputs.BroadbandWorkload(n_lambda=n_lambda, n_probe=n_probe)
    lw = bw.lyot
    lams = bw.wavelengths()
    lam_b = np.repeat(lams, bw.n_probe)
    B, n, npix = len(lam_b), lw.n, lw.npix
    dx = lw.diam_m / npix
    field = torch.empty((B, n, n), dtype=torch.complex64, device=device)
    coro.wavefront_init(ctx, field, 1.0)
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_APERTURE, radius=lw.diam_m / 2))
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_ZERNIKE, radius=lw.diam_m / 2, coeffs=lw.zernike(),
                                                           j_first=lw.zernike_first))
    heights = torch.from_numpy(np.tile(bw.probes(), (len(lams), 1, 1)).astype(np.float32)).to(device)
    pitch = lw.diam_m / bw.n_act
    opd = coro.dm_opd(ctx, heights, pitch, pitch, n, dx, 2.0)
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_OPD_MAP, opd=opd, flags=coro.ELF_MAP_BATCHED))
    torch.cuda.synchronize()
    del opd
    r = bw.lambda_c_m / lam_b
    items = [dict(m_occ=int(m), du_occ=lw.du_occ * rr, spot_radius=lw.spot_radius_lamd * rr, du_det=lw.du_det * rr,
                  dh_in=lw.dh_inner * rr, dh_out=lw.dh_outer * rr)
             for m, rr in zip(np.repeat(bw.occulter_sizes(), bw.n_probe), r)]
    return field, items, lw


PRECISION_NAMES = {1: "3xTF32", 2: "3xBF16", 4: "EXT (4 exact BF16 slices, two-float accumulation)"}
SAMPLED = (0, 0.5, 1.0)        # items compared for accuracy: first, middle, last


def sampled_items(batch: int) -> list:
    return sorted({min(batch - 1, int(f * batch)) for f in SAMPLED})


def darkhole_masks(items, md: int, device):
    """Boolean dark-hole masks [md][md] of the given items: dh_in <= |(i', j')| du_det <= dh_out."""
    import torch
    k = torch.arange(md, device=device, dtype=torch.float64) - md // 2
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    return [(k2 * it["du_det"] ** 2 >= it["dh_in"] ** 2) & (k2 * it["du_det"] ** 2 <= it["dh_out"] ** 2) for it in items]


def max_darkhole_error(inten, ref, items, md: int, device) -> float:
    """max |I - I_ref| over the dark holes of the sampled items (both normalised by their own peaks)."""
    idx = sampled_items(len(items))
    masks = darkhole_masks([items[b] for b in idx], md, device)
    return max(float((inten[b].double() - ref[b].double()).abs()[m].max()) for b, m in zip(idx, masks))


def coronagraph_bench(ctx, device, steps: int, warmup: int, precision: int, n_lambda: int = 21,
                      n_probe: int = 8, pupils=None, keep_output: bool = False, gemm_tile: int = 0) -> dict:
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro
    if pupils is None:
        pupils = broadband_pupils(ctx, device, n_lambda, n_probe)
    pupils, items, lw = pupils
    B, n, md = len(items), lw.n, lw.m_det
    plan = coro.LyotPlan(ctx, n=n, npix=lw.npix, lyot_frac=lw.lyot_frac, m_det=md, items=items, precision=precision)
    if gemm_tile:
        plan.set_gemm_tile(gemm_tile)
    peak = plan.peak(pupils)                          # normalisation, computed once
    psf = torch.empty((B, md, md), dtype=torch.float32, device=device)   # the PSFs, written every step
    stream = torch.cuda.current_stream(device)
    for _ in range(warmup):
        plan.execute(pupils, peak=peak, intensity=psf, want_dh=False)
    torch.cuda.synchronize()
    # the timed steps run as one CUDA graph (captured first, untimed); the per-stage times
    # (split, G1, G2, G3, G4 Babinet, detector G5 + G6) come from a second replay of the same
    # steps with event nodes inside the graph
    plan.use_graph(True)
    plan.execute_n(pupils, steps, peak=peak, intensity=psf)
    torch.cuda.synchronize()
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ga.record(stream)
    plan.execute_n(pupils, steps, peak=peak, intensity=psf)
    gb.record(stream)
    torch.cuda.synchronize()
    total_ms = ga.elapsed_time(gb)
    plan.set_timing(steps)
    plan.execute_n(pupils, steps, peak=peak, intensity=psf)
    torch.cuda.synchronize()
    plan.execute_n(pupils, steps, peak=peak, intensity=psf)
    per = plan.unit_times(steps)                      # [steps][6]
    plan.set_timing(0)
    plan.use_graph(False)
    # dense complex MACs of the six GEMMs; the plan's own counts weigh them by the products its
    # precision issues (3 split terms: 24 flops per complex MAC, EXT: 10 slice products, 80 flops)
    cmac = 0.0
    for it in items:
        mo = it["m_occ"]
        cmac += n * mo * n + mo * mo * n + mo * n * mo + n * n * mo + n * md * n + md * md * n
    per_cmac = 80.0 if precision == coro.MFT_EXT else 24.0
    # what the support-aware plan computes: only K ranges / tiles inside the spot and stop
    useful_flops, issued_flops = plan.flops()
    gemm_ms = float(per[:, 1:].sum())                 # stages 1-5 are tensor-core GEMM launches
    achieved = useful_flops * steps / (gemm_ms / 1e3) / 1e12
    pk, src = tensor_peak("tf32" if precision == coro.MFT_3XTF32 else "bf16", device)
    kernel = "tcx_cgemm_kernel" if precision == coro.MFT_EXT else "tc_cgemm_kernel"
    out = {"value": B * steps / (total_ms / 1e3), "unit": "PSFs/s", "batch": B,
           "precision": PRECISION_NAMES[precision],
           "workload": "broadband_lyot: 21 wavelengths (500-600 nm) x 8 DM sinc probes, 1024^2 pupil, "
                       "occulter 235-282 px at 0.05 lc/l lambda/D, detector 512^2",
           "ms_per_step": total_ms / steps, "gpu_launches_per_step": 8, "graph_replays": 1,
           "gemm_tile": list(plan.gemm_tile()),
           "roofline": {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": pk,
                        "unit": "TFLOP/s", "frac": achieved / pk, "traffic": None,
                        "flops_per_step": useful_flops, "time_share": gemm_ms / float(per.sum()),
                        "issued_flops_per_step": issued_flops, "issued_frac": issued_flops * steps / (gemm_ms / 1e3) / 1e12 / pk,
                        "dense_flops_per_step": per_cmac * cmac, "peak_source": src},
           "stage_ms": [round(float(x), 4) for x in per.mean(axis=0)]}
    plan.close()
    if keep_output:
        out["_psf"] = psf
    return out


def coronagraph_plain(device, steps: int, pupils) -> dict:
    """Plain per-wavelength FP32 GPU form of the same broadband batch: torch.matmul (cuBLAS
    cgemm, complex64) MFT chain per wavelength over its probe pupils, bases precomputed in FP64
    and rounded to complex64, no fusion, no graph; normalised by the peak of its own
    no-occulter chain. Returns the throughput and the PSFs (for the accuracy comparison)."""
    import math

    import torch
    field, items, lw = pupils
    B, n, md, npix = len(items), lw.n, lw.m_det, float(lw.npix)
    x = (torch.arange(n, device=device, dtype=torch.float64) - n // 2) / npix
    k = torch.arange(n, device=device, dtype=torch.float64) - n // 2
    lyot = ((k[None, :] ** 2 + k[:, None] ** 2) / npix ** 2 <= (0.5 * lw.lyot_frac) ** 2).to(torch.complex64)

    def basis(m, du, sign):
        u = (torch.arange(m, device=device, dtype=torch.float64) - m // 2) * du
        return torch.polar(torch.ones(m, n, device=device, dtype=torch.float64),
                           sign * 2 * math.pi * torch.outer(u, x)).to(torch.complex64)

    groups = {}                                       # one group per wavelength: consecutive items
    for b, it in enumerate(items):
        key = (it["m_occ"], it["du_occ"], it["du_det"], it["spot_radius"])
        groups.setdefault(key, []).append(b)
    chains = []
    for (mo, du_occ, du_det, spot_r), idx in groups.items():
        ko = torch.arange(mo, device=device, dtype=torch.float64) - mo // 2
        spot = ((ko[None, :] ** 2 + ko[:, None] ** 2) * du_occ ** 2 <= spot_r ** 2).to(torch.complex64)
        a = basis(mo, du_occ, -1)
        chains.append((idx[0], idx[-1] + 1, a, a.conj().T.contiguous(), basis(md, du_det, -1), spot,
                       du_occ / npix, du_det / npix))
    inten = torch.empty((B, md, md), dtype=torch.float32, device=device)
    peak = torch.empty((B,), dtype=torch.float32, device=device)
    for b0, b1, a, bt, ad, spot, s_occ, s_det in chains:   # normalisation, once
        det = s_det * (ad @ (field[b0:b1] * lyot) @ ad.T)
        peak[b0:b1] = (det.real ** 2 + det.imag ** 2).amax(dim=(1, 2))

    def step():
        for b0, b1, a, bt, ad, spot, s_occ, s_det in chains:
            e = field[b0:b1]
            eb = s_occ * (a @ e @ a.T)
            ec = (e - s_occ * (bt @ (spot * eb) @ bt.T)) * lyot
            det = s_det * (ad @ ec @ ad.T)
            inten[b0:b1] = (det.real ** 2 + det.imag ** 2) / peak[b0:b1, None, None]

    step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    return {"value": B * 1e3 / ms, "unit": "PSFs/s", "ms_per_step": ms,
            "form": "per-wavelength torch.matmul complex64 (cuBLAS FP32) MFT chain, probes batched, own peak",
            "_psf": inten}


def spc_system_bench(ctx, device, steps: int, npix: int = 1024) -> dict:
    """The nine-plane system of App. B's shape (telescope, 20 mm relay, shaped pupil, bow-tie
    mask, three foci) at N = 4 npix, one wavelength, through the pilot-beam plan: K systems
    replayed as one CUDA graph. The paper times this system in FP64 on CPUs and a K80."""
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    w = inputs.SpcWorkload(npix=npix)
    n, lam = w.n, w.wavelength_m
    maps = {"zero": torch.zeros((1, n, n), device=device), "shaped_pupil": torch.zeros((1, n, n), device=device),
            "fpm": torch.zeros((1, n, n), device=device)}
    els = []
    for p, plane in enumerate(w.layout()):
        for el in plane:
            if el[0] == "aperture":
                els.append(coro.element(coro.EL_APERTURE, plane=p, radius=w.d_prim_m / 2, obscuration=w.obscuration,
                                        n_spiders=w.n_spiders, spider_width=w.spider_width_frac * w.d_prim_m))
            elif el[0] == "lens":
                els.append(coro.element(coro.EL_LENS, plane=p, focal_length=el[1]))
            else:
                els.append(coro.element(coro.EL_OPD_MAP, plane=p, opd=maps["zero"], amplitude=maps[el[0]],
                                        flags=coro.ELF_MAP_BATCHED))
    plan = coro.FresnelSystem(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=lam, beam_radius=w.d_prim_m / 2,
                              distances=w.distances(), elements=els, init_uniform=True)
    maps["shaped_pupil"][0] = torch.from_numpy(w.shaped_pupil(n, plan.plane_pitch(4)[0])).to(device)
    maps["fpm"][0] = torch.from_numpy(w.bowtie(n, plan.plane_pitch(6)[0], lam)).to(device)
    _, legs = plan.info()
    field = torch.empty((1, n, n), dtype=torch.complex64, device=device)
    stream = torch.cuda.current_stream(device)
    plan.use_graph(True)
    plan.execute_n(field, steps)                      # capture
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.execute_n(field, steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out = {"value": 1e3 / ms, "unit": "systems/s", "ms_per_system": ms, "n": n, "npix": npix,
           "planes": len(w.layout()), "direct_legs": legs, "passes_per_system": plan.launch_count,
           "workload": "App.-B-shaped 9-plane shaped-pupil coronagraph system (2.37 m f/7.8 telescope, 20 mm "
                       "relay, f/20 optics, shaped pupil + bow-tie stand-in masks), complex64, pilot-beam hops",
           "paper_context_s": {"numpy_fp64_8core_sandy_bridge_N4096": 90.16, "k80_fp64_about": "5x faster than numpy"}}
    plan.close()
    return out


def wfc_bench(ctx, device, steps: int) -> dict:
    """Differentiable wavefront control at full size: loss and dL/dh for 2 x 48 x 48 DM heights,
    Fresnel 4096^2 between the DMs, Lyot chain at 11 wavelengths (3xTF32); one step is one
    forward + adjoint evaluation (each returns its loss to the host)."""
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs, wfc
    w = inputs.WfcWorkload()
    lw = w.lyot
    lams = list(w.wavelengths())
    plan = wfc.WfcPlan(ctx, wavelengths=lams, n_fresnel=w.n_fresnel, diam_m=w.diam_m, npix=lw.npix, z_m=w.z_m,
                       n_act=w.n_act, pitch_m=w.pitch_m, fwhm_m=w.pitch_m, lyot_frac=lw.lyot_frac, m_det=lw.m_det,
                       items=[w.item(l) for l in lams], precision=coro.MFT_3XTF32)
    plan.peak()
    h = torch.from_numpy(w.heights().astype(np.float32)).to(device)
    stream = torch.cuda.current_stream(device)
    for _ in range(2):
        plan.evaluate(h)
    torch.cuda.synchronize()

    def timed(want_grad):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            plan.evaluate(h, want_grad=want_grad)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    ms = timed(True)
    ms_fwd = timed(False)
    plan.close()
    return {"value": 1e3 / ms, "unit": "gradients/s", "ms_per_gradient": ms, "ms_forward_only": ms_fwd,
            "wavelengths": len(lams), "n_fresnel": w.n_fresnel,
            "workload": "two 48x48 DMs (+-5 nm) 0.3 m apart on a 4096^2 Fresnel grid, Lyot chain at 11 "
                        "wavelengths 525-575 nm (3xTF32); loss + dL/dh per step"}


def relay_mixed_bench(ctx, device, steps: int, n: int = 2800, npix: int = 700) -> dict:
    """The six-plane relay at a line length that is not a power of two (Sec. 3.1 times
    N = 2800 against the powers of two): mixed-radix passes, K relays replayed as one graph."""
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    w = inputs.RelayWorkload(n=n, npix=npix, seed=0)
    maps = [torch.from_numpy(m.astype(np.float32)).to(device) for m in w.psd_maps()]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=relay_elements(w, maps), init_uniform=True)
    field = torch.empty((1, n, n), dtype=torch.complex64, device=device)
    stream = torch.cuda.current_stream(device)
    plan.use_graph(True)
    plan.execute_n(field, steps)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plan.execute_n(field, steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    kernels = sorted({plan.pass_kernel(i) for i in range(plan.launch_count)})
    plan.close()
    return {"value": HOPS * 1e3 / ms, "unit": "planes/s", "ms_per_relay": ms, "n": n, "kernels": kernels,
            "workload": f"six-plane relay (5 hops) at N = {n} (npix {npix}), complex64, mixed-radix passes"}


def coronagraph_fp64(ctx, device, steps: int = 3) -> dict:
    """One PSF of the Lyot system through the FP64 calls on complex128 fields (MFT, spot,
    inverse MFT, Babinet axpy, Lyot stop, MFT to the detector): the path that meets the 1e-11
    dark-hole bar, timed for comparison with the split-precision plan."""
    import numpy as np
    import torch

    from paper_1806_06467_gb300 import coro, inputs
    w = inputs.LyotWorkload()
    npix = float(w.npix)
    e_a = torch.ones((1, w.n, w.n), dtype=torch.complex128, device=device)
    coro.apply_element(ctx, e_a, 1.0 / npix, w.wavelength_m, coro.element(coro.EL_APERTURE, radius=0.5))
    coro.apply_element(ctx, e_a, 1.0 / npix, w.wavelength_m,
                       coro.element(coro.EL_ZERNIKE, radius=0.5, coeffs=w.zernike(), j_first=w.zernike_first))
    spot = coro.element(coro.EL_CIRCLE, radius=w.spot_radius_lamd)
    stop = coro.element(coro.EL_CIRCLE, radius=0.5 * w.lyot_frac)

    def psf():
        e_b = coro.propagate_mft(ctx, e_a, npix, -1, w.m_occ, [w.du_occ])
        coro.apply_element(ctx, e_b, w.du_occ, w.wavelength_m, spot)
        e_s = coro.propagate_mft(ctx, e_b, npix, +1, w.n, [w.du_occ])
        coro.wavefront_axpy(ctx, -1.0, e_a, e_s)          # IMFT(spot . E_B) - E_A = -E_C (E_A kept)
        coro.apply_element(ctx, e_s, 1.0 / npix, w.wavelength_m, stop)
        return coro.propagate_mft(ctx, e_s, npix, -1, w.m_det, [w.du_det])   # -E_det: same PSF

    psf()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        psf()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # complex multiply-adds of the three MFTs (two GEMMs each), 8 real flops apiece
    n, mo, md = w.n, w.m_occ, w.m_det
    cmac = (mo * n * n + mo * mo * n) * 2 + md * n * n + md * md * n
    achieved = 8.0 * cmac / (ms * 1e-3) / 1e12
    fp64_peak = 1.25
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "flops_per_psf": 8.0 * cmac, "kernel": "zgemm_simt_kernel (split K)",
            "peak_source": "nominal GB300 FP64 rate (an FP64 FMA probe measured 1.19 TFLOP/s)"}
    return {"value": 1e3 / ms, "unit": "PSFs/s", "ms_per_psf": ms, "precision": "FP64 (complex128)", "roofline": roof,
            "workload": "Lyot system of the broadband batch at its centre wavelength, one PSF per call sequence"}


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
    if args.coronagraph_only:
        prec = {"tf32": coro.MFT_3XTF32, "bf16": coro.MFT_3XBF16, "ext": coro.MFT_EXT}[args.coronagraph_only]
        line = coronagraph_bench(ctx, device, args.steps, args.warmup, prec, args.psf_lambdas, args.psf_probes,
                                 gemm_tile=args.gemm_tile)
        line.update({"metric": METRIC, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                     "config": {"workload": f"broadband_lyot {args.psf_lambdas} x {args.psf_probes}"}})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    n = args.n
    w, maps_np, maps, els = relay_setup(n, seed=rank, device=device)
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=els, init_uniform=True)
    if args.pass_kernels:
        rv, cl = (int(v) for v in args.pass_kernels.split(","))
        plan.set_pass_kernel(rv, cl)
    n_pass = plan.launch_count
    info = [plan.pass_info(i) for i in range(n_pass)]
    flops = [plan.pass_flops(i) for i in range(n_pass)]
    kernels = [plan.pass_kernel(i) for i in range(n_pass)]
    field = torch.empty((1, n, n), dtype=torch.complex64, device=device)

    for _ in range(args.warmup):
        plan.execute(field)
    torch.cuda.synchronize()
    # the timed steps run as one CUDA graph, captured here, outside the timed region
    plan.use_graph(True)
    plan.execute_n(field, args.steps)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    # -------- timed region: K steps (one graph replay), bracketed by events on the plan's stream
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    plan.execute_n(field, args.steps)
    t1.record(stream)
    torch.cuda.synchronize()
    # -------- the same K steps again with the library's per-pass events recorded inside the
    # graph (event nodes add a few microseconds per pass, so they stay out of the value)
    plan.set_timing(args.steps)
    plan.execute_n(field, args.steps)                  # capture with event nodes
    torch.cuda.synchronize()
    plan.execute_n(field, args.steps)
    per_pass = plan.unit_times(args.steps)             # [K][passes]
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    value, t_max = replica_throughput(HOPS * args.steps, total_ms, world, device)

    # -------- roofline of the dominant pass kind
    kinds = {"row": [0.0, 0.0, 0, set(), 0.0], "col": [0.0, 0.0, 0, set(), 0.0]}
    for i, (is_row, nbytes) in enumerate(info):
        kk = "row" if is_row else "col"
        kinds[kk][0] += per_pass[:, i].sum()
        kinds[kk][1] += nbytes * args.steps
        kinds[kk][2] += args.steps
        kinds[kk][3].add(kernels[i])
        kinds[kk][4] += flops[i] * args.steps
    # the passes' FP32 arithmetic against the CUDA-core peak: SMs x 128 FP32 lanes x 2 flops
    # (one FMA) x the maximum SM clock
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    alu_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12

    def alu(kind):
        t_k, f_k = kinds[kind][0], kinds[kind][4]
        return {"achieved": f_k / (t_k / 1e3) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": f_k / (t_k / 1e3) / 1e12 / alu_peak, "flops_per_launch": f_k / kinds[kind][2],
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {sm_max:.0f} MHz (derived)",
                "flops": "5 N log2 N per line transform, 1 or 2 transforms per pass; elements not counted"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    t_dom, b_dom, l_dom, k_dom = kinds[dom][:4]
    k_name = ", ".join(sorted(k_dom))
    peak, peak_src = measured_peaks()
    achieved = b_dom / (t_dom / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(k_name) if len(k_dom) == 1 else None, "kernel": k_name,
                "bytes_per_launch": b_dom / l_dom, "us_per_launch": 1e3 * t_dom / l_dom,
                "time_share": t_dom / per_pass.sum(), "peak_source": f"{peak_src} hbm_gbs (copy)",
                "timing": "library CUDA events around each pass, inside a second graph replay of the K steps",
                "alu": alu(dom)}
    other = "col" if dom == "row" else "row"
    if kinds[other][2]:
        t_o, b_o, l_o, k_o = kinds[other][:4]
        roofline["other_kernel"] = {"kernel": ", ".join(sorted(k_o)), "achieved": b_o / (t_o / 1e3) / 1e9,
                                    "traffic": recorded_traffic(next(iter(k_o))) if len(k_o) == 1 else None,
                                    "frac": b_o / (t_o / 1e3) / 1e9 / peak, "us_per_launch": 1e3 * t_o / l_o,
                                    "time_share": t_o / per_pass.sum(), "alu": alu(other)}

    passes = [{"kernel": kernels[i], "us": round(1e3 * float(np.median(per_pass[:, i])), 2),
               "bytes": info[i][1]} for i in range(n_pass)]
    # per-step spread from the event-instrumented replay (sum of the step's pass times; the
    # value above is the uninstrumented replay)
    per_step = per_pass.sum(axis=1)
    step_stats = {"median_ms": float(np.median(per_step)), "mean_ms": float(per_step.mean()),
                  "std_ms": float(per_step.std(ddof=1)) if len(per_step) > 1 else 0.0,
                  "steps": int(len(per_step)), "source": "per-pass library events, second replay"}

    plan.set_timing(0)
    plan.use_graph(False)

    # -------- end to end through host buffers: every step copies its two surface maps in from
    # pinned host memory and its output field out, all inside the timed region. Two plan slots
    # (each with its own device maps and field) let step k's copies overlap steps k-1 / k+1's
    # propagation: H2D and D2H on their own streams, ordered with events.
    e2e = None
    if not args.no_e2e:
        k_e2e = max(4, args.steps)
        slots = []
        for sidx in range(2):
            dmaps = maps if sidx == 0 else [torch.empty_like(m) for m in maps]
            fld = field if sidx == 0 else torch.empty_like(field)
            pl = plan if sidx == 0 else coro.FresnelPlan(
                ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m, distances=list(w.distances()),
                elements=relay_elements(w, dmaps), init_uniform=True)
            if sidx:
                pl.copy_tuning(plan)                       # both slots run the same kernels
            pl.use_graph(True)
            slots.append({"maps": dmaps, "field": fld, "plan": pl,
                          "host_maps": [torch.from_numpy(m).pin_memory() for m in maps_np],
                          "host_out": torch.empty((1, n, n), dtype=torch.complex64).pin_memory(),
                          "h2d": torch.cuda.Event(), "done": torch.cuda.Event(), "d2h": torch.cuda.Event()})
        h2d_s, d2h_s = torch.cuda.Stream(device), torch.cuda.Stream(device)

        def e2e_step(sl):
            with torch.cuda.stream(h2d_s):
                h2d_s.wait_event(sl["done"])              # the slot's previous propagation has read its maps
                for hm, dm in zip(sl["host_maps"], sl["maps"]):
                    dm.copy_(hm, non_blocking=True)
                sl["h2d"].record(h2d_s)
            stream.wait_event(sl["h2d"])
            stream.wait_event(sl["d2h"])                  # the slot's previous field has been copied out
            sl["plan"].execute(sl["field"])
            sl["done"].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(sl["done"])
                sl["host_out"].copy_(sl["field"], non_blocking=True)
                sl["d2h"].record(d2h_s)

        for sl in slots:                                   # warm-up: captures both slots' graphs
            e2e_step(sl)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(h2d_s)
        stream.wait_event(a)
        d2h_s.wait_event(a)
        for k in range(k_e2e):
            e2e_step(slots[k % 2])
        b.record(d2h_s)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k_e2e
        e2e = {"value": HOPS * 1e3 / ms * world, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(m.nbytes for m in maps_np)),
               "d2h_bytes_per_step": int(field.numel() * 8), "ms_per_step": ms, "steps": k_e2e,
               "form": "plan.execute per step, pinned host maps in and field out on two copy streams, "
                       "two plan slots so copies overlap propagation"}
        slots[1]["plan"].close()
        plan.use_graph(False)

    extras = {}
    if not args.no_coronagraph:
        k_psf = max(3, args.steps // 2)
        pupils = broadband_pupils(ctx, device, args.psf_lambdas, args.psf_probes)
        items, md = pupils[1], pupils[2].m_det
        extras["coronagraph"] = coronagraph_bench(ctx, device, k_psf, max(1, min(3, args.warmup)), coro.MFT_3XTF32,
                                                  pupils=pupils, keep_output=True)
        extras["coronagraph"]["value"] *= world
        extras["coronagraph_ext"] = coronagraph_bench(ctx, device, k_psf, 1, coro.MFT_EXT, pupils=pupils,
                                                      keep_output=True)
        extras["coronagraph_ext"]["value"] *= world
        if args.bf16:
            extras["coronagraph_3xbf16"] = coronagraph_bench(ctx, device, k_psf, 1, coro.MFT_3XBF16, pupils=pupils)
        # accuracy at equal inputs: every form's dark-hole intensities on the sampled items against
        # the extended-precision plan's (which the GPU tests hold within 1e-11 of the FP64 oracle)
        ref = extras["coronagraph_ext"].pop("_psf")
        psf_tf32 = extras["coronagraph"].pop("_psf")
        extras["coronagraph"]["darkhole_max_abs_err_vs_ext"] = max_darkhole_error(psf_tf32, ref, items, md, device)
        del psf_tf32
        if rank == 0 and not args.no_plain:
            plain = coronagraph_plain(device, max(2, k_psf // 3), pupils)
            plain["darkhole_max_abs_err_vs_ext"] = max_darkhole_error(plain.pop("_psf"), ref, items, md, device)
            plain["speedup_of_3xtf32"] = extras["coronagraph"]["value"] / world / plain["value"]
            plain["speedup_of_ext"] = extras["coronagraph_ext"]["value"] / world / plain["value"]
            plain["accuracy_note"] = ("max |dI| over the dark holes of items " + str(sampled_items(len(items))) +
                                      ", each form normalised by its own peak, against the EXT plan")
            extras["coronagraph"]["plain_gpu"] = plain
        del ref, pupils
        torch.cuda.empty_cache()
    if not args.no_coronagraph:
        extras["spc_system"] = spc_system_bench(ctx, device, max(3, args.steps // 2))
        extras["wfc_gradient"] = wfc_bench(ctx, device, max(3, args.steps // 4))
        extras["relay_mixed_radix"] = relay_mixed_bench(ctx, device, max(3, args.steps // 2))
        # App. B's pupil (npix 1025) padded 4x: N = 4100 = 4 x 5^2 x 41, a radix-41 stage
        extras["relay_mixed_radix_4100"] = relay_mixed_bench(ctx, device, 3, n=4100, npix=1025)
        extras["coronagraph_fp64"] = coronagraph_fp64(ctx, device)
    if rank == 0 and not args.no_plain:
        extras["plain_gpu"] = plain_gpu(n, maps_np, w, max(3, args.steps // 4), 2, device)
        extras["plain_gpu"]["speedup_of_coro"] = value / world / extras["plain_gpu"]["value"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, args.psf_lambdas)

    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
               "config": {"workload": f"relay6_{n}", "n": n, "npix": n // 4, "planes_per_step": HOPS,
                          "batch": 1, "parallelism": f"replicas{world}",
                          "l2": f"inputs larger than L2 ({n * n * 8 / 1e6:.0f} MB field + 2 x {n * n * 4 / 1e6:.0f} MB maps)"},
               "gpu_launches": n_pass * args.steps, "graph_replays": 1, "roofline": roofline, "passes": passes,
               "step_stats": step_stats,
               "cpu_baseline": cpu,
               "e2e": e2e, "clocks": clk}
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
