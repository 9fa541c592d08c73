"""Benchmark: forward + backward propagations per second on the polarised 4f workload.

Workload (one step): 16 objects x 3 field components (Ex, Ey, Ez) x 8 wavelengths in
450-700 nm = 384 fields of 1024 x 1024, spacing 5 um, 2x zero padding (2048^2 FFTs),
angular-spectrum method; a 4f system with two thin lenses (f = 0.2 m) and a circular
pupil (R = 1 mm) carrying a trainable phase; detector intensity summed over each
object's components and wavelengths; MSE loss against seeded targets; gradient with
respect to the pupil phase. Per field: 4 forward and 2 backward propagations. The
metric counts fwd+bwd propagation pairs: (forward + backward propagations) / 2 per
second, whole job over all ranks (weak scaling, one replica of the workload per GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "fwd+bwd propagations/s at 1024² c64, % of HBM roofline, rel-L2 vs FP64"
UNIT = "fwd+bwd propagations/s"
FALLBACK_HBM = 6800.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM}, "fallback"


# The sources the passes of the 1024-point plan are compiled from (their unit and every header it
# includes): a change anywhere else in the library leaves the profiled kernels as they were.
KERNEL_SOURCES = ("top_unit_m1024.cu", "top_unit.cuh", "top_dispatch.h", "top_czt.cuh", "top_passes.cuh",
                  "top_pair_rows.cuh", "top_engine.cuh", "top_internal.h", "top_launch.h", "../../include/top.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2411_18591_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kind: str):
    """DRAM bytes per field of a kernel from the committed ncu summary, if it matches the current sources."""
    path = os.path.join(ROOT, "profiles", f"{kind}_summary.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_field:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def bus_id_of(dev_index: int):
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle sample

def oracle_sample_step(obj_field, lam, fourf_cfg, phase, target):
    """The oracle (FP64, host) on one field of the workload: 4 forward + 2 backward propagations.
    Returns (seconds, loss, pupil-phase gradient)."""
    import oracle as O
    c = fourf_cfg
    t0 = time.perf_counter()
    loss, g_phi, _ = O.fourf_loss_and_grad(obj_field[None], [lam], c["d"], c["f"], c["lens_radius"],
                                           c["pupil_radius"], phase, 1, target[None], c["pad"])
    return time.perf_counter() - t0, loss, g_phi


def _oracle_field(i: int):
    """The oracle's 4f step on field i of the workload's sample (object i, Ex, 450 nm); returns
    (seconds, loss, pupil-phase gradient). Runs in a worker process."""
    c = S.CFG4
    obj = S.cfg4_objects(1, 1, c["n"], first=i)[0, 0].astype(np.complex128)
    phase = S.cfg4_pupil_phase(c["n"])
    target = S.cfg4_target(1, c["n"], first=i)[0]
    lam = float(S.cfg4_wavelengths(c["wavelengths"])[0])
    cfg = dict(d=c["d"], f=c["f"], lens_radius=c["lens_radius"], pupil_radius=c["pupil_radius"], pad=c["pad"])
    return oracle_sample_step(obj, lam, cfg, phase, target)


def cpu_baseline(steps: int, warmup: int, budget_s: float = 25.0, want_sample: bool = False):
    """The oracle timed on the host cores: one worker process per core (spawned, so no GPU state is
    inherited), each running the full 4f chain of one field of the workload; rounds of one field a
    worker until the budget is spent. With want_sample, also returns the first field's inputs and
    the oracle's results on it (the 4f loss and pupil-phase gradient, and one AS propagation and
    its adjoint of the object field), for the parity of the GPU line."""
    import multiprocessing as mp
    n = S.CFG4["n"]
    c = S.CFG4
    workers = max(1, min(16, os.cpu_count() or 1))
    rounds, fields, t_total = 0, 0, 0.0
    loss = g_phi = None
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        t_start = time.perf_counter()
        while True:
            t0 = time.perf_counter()
            res = pool.map(_oracle_field, range(rounds * workers, (rounds + 1) * workers))
            dt = time.perf_counter() - t0
            if rounds == 0:
                _, loss, g_phi = res[0]
            rounds += 1
            if rounds > warmup:
                fields += workers
                t_total += dt
            if rounds >= warmup + max(1, steps) or time.perf_counter() - t_start > budget_s:
                if fields == 0:  # the budget ran out inside the warm-up: time the last round
                    fields, t_total = workers, dt
                break
    units = (4 + 2) / 2.0
    cb = {"value": units * fields / t_total, "unit": UNIT, "cores": workers, "kind": "oracle",
          "sample": f"{fields} of the workload's fields (object i, Ex, 450 nm), one per worker process at a time: "
                    "the full 4f chain in float64 numpy (4 forward + 2 backward propagations, 2048^2 FFTs) and "
                    f"the loss on that field's intensity; {t_total:.2f} s wall for them on {workers} cores"}
    if not want_sample:
        return cb
    import oracle as O
    obj = S.cfg4_objects(1, 1, n)[0, 0].astype(np.complex128)
    phase = S.cfg4_pupil_phase(n)
    target = S.cfg4_target(1, n)[0]
    lam = float(S.cfg4_wavelengths(c["wavelengths"])[0])
    fwd = O.propagate(obj[None], c["d"], c["d"], lam, c["f"], c["pad"])[0]
    bwd = O.propagate_adjoint(obj[None], c["d"], c["d"], lam, c["f"], c["pad"])[0]
    sample = dict(obj=obj, lam=lam, phase=phase, target=target, loss=float(loss), g_phi=g_phi, fwd=fwd, bwd=bwd)
    return cb, sample


def gpu_parity(dev, sample):
    """rel-L2 of the GPU path against the oracle's results on the sampled field: one AS propagation
    and its adjoint (the unit of the metric), and the 4f step's loss and pupil-phase gradient."""
    import torch
    from paper_2411_18591_gb300 import binding as Bd
    from paper_2411_18591_gb300.fourf import FourF
    c = S.CFG4
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    x = torch.from_numpy(sample["obj"].astype(np.complex64)[None]).to(dev)
    fwd = Bd.top_propagate(x, c["d"], c["d"], sample["lam"], c["f"], c["pad"]).cpu().numpy()[0]
    bwd = Bd.top_propagate_backward(x, c["d"], c["d"], sample["lam"], c["f"], c["pad"]).cpu().numpy()[0]
    one = FourF(n=c["n"], d=c["d"], f=c["f"], lens_radius=c["lens_radius"], pupil_radius=c["pupil_radius"],
                objects=1, comps=1, wavelengths=(sample["lam"],), pad=c["pad"])
    phase = torch.from_numpy(sample["phase"].astype(np.float32)).to(dev)
    target = torch.from_numpy(sample["target"].astype(np.float32)[None]).to(dev)
    gphase = torch.empty_like(phase)
    loss, _ = one.step(x, phase, target, gphase)
    torch.cuda.synchronize()
    return {"rel_l2_propagate": rel(fwd, sample["fwd"]), "rel_l2_propagate_backward": rel(bwd, sample["bwd"]),
            "rel_err_fourf_loss": abs(float(loss.item()) - sample["loss"]) / abs(sample["loss"]),
            "rel_l2_fourf_pupil_grad": rel(gphase.cpu().numpy().astype(np.float64), sample["g_phi"]),
            "sample": "object 0, Ex, 450 nm of the workload (1024^2, 2x padding) against the float64 oracle",
            "tolerance": 1e-5}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(args.steps, args.warmup, budget_s=150.0)  # rounds of one field per core
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 3.0 / cb["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(sample=True),
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(sample=False, objects=None):
    c = S.CFG4
    objects = c["objects"] if objects is None else objects
    return {"workload": "polarised 4f imaging, fwd+bwd w.r.t. pupil phase" + (" (oracle sample)" if sample else ""),
            "objects": objects, "components": c["comps"], "wavelengths": c["wavelengths"],
            "fields": objects * c["comps"] * c["wavelengths"], "grid": [c["n"], c["n"]], "spacing_m": c["d"],
            "pad": c["pad"], "fft": [2 * c["n"], 2 * c["n"]], "method": "angular spectrum", "focal_m": c["f"],
            "props_per_field": {"fwd": 4, "bwd": 2}, "l2": "inputs and intermediates (3.2 GB per plane) exceed L2"}


# ----------------------------------------------------------------------------- our arm

def context_paths(dev, c):
    """Per-field forward time of one 1024^2 AS propagation at 2x padding, three ways (context for
    the batched number, not part of it): the library batched (16 fields per call), the library
    unbatched (one field per call), and torch.fft (cuFFT) pad -> fft2 -> x H -> ifft2 -> crop as a
    reference path. Each is event-timed on the launching stream after warm-up; the 16 fields
    (128 MB, padded 512 MB) exceed L2."""
    import torch
    from paper_2411_18591_gb300 import binding as Bd
    n, d, lam, z, B = c["n"], c["d"], 532e-9, c["f"], 16
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.complex(torch.randn(B, n, n, generator=g), torch.randn(B, n, n, generator=g)).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    batched = timed(lambda: Bd.top_propagate(x, d, d, lam, z, 2.0, out=y), 5) / B
    unbatched = timed(lambda: [Bd.top_propagate(x[i], d, d, lam, z, 2.0, out=y[i]) for i in range(B)], 3) / B
    # cuFFT reference: H on the padded grid in float64, rounded to complex64 once
    P = 2 * n
    f = torch.fft.fftfreq(P, d=d, dtype=torch.float64, device=dev)
    rad = 1.0 / (lam * lam) - f[None, :] ** 2 - f[:, None] ** 2
    H = torch.where(rad >= 0, torch.exp(2j * math.pi * z * torch.sqrt(rad.clamp(min=0))),
                    torch.zeros((), dtype=torch.complex128, device=dev)).to(torch.complex64)
    buf = torch.zeros(B, P, P, dtype=torch.complex64, device=dev)
    o = n // 2

    def cufft():
        buf.zero_()
        buf[:, o:o + n, o:o + n] = x
        out = torch.fft.ifft2(torch.fft.fft2(buf) * H)
        y.copy_(out[:, o:o + n, o:o + n])

    ref = timed(cufft, 3) / B
    return {"fwd_ms_per_field_batched": batched, "fwd_ms_per_field_unbatched": unbatched,
            "fwd_ms_per_field_torch_fft": ref, "unbatched_over_batched": unbatched / batched,
            "torch_fft_over_batched": ref / batched,
            "note": "one 1024^2 AS forward propagation at 2x padding, 16 fields, event-timed; context only"}


def _event_ms(fn, reps, warm=2):
    """Mean milliseconds of fn() over reps runs on the current stream (CUDA events, after warm-up)."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def context_workloads(dev, peak_gbs, reps=5):
    """The other workloads' steps on their own, event-timed after warm-up, with the HBM fraction of
    their model bytes (context for the headline, not part of it):
    * large fields: one AS propagation forward + backward of a 2048^2 and of a 4096^2 field at 2x
      padding (the 4096^2 one is the large-field workload, 8192^2 transforms); model 160 n^2 B;
    * coherence: the 64^4 Gaussian Schell-model workload, P (M M* Gamma) P^H through the trainable
      mask, the intensity, its backward and the mask-phase gradient; compulsory bytes 4 x 134 MB
      (Gamma read and written once per direction);
    * Bluestein sizes: one AS forward propagation of 1021^2 fields at 2x padding (2042-point lines,
      4096-point chirp transforms), 4 fields a call; model 80 n^2 B per field;
    * the diffractive network: 64 fields of 512^2 through 5 phase masks, MSE and every mask's gradient
      (5 fwd + 5 bwd propagations a field); model 160 n^2 B per fwd+bwd pair;
    * the ragged batch: 200 fields of six sizes (250-1000^2) forward and backward in one call each;
      model 160 n^2 B per field."""
    import torch
    from paper_2411_18591_gb300 import binding as Bd
    out = {}
    g = torch.Generator(device="cpu").manual_seed(11)
    for n in (2048, 4096):
        x = torch.complex(torch.randn(1, n, n, generator=g), torch.randn(1, n, n, generator=g)).to(dev)
        ms = _event_ms(lambda: (Bd.top_propagate(x, 5e-6, 5e-6, 633e-9, 0.2, 2.0),
                                Bd.top_propagate_backward(x, 5e-6, 5e-6, 633e-9, 0.2, 2.0)), reps)
        gbs = 160.0 * n * n / (ms * 1e-3) / 1e9
        out[f"fwd_bwd_{n}"] = {"ms": ms, "model_bytes": 160 * n * n, "achieved_gbs": gbs, "frac": gbs / peak_gbs}
        del x
    c = S.cfg5a_coherence()
    gam = torch.from_numpy(c["gamma"]).to(dev)
    ph = torch.from_numpy(c["phase"]).to(dev)
    tgt = torch.from_numpy(c["target"]).to(dev)
    mask = Bd.Modulation(phase=ph)
    gp = torch.zeros_like(ph)

    def coherence_step():
        gz = Bd.top_propagate_coherence(gam, c["d"], c["d"], c["lam"], c["z"], c["pad"], mask=mask)
        inten = Bd.top_coherence_intensity(gz)
        _, gi = Bd.top_mse_loss(inten[None], tgt[None])
        G = Bd.top_coherence_intensity_backward(gi[0], gz)
        Bd.top_propagate_coherence_backward(G, c["d"], c["d"], c["lam"], c["z"], c["pad"], mask=mask, saved_in=gam,
                                            want_grad_in=False, grad_phase=gp)

    ms = _event_ms(coherence_step, reps)
    comp = 4 * gam.numel() * 8
    out["coherence_64_4"] = {"ms": ms, "compulsory_bytes": comp, "achieved_gbs": comp / (ms * 1e-3) / 1e9,
                             "frac": comp / (ms * 1e-3) / 1e9 / peak_gbs}
    n = 1021
    x = torch.complex(torch.randn(4, n, n, generator=g), torch.randn(4, n, n, generator=g)).to(dev)
    ms = _event_ms(lambda: Bd.top_propagate(x, 5e-6, 5e-6, 633e-9, 0.05, 2.0), reps) / 4
    gbs = 80.0 * n * n / (ms * 1e-3) / 1e9
    out["bluestein_1021_fwd_per_field"] = {"ms": ms, "model_bytes": 80 * n * n, "achieved_gbs": gbs,
                                           "frac": gbs / peak_gbs}
    del x
    # the diffractive network: 64 binary 512^2 inputs through 5 phase masks, MSE, every mask's gradient
    from paper_2411_18591_gb300.stack import MaskStack
    c2 = S.cfg2_diffractive()
    x2 = torch.from_numpy(c2["field"]).to(dev)
    ph2 = torch.from_numpy(c2["phases"]).to(dev)
    t2 = torch.from_numpy(c2["target"]).to(dev)
    K = ph2.shape[0]
    stack = MaskStack(c2["d"], c2["lam"], [c2["gap"]] * (K - 1) + [c2["detector"]], c2["pad"])

    def diffractive_step():
        inten, st = stack.forward(x2, ph2)
        _, gi = Bd.top_mse_loss(inten, t2)
        stack.backward(st, ph2, gi)

    ms = _event_ms(diffractive_step, reps)
    units = x2.shape[0] * K  # fwd+bwd propagation pairs per step
    n = x2.shape[-1]
    gbs = units * 160.0 * n * n / (ms * 1e-3) / 1e9
    out["diffractive_5x512"] = {"ms": ms, "fwd_bwd_per_s": units / (ms * 1e-3), "model_bytes": units * 160 * n * n,
                                "achieved_gbs": gbs, "frac": gbs / peak_gbs}
    del x2, t2
    # the ragged batch: 200 fields of six sizes with their own spacings, wavelengths and distances,
    # forward and backward in one call each (random fields of those shapes)
    descs = S.cfg3_ragged()
    xs = [torch.complex(torch.randn(f["n"], f["n"], generator=g), torch.randn(f["n"], f["n"], generator=g)).to(dev)
          for f in descs]
    outs = [torch.empty_like(v) for v in xs]
    sp, lm, zz = [f["d"] for f in descs], [f["lam"] for f in descs], [f["z"] for f in descs]
    ms = _event_ms(lambda: (Bd.top_propagate_ragged(xs, sp, lm, zz, 2.0, out=outs),
                            Bd.top_propagate_ragged(outs, sp, lm, zz, 2.0, backward=True, out=xs)), reps)
    model = sum(160 * f["n"] * f["n"] for f in descs)
    out["ragged_200"] = {"ms": ms, "fwd_bwd_per_s": len(descs) / (ms * 1e-3), "model_bytes": model,
                         "achieved_gbs": model / (ms * 1e-3) / 1e9, "frac": model / (ms * 1e-3) / 1e9 / peak_gbs}
    out["note"] = "event-timed after warm-up on the launching stream; fractions of the measured HBM copy bandwidth"
    return out


def run_ours(args, rank, world):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2411_18591_gb300 import binding as Bd
    from paper_2411_18591_gb300 import dist as D
    from paper_2411_18591_gb300.fourf import FourF

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = S.CFG4
    objects = args.objects
    sysm = FourF(n=c["n"], d=c["d"], f=c["f"], lens_radius=c["lens_radius"], pupil_radius=c["pupil_radius"],
                 objects=objects, comps=c["comps"], wavelengths=tuple(S.cfg4_wavelengths(c["wavelengths"])),
                 pad=c["pad"])
    # weak scaling: rank r takes objects [r K, (r + 1) K) of one seeded global set
    first = rank * objects
    obj_host = S.cfg4_objects(objects, c["comps"], c["n"], first=first).reshape(-1, c["n"], c["n"]).astype(np.complex64)
    obj_pinned = torch.from_numpy(obj_host).pin_memory()
    obj = obj_pinned.to(dev)
    phase = torch.from_numpy(S.cfg4_pupil_phase(c["n"]).astype(np.float32)).to(dev)
    target = torch.from_numpy(S.cfg4_target(objects, c["n"], first=first).astype(np.float32)).to(dev)
    gphase = torch.empty_like(phase)
    bufs = {}
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def step(x):
        loss, _ = sysm.step(x, phase, target, gphase, bufs)
        if dist:
            D.average_gradient(gphase)  # the one exchange of a step: mean pupil-phase gradient
        return loss

    # with --autotune, the pass variants measured on this geometry by the library's autotuner
    # (the defaults otherwise), then the warm-up
    tune_rows = tune_cols = None
    if args.autotune:
        tune_rows, tune_cols = Bd.top_autotune(16, c["n"], c["n"], c["d"], c["d"], c["pad"], device=dev)
    for _ in range(max(3, args.warmup)):
        step(obj)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(bus_id_of(local))

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    # device-resident timing of exactly K steps (library event timing off), with an event after
    # every step for the median step time
    barrier()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record(stream)
    for k in range(args.steps):
        step(obj)
        marks[k].record(stream)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    per_step = [e0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, args.steps)]
    ms_median = statistics.median(per_step)

    # the per-kernel split from a separate loop of the same steps with the library's CUDA-event
    # timing of every launch on the launching stream
    prof_steps = min(args.steps, 5)
    Bd.profile_enable(True, dev)
    Bd.profile_read(dev)
    for _ in range(prof_steps):
        step(obj)
    torch.cuda.synchronize()
    prof = Bd.profile_read(dev)
    Bd.profile_enable(False, dev)
    t = torch.tensor([ms], device=dev)
    if dist:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    ms = float(t.item())
    units_per_step = sysm.batch * (FourF.FWD_PROPS + FourF.BWD_PROPS) / 2.0
    value = units_per_step * world / (ms / 1000.0)

    # end to end: every step's inputs are copied from pinned host memory and its loss and
    # gradient read back, all inside the timed region; the copy of step k + 1's inputs runs on
    # a copy stream into the other of two input buffers while step k computes
    h2d = obj_pinned.numel() * 8
    host_g = torch.empty(phase.shape, dtype=torch.float32).pin_memory()
    host_l = torch.empty(1, dtype=torch.float64).pin_memory()
    xin = [torch.empty_like(obj), torch.empty_like(obj)]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]

    def stage_input(k):
        with torch.cuda.stream(copy_stream):
            xin[k % 2].copy_(obj_pinned, non_blocking=True)
            ready[k % 2].record(copy_stream)

    barrier()
    e0.record(stream)
    copy_stream.wait_event(e0)
    stage_input(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            if k >= 1:
                copy_stream.wait_event(free[(k + 1) % 2])  # step k - 1 is done with that buffer
            stage_input(k + 1)
        stream.wait_event(ready[k % 2])
        loss = step(xin[k % 2])
        free[k % 2].record(stream)
        host_l.copy_(loss.reshape(1), non_blocking=True)
        host_g.copy_(gphase, non_blocking=True)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    t = torch.tensor([ms_e2e], device=dev)
    if dist:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    ms_e2e = float(t.item())
    e2e = {"value": units_per_step * world / (ms_e2e / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(host_g.numel() * 4 + 8), "ms_per_step": ms_e2e,
           "note": "pinned host -> device copy of every step's objects on a copy stream (double-buffered, "
                   "step k + 1's copy overlaps step k), loss and gradient read back every step"}

    # roofline of the dominant kernel (the column pass), averaged over its launches in a step:
    # algorithmic bytes per step / column time per step. With u = Px ny 8 B (one field's
    # workspace): a column pass that starts from the workspace reads and writes it (2u per field);
    # the first forward propagation starts from the object broadcast over the wavelengths, so its
    # sources' spectra are made once (read u, write 2u per source) and every field's pass reads
    # its source's spectrum (2u once per source) and writes its workspace (u per field).
    peaks, peak_kind = measured_peaks()
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dominant = max(kinds, key=lambda k: kinds[k][0])
    cols_ms, cols_n = prof["cols"]
    u = (2 * c["n"]) * c["n"] * 8
    nsrc = sysm.batch // sysm.repeat
    full_passes = FourF.FWD_PROPS + FourF.BWD_PROPS - 1
    bytes_step = full_passes * sysm.batch * 2 * u + nsrc * 3 * u + nsrc * 2 * u + sysm.batch * u
    launches_step = cols_n / prof_steps
    cols_s_step = cols_ms / prof_steps / 1000.0
    achieved = bytes_step / cols_s_step / 1e9
    # ncu's DRAM bytes of a full column pass per field (workspace in and out, 2u algorithmic), as
    # bytes per algorithmic byte, times the algorithmic bytes of an average launch of the step
    traffic = profiled_traffic("cols")
    traffic_launch = None if traffic is None else traffic / (2 * u) * bytes_step / launches_step
    roofline = {"kernel": "cols (column pass: y-FFT x H x inverse y-FFT)", "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic_launch, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": bytes_step / launches_step,
                "avg_launch_ms": cols_s_step / launches_step * 1000.0,
                "algorithmic_bytes_per_step": bytes_step, "launches_per_step": launches_step,
                "traffic_note": "ncu dram bytes of a full column pass per field (profiles/cols_summary.md) per "
                                "algorithmic byte, times the algorithmic bytes of an average launch of the step",
                "dominant_by_time": dominant, "timing": f"CUDA events on the launching stream over {prof_steps} "
                "steps of a profiled loop after the timed one (the timed loop runs with the library's event timing off)",
                "kernel_ms_per_step": {k: v[0] / prof_steps for k, v in kinds.items()}}
    launches = int(round(sum(v[1] for v in prof.values()) / prof_steps * args.steps))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "ms_per_step_median": ms_median,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64/f32 (FP64 phase tables)", "data": "synthetic",
            "config": workload_config(objects=objects), "roofline": roofline, "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches,
            "autotune": None if tune_rows is None else {"rows_flags": tune_rows, "cols_flags": tune_cols,
                                                        "line_length": c["n"]}}
    if rank == 0 and world == 1 and not args.no_context:
        line["context"] = context_paths(dev, c)
        line["context"]["workloads"] = context_workloads(dev, peaks["hbm_gbs"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], sample = cpu_baseline(2, 1, want_sample=True)
        line["parity"] = gpu_parity(dev, sample)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the unbatched and torch.fft context timings")
    ap.add_argument("--context-only", action="store_true",
                    help="time only the other workloads (large fields, coherence, Bluestein sizes), --steps runs each")
    ap.add_argument("--autotune", action="store_true",
                    help="run the library's autotuner on the workload's geometry before the warm-up")
    ap.add_argument("--objects", type=int, default=S.CFG4["objects"],
                    help="objects per GPU (a smaller batch for profiler captures; the workload has 16)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)  # host-only; ranks other than 0 exit without work
        return
    if args.context_only:
        # the context workloads alone (for profiler captures of their kernels)
        import torch
        import __graft_entry__ as ge
        ge.build()
        peaks, _ = measured_peaks()
        print(json.dumps(context_workloads(torch.device("cuda", 0), peaks["hbm_gbs"], reps=args.steps)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
