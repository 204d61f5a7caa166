#!/usr/bin/env python
"""Throughput of the fluctuating two-species lattice Boltzmann update on GB300.

One "step" is one full lattice update (density pass + fused force, moment
collision, noise and streaming) of both species on the whole box.  Default
workload: D3Q19 256^3 periodic box, FP32 populations, rho_A = rho_B = 1,
G rho0 = 0.9, tau = 1, kT = 1e-5 (the 2.55 GB population array is far larger
than L2, so no flush is needed between steps).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead, on bounded samples of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU, weak scaling.
"""
from __future__ import annotations

import argparse
import glob
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

WORKLOADS = {
    "d3q19-256": dict(lattice=1, nx=256, ny=256, nz=256, storage="f32", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                      rho0=1.0, desc="D3Q19 256^3 periodic two-species Shan-Chen mixture, FP32 populations, "
                                     "rho_A=rho_B=1, G*rho0=0.9, tau=1.0, kT=1e-5"),
    "d3q19-256-f16": dict(lattice=1, nx=256, ny=256, nz=256, storage="f16", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                          rho0=1.0, desc="D3Q19 256^3 mixture, populations stored as FP16 deviations from "
                                         "w_i*rho0, FP32 collision"),
    "d3q19-256-bf16": dict(lattice=1, nx=256, ny=256, nz=256, storage="bf16", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                           rho0=1.0, desc="D3Q19 256^3 mixture, populations stored as BF16 deviations from "
                                          "w_i*rho0, FP32 collision"),
    "d3q19-128": dict(lattice=1, nx=128, ny=128, nz=128, storage="f32", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                      rho0=1.0, desc="D3Q19 128^3 mixture, FP32 (profiling case: 319 MB of populations, "
                                     "larger than L2)"),
    "d2q9-512": dict(lattice=0, nx=512, ny=512, nz=1, storage="f32", tau=(0.8, 1.0), kT=1e-5, G=0.9,
                     rho0=1.0, desc="D2Q9 512^2 periodic Shan-Chen mixture, FP32, G*rho0=0.9, tau=0.8/1.0, "
                                    "kT=1e-5 (fits in L2)"),
    "d2q9-4096": dict(lattice=0, nx=4096, ny=4096, nz=1, storage="f32", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                      rho0=1.0, desc="D2Q9 4096^2 periodic Shan-Chen mixture, FP32, G*rho0=0.9, tau=1.0, "
                                     "kT=1e-5 (as many sites as D3Q19 256^3; larger than L2)"),
    "d2q9-2048": dict(lattice=0, nx=2048, ny=2048, nz=1, storage="f32", tau=(1.0, 1.0), kT=1e-5, G=0.9,
                      rho0=1.0, desc="D2Q9 2048^2 mixture, FP32, tau=1.0 (profiling case: 302 MB of "
                                     "populations, larger than L2)"),
}
BYTES_PER_POP = {"f32": 4, "f16": 2, "bf16": 2}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="d3q19-256")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/BF16 storage and batching forms")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch settings")
    ap.add_argument("--schedule", choices=["fused", "two_kernels", "overlap", "tiled"], default=None,
                    help="force one step schedule (implies --no-autotune); fused with two arrays is the "
                         "pipelined step, fused in place the in-place persistent step")
    ap.add_argument("--streaming", choices=["two_arrays", "in_place"], default="two_arrays",
                    help="population streaming: two arrays (default) or one array updated in place")
    ap.add_argument("--form", choices=["species2", "species3", "species4"], default=None,
                    help="time only this N-species form (--steps steps on a --form-box^3 D3Q19 box) and print it")
    ap.add_argument("--form-box", type=int, default=256)
    ap.add_argument("--form-full", action="store_true", help="the N-species form with every tau 1 (moment-fed)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the files that define the step kernels (device code and the structures they
# take); the host runtime around them can change without touching the kernels
KERNEL_SOURCES = ("flbm_internal.h", "flbm_kernels.cuh", "flbm_lattice.cuh", "flbm_launch.h", "flbm_noise.cuh", "flbm_pair.cuh",
                  "flbm_transform.cuh", "inst_d*.cu")


def sources_digest():
    """sha256 over the kernel sources' code: comments and whitespace are left
    out, so that documentation edits keep a recorded capture valid."""
    import re

    h = hashlib.sha256()
    files = set()
    for pat in KERNEL_SOURCES:
        files.update(glob.glob(os.path.join(ROOT, "paper_1410_5584_gb300", "csrc", pat)))
    for p in sorted(files):
        with open(p, encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(os.path.basename(p).encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def recorded_capture(workload, sites, schedule=None):
    """DRAM bytes and executed warp-instructions per step (all of the step's
    kernels) from the committed ncu record, scaled to `sites`, if it was taken
    on the current kernel sources (and, when given, the same schedule); else
    None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    rec = d.get(workload)
    if not rec or rec.get("sources_sha256") != sources_digest():
        return None
    if schedule is not None and rec.get("schedule") != schedule:
        return None
    scale = sites / rec["sites"]
    inst = rec.get("warp_instructions_per_step")
    return {"traffic": rec["dram_bytes_per_step"] * scale, "inst": None if inst is None else inst * scale}


SMS, SCHEDULERS_PER_SM = 152, 4  # GB300: each scheduler issues at most one warp-instruction a cycle


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def storage_forms(wl, seed, steps, device):
    """The FP16 / BF16 deviation-storage forms beside the float run: MLUPS on the
    bench box, and their errors against the float-storage GPU run on a 32^3
    sub-case (densities, velocities, axis S(k) sampled along the same noise
    history, mass drift).  Errors against the FP64 oracle are measured by the
    test suite (tests/test_precision_gpu.py)."""
    import numpy as np
    import torch

    from paper_1410_5584_gb300 import Lattice
    from paper_1410_5584_gb300 import inputs

    out = {}
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    for st in ("f16", "bf16"):
        lat = Lattice(wl["lattice"], nx, ny, nz, wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"], seed,
                      storage=st, device=device, rho0_a=wl["rho0"], rho0_b=wl["rho0"])
        lat.init()
        lat.step(10)
        lat.sync()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(lat.stream)
        lat.step(steps)
        s1.record(lat.stream)
        lat.sync()
        out[st] = {"value": nx * ny * nz * steps / (s0.elapsed_time(s1) / 1e3) / 1e6, "unit": "MLUPS",
                   "steps": steps, "bytes_per_site": 2 * (19 if wl["lattice"] == 1 else 9) * 2 * 2}
        lat.close()
    # accuracy on a small box of the same lattice and parameters
    n3 = 32
    shape = (n3, n3, n3) if wl["lattice"] == 1 else (1, 256, 256)
    runs = {}
    for st in ("f32", "f16", "bf16"):
        lat = Lattice(wl["lattice"], shape[2], shape[1], shape[0], wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"],
                      seed, storage=st, device=device)
        lat.init(inputs.perturbed_density(shape, wl["rho0"], 1e-3, seed, 0),
                 inputs.perturbed_density(shape, wl["rho0"], 1e-3, seed, 1))
        c0 = lat.moments(fields=False)
        for _ in range(20):
            lat.step(10)
            lat.sf_sample()
        ra, rb, u, c1 = lat.moments()
        runs[st] = dict(ra=ra, rb=rb, u=u, drift=max(abs(c1[k] - c0[k]) / c0[k] for k in (0, 1)),
                        sk=np.stack(lat.structure_factor(0)[:3]))
        lat.close()
    ref = runs["f32"]
    for st in ("f16", "bf16"):
        r = runs[st]
        s_ref = ref["sk"][0] + ref["sk"][2]
        out[st]["error_vs_f32"] = {
            "case": f"{'x'.join(str(v) for v in shape[::-1])}, 200 steps, S(k) every 10",
            "rho_abs": float(max(np.max(np.abs(r["ra"] - ref["ra"])), np.max(np.abs(r["rb"] - ref["rb"])))),
            "u_rel": float(np.max(np.abs(r["u"] - ref["u"])) / np.max(np.abs(ref["u"]))),
            "sk_rel": float(np.max(np.abs(r["sk"][0] + r["sk"][2] - s_ref) / s_ref)),
            "mass_drift": float(r["drift"]), "mass_drift_f32": float(ref["drift"])}
    return out


def recorded_precision():
    """Errors of the FP32, FP16 and BF16 storage forms against the FP64
    oracle, from the committed record that tests/precision_vs_oracle.py
    writes on the GPU (profiles/precision_vs_oracle.json); None unless it was
    taken on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "precision_vs_oracle.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("sources_sha256") != sources_digest():
        return None
    return rec


def timed_step_form(wl, seed, steps, device, schedule=None, tune=False):
    """MLUPS of one workload's step (device-timed, CUDA events); tune: launch
    settings from flbm_autotune first (CUDA graphs for small boxes)."""
    import torch

    from paper_1410_5584_gb300 import Lattice
    from paper_1410_5584_gb300 import flbm as F

    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    lat = Lattice(wl["lattice"], nx, ny, nz, wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"], seed,
                  storage=wl["storage"], device=device, rho0_a=wl["rho0"], rho0_b=wl["rho0"])
    if schedule is not None:
        lat.set_option("schedule", F.SCHEDULE[schedule])
    lat.init()
    launch = lat.autotune(steps=200) if tune else None
    lat.step(10 + (launch or {}).get("graph_steps", 0) * 2)
    lat.sync()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(lat.stream)
    lat.step(steps)
    s1.record(lat.stream)
    lat.sync()
    t = s0.elapsed_time(s1) / 1e3
    lat.close()
    sites = nx * ny * nz
    q = 19 if wl["lattice"] == 1 else 9
    peak, _ = measured_peaks()
    bps = 2 * q * 2 * BYTES_PER_POP[wl["storage"]]
    return {"value": sites * steps / t / 1e6, "unit": "MLUPS", "steps": steps, "ms_per_step": t / steps * 1e3,
            "schedule": schedule or "default", "launch": launch, "workload": wl["desc"],
            "hbm": {"achieved": bps * sites * steps / t / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": bps * sites * steps / t / 1e9 / peak, "bytes_per_site": bps}}


def batched_form(seed, steps, device, nrep=64):
    """The batching form: nrep independent D2Q9 replicas, n_x and n_y drawn from
    {64, 128, 256, 512}, kT log-uniform in [1e-6, 1e-4], G rho0 uniform in
    [0, 0.9], distinct Philox keys, rho = 1, tau = 1, two arrays; every
    replica in one tiled launch a step, or in one density and one collide
    launch, replayed from CUDA graphs, as the autotuner picks.  Compared with
    the same replicas stepped as separate contexts, 5000 steps each (the
    batching workload's length)."""
    import torch

    from paper_1410_5584_gb300 import Batch, Lattice
    from paper_1410_5584_gb300 import inputs

    cfg = inputs.batch_replica_configs(nrep, seed)
    reps = [dict(nx=c["nx"], ny=c["ny"], tau_a=1.0, tau_b=1.0, kT=c["kT"], G=c["G"], seed=c["seed"]) for c in cfg]
    sites = sum(c["nx"] * c["ny"] for c in cfg)

    def timed(run, stream):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        s0.record(stream)
        run()
        s1.record(stream)
        torch.cuda.synchronize(device)
        return s0.elapsed_time(s1) / 1e3

    b = Batch(0, reps, device=device)
    b.init()
    tuned = b.autotune(steps=200)
    graph_steps = tuned["graph_steps"]
    b.step(2 * max(graph_steps, 1))
    b.sync()
    t_batch = timed(lambda: b.step(steps), b.stream)
    b.sync()
    ensemble = ensemble_structure_factor(b, cfg)
    b.close()
    stream = torch.cuda.Stream(device=device)
    lats = [Lattice(0, r["nx"], r["ny"], 1, 1.0, 1.0, r["kT"], r["G"], r["seed"], device=device, stream=stream)
            for r in reps]
    for g in lats:
        g.init()
        g.step(2)
    t_sep = timed(lambda: [g.step(steps) for g in lats], stream)
    for g in lats:
        g.sync()
        g.close()
    peak, _ = measured_peaks()
    ach = sites * steps * 2 * 9 * 4 * 2 / t_batch / 1e9
    return {"value": sites * steps / t_batch / 1e6, "unit": "MLUPS", "replicas": nrep, "sites": sites,
            "steps": steps, "graph_steps": graph_steps,
            "schedule": {1: "two_kernels", 3: "tiled"}.get(tuned["schedule"], tuned["schedule"]),
            "per_replica_launches_mlups": sites * steps / t_sep / 1e6,
            "speedup_vs_per_replica_launches": t_sep / t_batch,
            "hbm": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "bytes_per_site": 144},
            "ensemble_sk": ensemble}


def ensemble_structure_factor(b, cfg, burn=10000, nsnap=100, every=50):
    """Ensemble statistics of the batch from one submission: every replica's
    axis structure factor S_AA(k) sampled together (one flbm_sf_sample call
    per snapshot for all 64 replicas), divided by the continuum prediction of
    Eq. str-bin-hom at that replica's kT and G (rho0 = 1, alpha = G sin k/k),
    averaged over k bands per replica, then over replicas: mean and standard
    error over the replicas (independent runs).  Below k = 0.5 the continuum
    form and the lattice agree; above it the lattice corrections of the
    update show as a departure from 1.  The burn-in covers the slowest
    relaxation in the ensemble (inter-diffusion at k = 2 pi / 512 slowed by
    1 - (G rho0)^2 near G rho0 = 0.9: a few thousand steps)."""
    import numpy as np

    b.step(burn)
    for _ in range(nsnap):
        b.step(every)
        b.sf_sample()
    b.sync()
    bands = [(0.0, 0.5), (0.5, 1.0), (1.0, 2.0), (2.0, np.pi + 1e-9)]
    per = [[] for _ in bands]
    for k, c in enumerate(cfg):
        s_aa = np.asarray(b.replicas[k].structure_factor(0)[0])
        n = c["nx"]
        kk = 2 * np.pi * np.arange(1, len(s_aa) + 1) / n
        alpha = c["G"] * np.sinc(kk / np.pi)
        pred = 3.0 * c["kT"] / (1.0 - alpha ** 2)
        er = s_aa / pred
        for q, (lo, hi) in enumerate(bands):
            sel = (kk >= lo) & (kk < hi)
            if sel.any():
                per[q].append(float(er[sel].mean()))
    out = {"snapshots": nsnap, "every": every, "burn_in": burn, "quantity": "S_AA(k) / (3 kT / (1 - (G sin k / k)^2))"}
    for (lo, hi), vals in zip(bands, per):
        v = np.array(vals)
        out[f"k_{lo:.1f}_{min(hi, np.pi):.2f}"] = {"mean": float(v.mean()), "se": float(v.std(ddof=1) / np.sqrt(len(v))),
                                                   "replicas": len(v)}
    return out


def capillary_form(seed, device, steps=20000):
    """The capillary-fluctuation workload of Sec. VI B: a D2Q9 100 x 512 box
    with an A-rich stripe 50 wide (G = 1.5, kT = 1e-5, all rates 1): MLUPS of a
    lone context launching each step, of the same context replaying 64-step
    CUDA graphs, and of the box as a one-replica batch replayed from graphs
    (51,200 sites are too few to hide launch latency), and the time of one
    tracked height-spectrum snapshot."""
    import numpy as np
    import torch

    from paper_1410_5584_gb300 import Batch, Lattice

    nx, ny = 100, 512
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    phi = 0.25 * (1 + np.tanh((x - 25) / 2.0)) * (1 - np.tanh((x - 75) / 2.0))
    ra, rb = (0.06 + 2.24 * phi).ravel(), (0.06 + 2.24 * (1 - phi)).ravel()

    def timed(run, stream):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        s0.record(stream)
        run()
        s1.record(stream)
        torch.cuda.synchronize(device)
        return s0.elapsed_time(s1) / 1e3

    g = Lattice(0, nx, ny, 1, 1.0, 1.0, 1e-5, 1.5, seed, device=device, rho0_a=1.18, rho0_b=1.18)
    g.init(ra, rb)
    g.step(2000)
    t_lone = timed(lambda: g.step(steps), g.stream)
    g.set_option("graph_steps", 64)
    g.step(128)
    t_graph = timed(lambda: g.step(steps), g.stream)
    g.set_option("graph_steps", 0)
    g.cap_sample(-1, -1)
    t_cap = timed(lambda: [g.cap_sample(-1, -1) for _ in range(100)], g.stream) / 100
    g.sync()
    b = Batch(0, [dict(nx=nx, ny=ny, tau_a=1.0, tau_b=1.0, kT=1e-5, G=1.5, seed=seed, rho0_a=1.18, rho0_b=1.18)],
              device=device)
    b.init(ra, rb)
    tuned = b.autotune(steps=2000)
    graph_steps = tuned["graph_steps"]
    b.step(2000)
    t_batch = timed(lambda: b.step(steps), b.stream)
    b.sync()
    b.close()
    sites = nx * ny
    return {"unit": "MLUPS", "sites": sites, "steps": steps, "lone_context": sites * steps / t_lone / 1e6,
            "lone_context_graphs_64": sites * steps / t_graph / 1e6,
            "one_replica_batch": sites * steps / t_batch / 1e6, "graph_steps": graph_steps,
            "batch_schedule": {1: "two_kernels", 3: "tiled"}.get(tuned["schedule"], tuned["schedule"]),
            "ms_per_height_snapshot": t_cap * 1e3}


def multi_form(seed, device, steps=100, n=256, ns=3, full=False):
    """The N-species form (App. C-D): a D3Q19 n^3 box of three species, rho =
    (1, 0.8, 0.6), tau = (1, 0.8, 1.25) (full: every tau 1, the moment-fed
    pair), G = 0.3 between every pair, kT = 1e-5: GLUPS of the whole step and
    its achieved bandwidth on the algorithmic bytes (every population read and
    written once) against the measured HBM copy rate, and each kernel's
    bandwidth on the bytes it moves by design."""
    import numpy as np
    import torch

    from paper_1410_5584_gb300 import MultiLattice
    from paper_1410_5584_gb300 import flbm as F

    rhos = [1.0, 0.8, 0.6, 0.9][:ns]
    taus = [1.0] * ns if full else [1.0, 0.8, 1.25, 0.9][:ns]
    G = 0.3 * (1 - np.eye(ns))
    g = MultiLattice(1, ns, n, n, n, taus, 1e-5, G, seed, rho0=rhos, device=device)
    g.init()
    g.step(5)
    g.sync()
    g.set_option(F.OPT_KERNEL_TIMING, 1)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(g.stream)
    g.step(steps)
    s1.record(g.stream)
    g.sync()
    t = s0.elapsed_time(s1) / 1e3
    ms, launches = g.kernel_times()
    g.close()
    sites = n ** 3
    q, d = 19, 3
    pops = ns * q * 4
    mom = ns * (d + 1) * 4 if full else 0  # the moment planes of the moment-fed pair
    collide_bytes = sites * ((mom if full else pops) + 16 + pops)
    density_bytes = sites * (pops + 16 + mom)
    peak, kind = measured_peaks()
    t_col = ms["collide"] / 1e3 / launches["collide"]
    t_den = ms["density"] / 1e3 / launches["density"]
    step_gbs = sites * 2 * pops * steps / t / 1e9
    return {"value": sites * steps / t / 1e9, "unit": "GLUPS", "species": ns, "box": f"{n}^3 D3Q19",
            "tau": taus, "moment_fed": full, "steps": steps, "ms_density": t_den * 1e3, "ms_collide": t_col * 1e3,
            "hbm": {"achieved": step_gbs, "peak": peak, "unit": "GB/s", "frac": step_gbs / peak,
                    "bytes_per_site": 2 * pops, "peak_kind": kind},
            "roofline_collide": {"bound": "hbm", "achieved": collide_bytes / t_col / 1e9, "peak": peak,
                                 "unit": "GB/s", "frac": collide_bytes / t_col / 1e9 / peak, "peak_kind": kind,
                                 "bytes_per_site": collide_bytes // sites},
            "density_gbs": density_bytes / t_den / 1e9}


def cpu_baseline(wl, seed, budget_s=15.0):
    """The FP64 oracle as it stands, on a bounded sample (the same lattice and
    parameters on a smaller periodic box): single-threaded, and beside it the
    same loop split over every host core (`all_cores`)."""
    import numpy as np

    import oracle

    side = 64 if wl["lattice"] == 1 else 512
    shape = (side, side, side) if wl["lattice"] == 1 else (1, side, side)
    nz, ny, nx = shape
    sites = nx * ny * nz

    def timed(threads, budget):
        o = oracle.Oracle(wl["lattice"], nx, ny, nz, wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"], seed)
        o.set_threads(threads)
        o.init(np.full(sites, wl["rho0"]), np.full(sites, wl["rho0"]))
        t0 = time.perf_counter()
        o.step(1)
        dt1 = time.perf_counter() - t0
        n = max(1, min(50, int(budget / max(dt1, 1e-6)) - 1))
        t0 = time.perf_counter()
        o.step(n)
        dt = time.perf_counter() - t0
        o.close()
        return sites * n / dt / 1e6, n

    lat = "D3Q19" if wl["lattice"] == 1 else "D2Q9"
    v1, n1 = timed(1, budget_s)
    cores = os.cpu_count() or 1
    vall, nall = timed(cores, budget_s / 2)
    return {"value": v1, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{lat} {nx}x{ny}x{nz} periodic box, same tau/kT/G/rho0, {n1} steps timed after 1, FP64, 1 thread",
            "all_cores": {"value": vall, "unit": "MLUPS", "cores": cores,
                          "sample": f"the same box, {nall} steps timed after 1, sites split over {cores} threads"}}


def run_reference(args, wl):
    """--impl reference: the FP64 oracle on the host cores; each step is one
    oracle step on a small periodic box of the same workload, sized so the
    whole run stays within a few minutes."""
    import numpy as np

    import oracle

    world, rank, _ = dist_env()
    if rank != 0:
        return
    lat = wl["lattice"]

    def make(side):
        shape = (side, side, side) if lat == 1 else (1, side, side)
        nz, ny, nx = shape
        o = oracle.Oracle(lat, nx, ny, nz, wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"], args.seed)
        o.set_threads(1)
        o.init(np.full(nx * ny * nz, wl["rho0"]), np.full(nx * ny * nz, wl["rho0"]))
        return o, nx * ny * nz, shape

    o, sites, _ = make(8 if lat == 1 else 32)
    t0 = time.perf_counter()
    o.step(2)
    rate = 2 * sites / (time.perf_counter() - t0)
    o.close()
    budget = 150.0
    side = 4 if lat == 1 else 8
    for cand in range(4, 257):
        if (cand ** 3 if lat == 1 else cand * cand) * (args.steps + args.warmup) / rate <= budget:
            side = cand
    o, sites, shape = make(side)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    o.close()
    value = sites * args.steps / dt / 1e6
    sample = (f"{'D3Q19' if lat == 1 else 'D2Q9'} {shape[2]}x{shape[1]}x{shape[0]} periodic box per step "
              f"(same tau/kT/G/rho0), FP64, 1 thread")
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "reference_sample": sample},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, wl):
    import numpy as np
    import torch

    from paper_1410_5584_gb300 import Lattice
    from paper_1410_5584_gb300.replicas import aggregate, replica_seed

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    seed = replica_seed(args.seed, rank)
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    sites = nx * ny * nz
    Q = 19 if wl["lattice"] == 1 else 9
    from paper_1410_5584_gb300 import flbm as F
    streaming = args.streaming
    lat = Lattice(wl["lattice"], nx, ny, nz, wl["tau"][0], wl["tau"][1], wl["kT"], wl["G"], seed,
                  storage=wl["storage"], device=device, rho0_a=wl["rho0"], rho0_b=wl["rho0"],
                  streaming=F.STREAMING[streaming])
    lat.init()
    # launch settings from the autotuner (untimed; the state is left as it was)
    launch = None
    if args.schedule:
        lat.set_option("schedule", F.SCHEDULE[args.schedule])
        launch = {"schedule": F.SCHEDULE[args.schedule]}
    elif not args.no_autotune:
        launch = lat.autotune(steps=20)
    lat.step(args.warmup)
    # with CUDA graphs, one untimed call of a graph's length captures the graph
    # the timed steps replay (graphs are kept per starting parity; an even
    # length leaves the parity as it was), so no capture is timed
    capture_steps = int(lat.get_option("graph_steps"))
    if capture_steps > 0:
        lat.step(capture_steps + capture_steps % 2)
    lat.sync()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-timed region: inputs resident in HBM, the launch settings as
    # tuned (CUDA graphs included), no per-kernel events ----
    def timed_region():
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(device)
        start.record(lat.stream)
        lat.step(args.steps)
        end.record(lat.stream)
        torch.cuda.synchronize(device)
        barrier()
        lat.sync()
        return aggregate(start.elapsed_time(end) / 1e3, sites * args.steps, device=device)

    with ClockSampler(local) as clk:
        t_max, units = timed_region()
        # the same region five times more: their median beside the reported one
        rep_s = [timed_region()[0] for _ in range(5)]
    value = units / t_max / 1e6
    repeats = {"n": len(rep_s), "median_ms_per_step": statistics.median(rep_s) / args.steps * 1e3,
               "min_ms_per_step": min(rep_s) / args.steps * 1e3, "max_ms_per_step": max(rep_s) / args.steps * 1e3,
               "median_value": units / statistics.median(rep_s) / 1e6}
    # per-kernel times and launch counts: K more steps with CUDA events around
    # each kernel (launched directly: graphs are replayed only without them)
    lat.set_option("kernel_timing", 1)
    lat.step(args.steps)
    lat.sync()
    kms, kn = lat.kernel_times()
    lat.set_option("kernel_timing", 0)

    # ---- end to end through the C-ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        ra = np.full(sites, wl["rho0"])
        rb = np.full(sites, wl["rho0"])
        out_a, out_b = np.empty(sites), np.empty(sites)
        D = 3 if wl["lattice"] == 1 else 2
        out_u = np.empty(D * sites)
        import ctypes

        from paper_1410_5584_gb300 import flbm as F
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cons = np.empty(5)
        barrier()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        F.check(lat._h, F.lib().flbm_init(lat._h, dp(ra), dp(rb)))
        F.check(lat._h, F.lib().flbm_step(lat._h, args.steps))
        F.check(lat._h, F.lib().flbm_moments(lat._h, dp(out_a), dp(out_b), dp(out_u), dp(cons)))
        t1 = time.perf_counter()
        barrier()
        te, ue = aggregate(t1 - t0, sites * args.steps, device=device)
        # the two density planes: read as doubles by a kernel straight from the
        # caller's arrays where the GPU shares the host's page tables, else
        # converted to float on the host and copied from pinned staging
        direct = lat.get_option("direct_host") == 1
        h2d = 2 * sites * (8 if direct else 4)
        d2h = (2 + D) * sites * 8 + 5 * 8
        e2e = {"value": ue / te / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "route": "direct (kernels read and write the caller's pageable arrays)" if direct
               else "pinned staging",
               "note": "flbm_init from host densities + K steps + flbm_moments to host, per-step averages"}

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    bpp = BYTES_PER_POP[wl["storage"]]
    D = 3 if wl["lattice"] == 1 else 2
    sched = (launch or {}).get("schedule", F.SCHEDULE["two_kernels"])
    # the pipelined step: the fused schedule with two arrays (one launch a step)
    pipelined = streaming == "two_arrays" and sched == F.SCHEDULE["fused"] and kn["density"] == 0
    # the tiled step of a 2D box (one launch a step, densities in shared memory)
    tiled = streaming == "two_arrays" and sched == F.SCHEDULE["tiled"] and kn["density"] == 0
    one_launch = pipelined or tiled
    one_name = "k_step_pipe" if pipelined else "k_step_tiled"
    full = all(t == 1.0 for t in wl["tau"])
    moment_fed = streaming == "two_arrays" and full and sched == F.SCHEDULE["two_kernels"]
    # Algorithmic bytes of one site update (every population of both species
    # read once and written once), the roofline's numerator for the whole step
    alg_site = 2 * Q * 2 * bpp
    step_s = t_max / args.steps
    achieved = alg_site * sites / step_s / 1e9
    # the bytes the implementation moves by design: the pipelined step keeps
    # its densities and moments in an L2-resident ring, the tiled step in shared
    # memory (its ring of neighbouring sites is read again from L2); the
    # two-kernel step re-reads the populations for the densities (moment-fed:
    # the collide reads m_0 .. m_D and rho instead of the populations)
    if one_launch:
        design = alg_site
    elif moment_fed:
        design = alg_site + 2 * (2 * (D + 1) * 4 + 8)
    else:
        design = alg_site + 2 * Q * bpp + 8 + 8
    cap = recorded_capture(args.workload, sites, "pipelined" if pipelined else "tiled" if tiled else "two_kernels")
    traffic = cap["traffic"] if cap else None
    clocks = clk.summary()
    coll_ms = kms["collide"] / max(kn["collide"], 1)
    den_ms = kms["density"] / max(kn["density"], 1) if kn["density"] else 0.0
    roofline = {"bound": "hbm", "kernel": one_name + " (one launch a step)" if one_launch
                else "whole step (density pass + k_collide)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes_per_site": alg_site, "algorithmic_bytes_per_launch": alg_site * sites,
                "launches_per_step": 1 if one_launch else 2, "design_bytes_per_site": design,
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    kernels = {"collide" if not one_launch else one_name: {"ms": coll_ms}}
    if not one_launch:
        coll_bytes = (2 * (D + 1) * 4 + 8 if moment_fed else 2 * Q * bpp + 8) + 2 * Q * bpp
        den_bytes = 2 * Q * bpp + 8 + (2 * (D + 1) * 4 if moment_fed else 0)
        kernels["collide"].update(bytes_per_site=coll_bytes, gbs=coll_bytes * sites / (coll_ms / 1e3) / 1e9)
        kernels["density"] = {"ms": den_ms, "bytes_per_site": den_bytes,
                              "gbs": den_bytes * sites / (den_ms / 1e3) / 1e9 if den_ms else None}
    if cap and cap.get("inst"):
        # issue view of the step's kernels: executed warp-instructions per step
        # (the recorded ncu count, scaled by the site count) over the event-timed
        # kernel time, against one warp-instruction per scheduler per cycle
        mhz = clocks["sm_mhz"] if clocks else 2070.0
        issue_peak = SMS * SCHEDULERS_PER_SM * mhz * 1e6 / 1e9
        ach_i = cap["inst"] / ((coll_ms + den_ms) / 1e3) / 1e9
        roofline["issue"] = {"achieved": ach_i, "peak": issue_peak, "unit": "G warp-instructions/s",
                             "frac": ach_i / issue_peak, "instructions_per_step": cap["inst"],
                             "source": "ncu smsp__inst_executed of a recorded capture on the current kernel "
                                       "sources, scaled by the site count; peak at the median SM clock sampled "
                                       f"during the run ({mhz:.0f} MHz)"}
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "lattice": "D3Q19" if wl["lattice"] == 1 else "D2Q9",
                   "nx": nx, "ny": ny, "nz": nz, "storage": wl["storage"], "replicas": world,
                   "l2": "inputs larger than L2" if sites * 2 * Q * bpp > 129e6 else "working set fits in L2",
                   "launch": launch, "streaming": streaming,
                   "untimed_graph_capture_steps": capture_steps + capture_steps % 2 if capture_steps > 0 else 0},
        "roofline": roofline,
        "step_hbm_frac": achieved / peak,
        "step_bytes_per_site": alg_site,
        "kernels": kernels,
        "kernel_ms": {"density": den_ms, "collide": coll_ms},
        "gpu_launches": kn["density"] + kn["collide"],
        "repeats": repeats,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_forms:
        # one full-wavevector structure-factor snapshot on the bench box (observables,
        # packing, three axes of line FFTs, FP64 accumulation), event-timed
        lat.sfk_sample()
        lat.sync()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(lat.stream)
        for _ in range(5):
            lat.sfk_sample()
        s1.record(lat.stream)
        lat.sync()
        sfk_ms = s0.elapsed_time(s1) / 5
        lat.sfk_reset()
        line["sk_full"] = {"ms_per_snapshot": sfk_ms, "sites": sites,
                           "note": "S_aa, S_ab, S_bb at every wavevector: fluctuation fields, float line FFTs, FP64 sums"}
    if not args.no_forms and wl["storage"] == "f32":
        line["forms"] = storage_forms(wl, args.seed, max(50, args.steps // 4), device)
        prec = recorded_precision()
        for st in ("f16", "bf16"):
            line["forms"][st]["error_vs_oracle"] = prec["forms"][st] if prec else None
        line["forms"]["f32_error_vs_oracle"] = prec["forms"]["f32"] if prec else None
        if prec:
            line["forms"]["error_vs_oracle_case"] = prec["case"]
        line["forms"]["general_tau"] = timed_step_form(
            dict(wl, tau=(0.8, 1.0), desc=wl["desc"].replace("tau=1.0", "tau=0.8/1.0")), args.seed,
            max(50, args.steps // 4), device, schedule=args.schedule)
        line["forms"]["d2q9_512"] = timed_step_form(WORKLOADS["d2q9-512"], args.seed, 5000, device, tune=True)
        line["forms"]["d2q9_4096"] = timed_step_form(WORKLOADS["d2q9-4096"], args.seed, 200, device, tune=True)
        line["forms"]["batched"] = batched_form(args.seed, 5000, device)
        line["forms"]["capillary"] = capillary_form(args.seed, device)
        line["forms"]["species3"] = multi_form(args.seed, device)
        line["forms"]["species3_full"] = multi_form(args.seed, device, full=True)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.seed)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.form:
        print(json.dumps(multi_form(args.seed, "cuda:0", steps=args.steps, n=args.form_box, ns=int(args.form[-1]),
                                    full=args.form_full)))
        return
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)
    world, _, _ = dist_env()
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
